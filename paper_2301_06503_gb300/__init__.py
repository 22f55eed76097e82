"""GB300 (sm_103a) implementation of the localizing gradient damage method hot path.

The compute lives in ``liblgdm.so`` (CUDA C++ behind the C ABI declared in
``include/lgdm.h``); this package only builds it, declares its functions and
marshals arguments.  Importing the package does not load the library; the
first ``Sim`` does, and raises if the library has not been built.
"""
from . import _lib
from .build import build

__all__ = ["build", "Sim", "Batch", "workspace_bytes", "make_options", "_lib"]


def __getattr__(name):
    if name in ("Sim", "workspace_bytes", "make_options"):
        from . import sim
        return getattr(sim, name)
    if name == "Batch":
        from . import batch
        return batch.Batch
    raise AttributeError(name)
