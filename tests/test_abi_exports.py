"""The C-ABI library builds, loads without a GPU and exports every declared call."""
import ctypes
import os
import re

import pytest

from paper_2301_06503_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(lgdm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build()
    return ctypes.CDLL(_lib.LIB_PATH)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 19
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol():
    assert set(_declared()) == set(_lib.abi_names())


def test_loads_and_reports_version_without_gpu(lib):
    L = _lib.load()
    assert L.lgdm_abi_version() == _lib.ABI_VERSION == 2
    assert L.lgdm_status_string(4) == b"Newton did not converge"
    o = _lib.Options()
    assert L.lgdm_default_options(ctypes.byref(o)) == 0
    assert o.max_newton == 50 and o.newton_tol == 1e-8 and o.wait_limit_s == 2.0


def test_workspace_size_host_only(lib):
    """Sizing runs on the host: pattern counting needs no device."""
    import lgdm_inputs as li
    from paper_2301_06503_gb300 import sim
    p = li.sen_plate_problem(8, 6)
    n = sim.workspace_bytes(p.mesh)
    nd, nnode = 3, 9 * 7
    pairs = (3 * 9 - 2) * (3 * 7 - 2)            # node pairs of a structured quad grid
    assert n > nd * nd * pairs * 8               # at least the CSR values
    bad = li.sen_plate_problem(4, 4).mesh
    bad.conn = bad.conn.copy()
    bad.conn[0, 0] = 10_000
    with pytest.raises(_lib.LgdmError):
        sim.workspace_bytes(bad)
