"""Python handle over an LGDM batch: several simulations advanced together.

Marshalling only: the members are ``Sim`` handles created on the same CUDA
stream with the same precision; the batch workspace comes from PyTorch.
"""
import ctypes as C

import numpy as np
import torch

from . import _lib as L


class Batch:
    def __init__(self, sims):
        if not sims:
            raise ValueError("empty batch")
        lib = L.load()
        self._lib = lib
        self.sims = list(sims)
        self.n = len(self.sims)
        self.h = None
        n = C.c_size_t()
        L.check(lib.lgdm_batch_workspace_size(self.n, C.byref(n)))
        self.stream = self.sims[0].stream
        self.workspace = torch.empty(int(n.value), dtype=torch.uint8, device=self.sims[0].device)
        arr = (C.c_void_p * self.n)(*[s.h.value for s in self.sims])
        h = C.c_void_p()
        L.check(lib.lgdm_batch_create(arr, self.n, C.c_void_p(self.workspace.data_ptr()), int(n.value),
                                      C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h

    def close(self):
        if self.h is not None:
            torch.cuda.synchronize(self.sims[0].device)
            self._lib.lgdm_batch_destroy(self.h)
            self.h = None
            self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st):
        if st != 0:
            msg = self._lib.lgdm_batch_last_error(self.h)
            raise L.LgdmError(st, msg.decode() if msg else "")

    def set_tuning(self, block_threads=128, grid_factor=2, graph=True):
        self._ck(self._lib.lgdm_batch_set_tuning(self.h, block_threads, grid_factor, 1 if graph else 0))

    def tuning(self):
        bt, gf, g = C.c_int32(), C.c_int32(), C.c_int32()
        self._ck(self._lib.lgdm_batch_get_tuning(self.h, C.byref(bt), C.byref(gf), C.byref(g)))
        return {"block_threads": bt.value, "grid_factor": gf.value, "graph": int(g.value)}

    def set_solve_tuning(self, nodes_per_block=4096):
        self._ck(self._lib.lgdm_batch_set_solve_tuning(self.h, int(nodes_per_block)))

    def solve_tuning(self):
        npb, w = C.c_int32(), C.c_int32()
        self._ck(self._lib.lgdm_batch_get_solve_tuning(self.h, C.byref(npb), C.byref(w)))
        return {"nodes_per_block": npb.value, "waves": w.value}

    def launches(self):
        """Kernels issued by the batched passes since creation."""
        n = C.c_int64()
        self._ck(self._lib.lgdm_batch_get_launches(self.h, C.byref(n)))
        return int(n.value)

    def autotune(self):
        bt, gf, ms = C.c_int32(), C.c_int32(), C.c_double()
        self._ck(self._lib.lgdm_batch_autotune(self.h, C.byref(bt), C.byref(gf), C.byref(ms)))
        return {"block_threads": bt.value, "grid_factor": gf.value, "assembly_ms": ms.value}

    def _flags(self, active):
        a = np.ones(self.n, np.int32) if active is None else np.ascontiguousarray(active, dtype=np.int32)
        return a, a.ctypes.data_as(C.POINTER(C.c_int32))

    def assemble(self, active=None):
        a, pa = self._flags(active)
        self._ck(self._lib.lgdm_batch_assemble(self.h, pa))

    def newton_step(self, active=None):
        a, pa = self._flags(active)
        conv = np.zeros(self.n, np.int32)
        its = np.zeros(self.n, np.int32)
        self._ck(self._lib.lgdm_batch_newton_step(self.h, pa, conv.ctypes.data_as(C.POINTER(C.c_int32)),
                                                  its.ctypes.data_as(C.POINTER(C.c_int32))))
        return conv, its

    def run_step(self, loads):
        """Advance every member one load step (NaN = sit out); returns (newton_iters, status)."""
        ld = np.ascontiguousarray(loads, dtype=np.float64)
        its = np.zeros(self.n, np.int32)
        st = np.zeros(self.n, np.int32)
        self._ck(self._lib.lgdm_batch_run_step(self.h, ld.ctypes.data_as(C.POINTER(C.c_double)),
                                               its.ctypes.data_as(C.POINTER(C.c_int32)),
                                               st.ctypes.data_as(C.POINTER(C.c_int32))))
        return its, st

    PHASES = ("element", "gather", "precond", "krylov")

    def enable_timers(self, on=True):
        self._ck(self._lib.lgdm_batch_enable_timers(self.h, 1 if on else 0))

    def timers(self, reset=False):
        """{phase: (milliseconds, timed Newton steps)} for element, gather, precond, krylov."""
        ms = (C.c_double * 4)()
        n = (C.c_int64 * 4)()
        self._ck(self._lib.lgdm_batch_get_timers(self.h, ms, n, 1 if reset else 0))
        return {k: (ms[i], n[i]) for i, k in enumerate(self.PHASES)}
