"""lgdm_solve_noalloc: the solve for callers that cannot allocate device memory.

The entry point takes its working storage from a statically reserved device
array instead of a caller workspace.  It must give the same solution as the
workspace-based lgdm_solve on the same system, on consecutive calls (the
array keeps the previous call's contents), and refuse systems too large for
the array without touching device memory.  This file is collected last so
that a stopping run has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import lgdm_inputs as li

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _node_pattern(rowptr, col, nd, nnode):
    """Neighbour lists of the node-block CSR returned by lgdm_get_system."""
    ptr = np.zeros(nnode + 1, np.int32)
    nbr = []
    for a in range(nnode):
        cols = col[rowptr[nd * a]:rowptr[nd * a + 1]]
        nodes = cols[::nd] // nd
        nbr.append(nodes)
        ptr[a + 1] = ptr[a] + len(nodes)
    return ptr, np.concatenate(nbr).astype(np.int32)


def _state(p, seed):
    u, _ = li.random_state(p.mesh, seed=seed, kappa0=p.material.kappa0, strain=2e-5)
    return u, np.full(p.mesh.nel * p.mesh.ngp, 1.0)     # undamaged: a well-conditioned system


def test_noalloc_solve_matches_workspace_solve_twice():
    from paper_2301_06503_gb300 import Sim, _lib
    lib = _lib.load()
    p = li.sen_plate_problem(30, 20)
    s = Sim(p.mesh, p.material, p.bcs, krylov_rtol=1e-12)
    stream = torch.cuda.current_stream()
    for seed in (31, 32):                                  # two calls in a row, different systems
        u, kh = _state(p, seed)
        s.set_state(u, kh)
        s.assemble()
        rowptr, col, vals, rhs = s.system()
        s.solve()
        x_ref = s.field("delta")
        ptr, nbr = _node_pattern(rowptr, col, s.nd, p.mesh.nnode)
        d_ptr = torch.from_numpy(ptr).cuda()
        d_nbr = torch.from_numpy(nbr).cuda()
        d_vals = torch.from_numpy(vals).cuda()
        d_rhs = torch.from_numpy(rhs).cuda()
        d_x = torch.full((s.ndof,), float("nan"), dtype=torch.float64, device="cuda")
        it, rel = C.c_int32(), C.c_double()
        st = lib.lgdm_solve_noalloc(s.nd, p.mesh.nnode, d_ptr.data_ptr(), d_nbr.data_ptr(), d_vals.data_ptr(),
                                    d_rhs.data_ptr(), d_x.data_ptr(), 1e-12, 5000, stream.cuda_stream,
                                    C.byref(it), C.byref(rel))
        assert st == 0, lib.lgdm_last_error(None)
        assert rel.value <= 1e-12 and it.value > 0
        x = d_x.cpu().numpy()
        assert np.abs(x - x_ref).max() <= 1e-10 * np.abs(x_ref).max()
    s.close()


def test_noalloc_rejects_oversize_system():
    from paper_2301_06503_gb300 import _lib
    lib = _lib.load()
    d = torch.zeros(16, dtype=torch.float64, device="cuda")
    i = torch.zeros(16, dtype=torch.int32, device="cuda")
    it, rel = C.c_int32(), C.c_double()
    # 4 million nodes x 3 dofs need far more than the static array: refused before any launch
    st = lib.lgdm_solve_noalloc(3, 4_000_000, i.data_ptr(), i.data_ptr(), d.data_ptr(), d.data_ptr(),
                                d.data_ptr(), 1e-8, 10, torch.cuda.current_stream().cuda_stream,
                                C.byref(it), C.byref(rel))
    assert st == 2                                          # LGDM_ERR_OOM
    assert b"static array" in lib.lgdm_last_error(None)
