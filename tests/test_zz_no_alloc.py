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


def _state(p, seed, damaged=False):
    u, kh = li.random_state(p.mesh, seed=seed, kappa0=p.material.kappa0, strain=2e-4 if damaged else 2e-5)
    if damaged:
        return u, kh                                    # loading and damaged points: a nonsymmetric system
    return u, np.full(p.mesh.nel * p.mesh.ngp, 1.0)     # undamaged: a well-conditioned system


ARRAY_BYTES = 64 << 20


def _need(nd, nnode):
    """Scratch bytes of a system, as the entry point carves the array: nine
    vectors, the node-block inverses, the reduction tiles, the barrier words,
    the result block and one diagonal index per node, each rounded to 256."""
    up = lambda n: (n + 255) // 256 * 256
    t = 32
    while (nnode + t - 1) // t > 2048:
        t *= 2
    ntiles = (nnode + t - 1) // t
    return (9 * up(8 * nd * nnode) + up(8 * nnode * nd * nd) + up(8 * 12 * ntiles) + up(8) + up(64)
            + up(4 * nnode))


def _compare(lib, p, seeds, damaged, rtol, tol):
    """Solve the same assembled systems with lgdm_solve (workspace) and with
    lgdm_solve_noalloc (static array), calls in a row, and compare."""
    from paper_2301_06503_gb300 import Sim
    s = Sim(p.mesh, p.material, p.bcs, krylov_rtol=rtol, precond="block")   # the entry point's preconditioner
    stream = torch.cuda.current_stream()
    for seed in seeds:
        u, kh = _state(p, seed, damaged)
        s.set_state(u, kh)
        s.assemble()
        rowptr, col, vals, rhs = s.system()
        s.solve()
        x_ref = s.field("delta")
        ptr, nbr = _node_pattern(rowptr, col, s.nd, p.mesh.nnode)
        assert _need(s.nd, p.mesh.nnode) <= ARRAY_BYTES
        d_ptr = torch.from_numpy(ptr).cuda()
        d_nbr = torch.from_numpy(nbr).cuda()
        d_vals = torch.from_numpy(vals).cuda()
        d_rhs = torch.from_numpy(rhs).cuda()
        d_x = torch.full((s.ndof,), float("nan"), dtype=torch.float64, device="cuda")
        it, rel = C.c_int32(), C.c_double()
        st = lib.lgdm_solve_noalloc(s.nd, p.mesh.nnode, d_ptr.data_ptr(), d_nbr.data_ptr(), d_vals.data_ptr(),
                                    d_rhs.data_ptr(), d_x.data_ptr(), rtol, 5000, stream.cuda_stream,
                                    C.byref(it), C.byref(rel))
        assert st == 0, lib.lgdm_last_error(None)
        assert rel.value <= rtol and it.value > 0
        x = d_x.cpu().numpy()
        assert np.abs(x - x_ref).max() <= tol * np.abs(x_ref).max()
    s.close()


def test_noalloc_setup_call_only():
    """nnode = 0 performs only the per-device set-up (reserving the array and
    looking up its address) and touches no system."""
    from paper_2301_06503_gb300 import _lib
    lib = _lib.load()
    assert lib.lgdm_solve_noalloc(0, 0, None, None, None, None, None, 0.0, 0, None, None, None) == 0


def test_noalloc_solve_matches_workspace_solve_twice():
    from paper_2301_06503_gb300 import _lib
    _compare(_lib.load(), li.sen_plate_problem(30, 20), (31, 32), False, 1e-12, 1e-10)


@pytest.mark.parametrize("name", ["bar", "beam", "damaged_plate"])
def test_noalloc_other_block_sizes_and_damaged_state(name):
    """nd = 2 (bar), nd = 4 (hexahedra) and a damaged, nonsymmetric plate
    state (loading points: the K_ue and K_ee coupling terms of Eq. 11b/d)."""
    from paper_2301_06503_gb300 import _lib
    p = {"bar": li.bar_problem(n=301), "beam": li.tpb_beam_problem(12, 6, 6, 120.0, 60.0, 60.0),
         "damaged_plate": li.sen_plate_problem(24, 16)}[name]
    damaged = name == "damaged_plate"
    # the same BiCGSTAB arithmetic on both sides (tile-ordered inner products do
    # not depend on the block count): equal up to rounding-free reordering
    _compare(_lib.load(), p, (41, 42), damaged, 1e-12 if not damaged else 1e-8, 1e-12)


def test_noalloc_system_just_under_the_limit():
    """A 477 x 477 plate (228,484 nodes, 685k dofs) fills more than 99 % of the
    array; its solve matches the workspace solve.  One more node row beyond
    the limit is refused before anything is launched."""
    from paper_2301_06503_gb300 import _lib
    lib = _lib.load()
    p = li.sen_plate_problem(477, 477)
    need = _need(3, p.mesh.nnode)
    assert 0.99 * ARRAY_BYTES < need <= ARRAY_BYTES
    _compare(lib, p, (51,), False, 1e-8, 1e-12)
    n_over = p.mesh.nnode + 478 * 3
    assert _need(3, n_over) > ARRAY_BYTES
    d = torch.zeros(16, dtype=torch.float64, device="cuda")
    i = torch.zeros(16, dtype=torch.int32, device="cuda")
    it, rel = C.c_int32(), C.c_double()
    st = lib.lgdm_solve_noalloc(3, n_over, i.data_ptr(), i.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr(),
                                1e-8, 10, torch.cuda.current_stream().cuda_stream, C.byref(it), C.byref(rel))
    assert st == 2 and b"static array" in lib.lgdm_last_error(None)


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
