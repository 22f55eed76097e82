"""Algorithmic work of the hot path, for roofline fractions.

Flops are counted from the formulas of Eq. 11a-f (FMA = 2 flops) in the
factorisation the element kernel evaluates: per Gauss point the geometry,
strain, equivalent strain, damage and interaction (Eq. A.1-A.4) once; per
(row node a, Gauss point q) the block-row constants; per (a, q, column node
b) the isotropic K_uu block (lam' a_i b_j + mu' a_j b_i + mu' a.b delta_ij),
the K_ue / K_eu rank-one terms and the K_ee term.  Exponentials, square roots
and divisions count one flop each.  Bytes are the minimum the method moves
per assembly: nodal coordinates, connectivity, dofs, Gauss-point history and
element scales read once; every CSR value and residual entry written once.
"""

_DIMS = {1: (1, 2, 1), 2: (2, 4, 3), 3: (3, 8, 6)}          # elem -> (dim, nen, nv)


def _btv(d):
    return {1: 1, 2: 6, 3: 15}[d]


def element_flops(elem: int):
    """(residual-path flops, tangent-path flops) per element."""
    d, n, v = _DIMS[elem]
    geo = 2 * d * d * n + {1: 1, 2: 8, 3: 42}[d] + 2 * n * d * d        # J, inverse, dN/dx
    strain = 2 * n * (d + 2 * (v - d)) if d > 1 else 2 * n
    fields = 2 * n + 2 * n * d                                           # ebar, grad ebar
    evm = {1: 0, 2: 25, 3: 35}[d]
    damage = 15 + 5                                                      # Eq. A.1, A.4
    stress = {1: 1, 2: 8, 3: 15}[d]
    rec_res = v + 4
    rec_tan = n * _btv(d) + v + 10                                       # z_b, tangent factors
    per_gp_res = geo + strain + fields + evm + damage + stress + rec_res
    per_aq_res = _btv(d) + d + 2 * d + 4
    per_b = 2 * ({1: 1, 2: 8, 3: 21}[d] + d + d + 1 + d)
    per_aq_tan = 5 * d + _btv(d) + 3 + n * per_b
    res = n * per_gp_res + n * n * per_aq_res
    tan = n * rec_tan + n * n * per_aq_tan
    return res, tan


def assembly_bytes(elem: int, nnode: int, nel: int, nnz: int, tangent_bytes: int) -> int:
    d, n, _ = _DIMS[elem]
    nd = d + 1
    ndof = nd * nnode
    reads = nnode * d * 8 + nel * n * 4 + ndof * 8 + nel * n * 8 + nel * 16
    writes = nnz * tangent_bytes + 2 * ndof * 8
    return reads + writes


def _spmv(nnode, nd, npairs, tb):
    """(flops, bytes) of y = A x on a node-block CSR level: nd*nd values per
    node pair, one neighbour index per pair, x read and y written once."""
    nnz = nd * nd * npairs
    return 2 * nnz, nnz * tb + npairs * 4 + (nnode + 1) * 4 + 2 * nd * nnode * 8


def _jacobi(nnode, nd, tb):
    """(flops, bytes) of one node-block Jacobi apply."""
    return 2 * nnode * nd * nd, nnode * nd * nd * tb + 2 * nd * nnode * 8


def vcycle(levels, nd, tb):
    """(flops, bytes) of one multigrid V-cycle; levels = [(nnode, npairs), ...]
    from the finest: per level above the coarsest a Jacobi pre-smoothing, a
    residual (SpMV), the restriction sum, and the post-smoothing (SpMV on the
    prolonged iterate, Jacobi apply, update); the coarsest a dense N x N
    product (N = nd * its nodes)."""
    f = b = 0
    for n, np_ in levels[:-1]:
        fj, bj = _jacobi(n, nd, tb)
        fs, bs = _spmv(n, nd, np_, tb)
        f += 2 * fj + 2 * fs + 4 * nd * n
        b += 2 * bj + 2 * bs + 6 * nd * n * 8 + n * 8
    nc = nd * levels[-1][0]
    f += 2 * nc * nc
    b += nc * nc * 8 + 2 * nc * 8
    return f, b


def krylov_iteration(nnode: int, nd: int, nnz: int, npairs: int, tangent_bytes: int, levels=None):
    """(flops, bytes) of one BiCGSTAB iteration: 2 SpMV, 2 preconditioner
    applies (node-block Jacobi, or a multigrid V-cycle when ``levels`` lists
    the multigrid levels), 4 inner products and 6 vector updates."""
    ndof = nd * nnode
    fs, bs = _spmv(nnode, nd, npairs, tangent_bytes)
    if levels and len(levels) > 1:
        fp, bp = vcycle(levels, nd, tangent_bytes)
    else:
        fp, bp = _jacobi(nnode, nd, tangent_bytes)
    flops = 2 * fs + 2 * fp + 2 * 4 * ndof + 2 * 8 * ndof
    vec = 26 * ndof * 8
    return flops, 2 * bs + 2 * bp + vec
