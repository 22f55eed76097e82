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

# elem -> (dim, nen, nv, nve): nve nodes carry the micro-equivalent strain
_DIMS = {1: (1, 2, 1, 2), 2: (2, 4, 3, 4), 3: (3, 8, 6, 8), 4: (1, 3, 1, 2), 5: (2, 9, 3, 4)}


def _btv(d):
    return {1: 1, 2: 6, 3: 15}[d]


def element_flops(elem: int):
    """(residual-path flops, tangent-path flops) per element.  Mixed-order
    elements count the micro-strain terms on their nve vertex nodes only."""
    d, n, v, ne = _DIMS[elem]
    q = n                                                                # Gauss points
    geo = 2 * d * d * n + {1: 1, 2: 8, 3: 42}[d] + 2 * n * d * d        # J, inverse, dN/dx
    if ne < n:
        geo += 2 * ne * d * d                                            # dNe/dx
    strain = 2 * n * (d + 2 * (v - d)) if d > 1 else 2 * n
    fields = 2 * ne + 2 * ne * d                                         # ebar, grad ebar
    evm = {1: 0, 2: 25, 3: 35}[d]
    damage = 15 + 5                                                      # Eq. A.1, A.4
    stress = {1: 1, 2: 8, 3: 15}[d]
    rec_res = v + 4
    rec_tan = n * _btv(d) + v + 10                                       # z_b, tangent factors
    per_gp_res = geo + strain + fields + evm + damage + stress + rec_res
    res = q * per_gp_res + q * n * _btv(d) + q * ne * (3 * d + 4)       # u rows, micro-strain rows
    kuu = {1: 1, 2: 8, 3: 21}[d]
    per_aq_tan = 5 * d + _btv(d) + 3
    per_q_pairs = 2 * (n * n * kuu + n * ne * d + ne * n * d + ne * ne * (1 + d))   # K_uu, K_ue, K_eu, K_ee
    tan = q * rec_tan + q * (n * per_aq_tan + per_q_pairs)
    return res, tan


def assembly_bytes(elem: int, nnode: int, nel: int, nnz: int, tangent_bytes: int) -> int:
    d, n, _, _ = _DIMS[elem]
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


def vcycle(levels, nd, tb, float_pairs=False):
    """(FP64 flops, bytes, FP32-pipe flops) of one multigrid V-cycle; levels =
    [(nnode, npairs), ...] from the finest: per level above the coarsest a
    Jacobi pre-smoothing, a residual (SpMV), the restriction sum, and the
    post-smoothing (SpMV on the prolonged iterate, Jacobi apply, update); the
    coarsest a dense N x N product (N = nd * its nodes).  With float_pairs
    (FP32 tangent) the finest level's residual SpMV runs on the FP32 pipe from
    the float-pair copy of its iterate (written once more per V-cycle)."""
    f = b = f32 = 0
    for k, (n, np_) in enumerate(levels[:-1]):
        fj, bj = _jacobi(n, nd, tb)
        fs, bs = _spmv(n, nd, np_, tb)
        f += 2 * fj + fs + 4 * nd * n
        if float_pairs and k == 0:
            f32 += fs
            b += nd * n * 8                       # the float-pair copy of X
        else:
            f += fs
        b += 2 * bj + 2 * bs + 6 * nd * n * 8 + n * 8
    nc = nd * levels[-1][0]
    f += 2 * nc * nc
    b += nc * nc * 8 + 2 * nc * 8
    return f, b, f32


def krylov_iteration(nnode: int, nd: int, nnz: int, npairs: int, tangent_bytes: int, levels=None,
                     float_pairs=False):
    """(FP64 flops, bytes, FP32-pipe flops) of one BiCGSTAB iteration: 2 SpMV,
    2 preconditioner applies (node-block Jacobi, or a multigrid V-cycle when
    ``levels`` lists the multigrid levels), 4 inner products and 6 vector
    updates.  With float_pairs (FP32 tangent) the 2 SpMVs (and the finest
    residual of each V-cycle) are FP32-pipe products from float-pair copies
    of the preconditioned vectors; the flops are the algorithmic 2 per
    nonzero either way."""
    ndof = nd * nnode
    fs, bs = _spmv(nnode, nd, npairs, tangent_bytes)
    if levels and len(levels) > 1:
        fp, bp, fp32 = vcycle(levels, nd, tangent_bytes, float_pairs)
    else:
        (fp, bp), fp32 = _jacobi(nnode, nd, tangent_bytes), 0
    flops = 2 * fp + 2 * 4 * ndof + 2 * 8 * ndof
    f32 = 2 * fp32
    if float_pairs:
        f32 += 2 * fs
    else:
        flops += 2 * fs
    vec = 26 * ndof * 8 + (2 * ndof * 8 if float_pairs else 0)
    return flops, 2 * bs + 2 * bp + vec, f32
