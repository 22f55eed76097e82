"""Element integration of the coupled u / micro-equivalent-strain system.

One call evaluates, for a set of elements and all their Gauss points at once
(the whole-array style of the paper's Algorithm 2), the element blocks of the
tangent (Eq. 11a-d) and of the residual (Eq. 11e-f, written as r = -F):

  r_u   = sum_q B_u^T sigma dV,          sigma = (1 - D) C_e eps
  r_e   = sum_q [N h (ebar - eps_eq) + B_e^T g h c grad(ebar)] dV
  K_uu  = sum_q B_u^T (1 - D) C_e B_u dV                              (11a)
  K_ue  = -sum_q B_u^T (C_e eps) D' chi N^T dV                         (11b)
  K_eu  = -sum_q N h (d eps_eq/d eps)^T B_u dV                         (11c)
  K_ee  = sum_q [h N N^T + g h c B_e^T B_e + h c g' D' chi (B_e^T grad ebar) N^T] dV  (11d)

N and B_e are the micro-equivalent-strain interpolation, B_u the
displacement one.  Readings: sigma carries no h-term (the paper's own element
code forms f_u = -k_uu u_e and passes no h to its K_ue routine) unless the
material asks for the Eq. 2-literal stress (``h_stress`` = 1):
sigma = (1 - D) C eps + h (eps_eq - ebar) d eps_eq/d eps, whose consistent
tangent adds B_u^T [h d (x) d + h (eps_eq - ebar) d2 eps_eq/d eps2] B_u dV to
K_uu and -B_u^T h d N^T dV to K_ue (Eq. 11a-b in full); the gradient term of
F_e takes the sign that makes F_e = -r_e; dg/dkappa in Eq. 11d is
g'(D) D'(kappa) chi.

Elements.  Equal order: 2-node bar, 4-node quad and 8-node hex for both
fields, with 2, 2x2, 2x2x2 Gauss points at +-1/sqrt(3) and unit weights.
Mixed order (Sec. 2.2, the paper's 1D and 2D discretisation): a 3-node
quadratic bar and a 9-node biquadratic quad for u, whose first 2 / 4 local
nodes (the vertices) carry the linear / bilinear micro-equivalent strain,
with 3 and 3x3 Gauss points at 0, +-sqrt(3/5) and weights 8/9, 5/9.  The
geometry is interpolated like u.  In every element Gauss point q sits at the
reference position of local node q scaled by the rule's abscissa, so
Gauss-point arrays follow the node order.
"""
import numpy as np

from . import constitutive as cm

L2, Q4, H8, L3, Q9 = 1, 2, 3, 4, 5
_REF = {
    L2: np.array([[-1.0], [1.0]]),
    Q4: np.array([[-1.0, -1.0], [1.0, -1.0], [1.0, 1.0], [-1.0, 1.0]]),
    H8: np.array([[-1.0, -1.0, -1.0], [1.0, -1.0, -1.0], [1.0, 1.0, -1.0], [-1.0, 1.0, -1.0],
                  [-1.0, -1.0, 1.0], [1.0, -1.0, 1.0], [1.0, 1.0, 1.0], [-1.0, 1.0, 1.0]]),
    L3: np.array([[-1.0], [1.0], [0.0]]),
    Q9: np.array([[-1.0, -1.0], [1.0, -1.0], [1.0, 1.0], [-1.0, 1.0],
                  [0.0, -1.0], [1.0, 0.0], [0.0, 1.0], [-1.0, 0.0], [0.0, 0.0]]),
}
# element of the micro-equivalent strain: its nodes are the first local nodes
EBAR_ELEM = {L2: L2, Q4: Q4, H8: H8, L3: L2, Q9: Q4}
QUADRATIC = (L3, Q9)


def reference_nodes(elem):
    return _REF[elem]


def ebar_nodes(elem):
    """Number of local nodes carrying the micro-equivalent strain."""
    return _REF[EBAR_ELEM[elem]].shape[0]


def gauss_rule(elem):
    """Gauss points (ngp, d) and weights (ngp,): the tensor 2-point rule
    (abscissae +-1/sqrt(3), weights 1) for the linear elements, the tensor
    3-point rule (0, +-sqrt(3/5); weights 8/9, 5/9) for the quadratic ones."""
    ref = _REF[elem]
    if elem in QUADRATIC:
        xi = ref * np.sqrt(3.0 / 5.0)
        w = np.prod(np.where(ref == 0.0, 8.0 / 9.0, 5.0 / 9.0), axis=1)
        return xi, w
    return ref / np.sqrt(3.0), np.ones(ref.shape[0])


def _lagrange_1d(order, r, t):
    """1D Lagrange polynomial of the node at r (-1, 0 or 1) and its derivative
    at t: linear on {-1, 1}, quadratic on {-1, 0, 1}."""
    if order == 1:
        return (1.0 + r * t) / 2.0, np.full_like(t, r / 2.0)
    if r == 0.0:
        return 1.0 - t * t, -2.0 * t
    return t * (t + r) / 2.0, t + r / 2.0


def shape_functions(elem, xi):
    """Lagrange shape functions and reference derivatives at points xi.

    N_a(xi) = prod_i l_a(xi_i), the 1D Lagrange polynomials of the element's
    order; returns N (np, nen) and dN/dxi (np, nen, d).
    """
    ref = _REF[elem]
    order = 2 if elem in QUADRATIC else 1
    npt, nen, d = xi.shape[0], ref.shape[0], ref.shape[1]
    val = np.empty((npt, nen, d))
    der = np.empty((npt, nen, d))
    for a in range(nen):
        for i in range(d):
            val[:, a, i], der[:, a, i] = _lagrange_1d(order, ref[a, i], xi[:, i])
    N = np.prod(val, axis=2)
    dN = np.empty((npt, nen, d))
    for j in range(d):
        dN[:, :, j] = der[:, :, j] * (np.prod(np.delete(val, j, axis=2), axis=2) if d > 1 else 1.0)
    return N, dN


def ebar_shape_functions(elem, xi):
    """Shape functions of the micro-equivalent strain at points xi: those of
    the linear element on the first ebar_nodes(elem) local nodes."""
    return shape_functions(EBAR_ELEM[elem], xi)


def strain_displacement(dNdx):
    """B_u in Voigt form (engineering shear) from physical derivatives.

    dNdx: (..., nen, d) -> B: (..., nv, nen*d), dofs ordered (a, i) -> d*a + i.
    """
    lead = dNdx.shape[:-2]
    nen, d = dNdx.shape[-2:]
    nv = {1: 1, 2: 3, 3: 6}[d]
    B = np.zeros(lead + (nv, nen * d), dtype=dNdx.dtype)
    for a in range(nen):
        gx = dNdx[..., a, 0]
        if d == 1:
            B[..., 0, a] = gx
            continue
        gy = dNdx[..., a, 1]
        if d == 2:
            B[..., 0, 2 * a] = gx
            B[..., 1, 2 * a + 1] = gy
            B[..., 2, 2 * a] = gy
            B[..., 2, 2 * a + 1] = gx
            continue
        gz = dNdx[..., a, 2]
        c = 3 * a
        B[..., 0, c] = gx
        B[..., 1, c + 1] = gy
        B[..., 2, c + 2] = gz
        B[..., 3, c + 1] = gz
        B[..., 3, c + 2] = gy
        B[..., 4, c] = gz
        B[..., 4, c + 2] = gx
        B[..., 5, c] = gy
        B[..., 5, c + 1] = gx
    return B


def _jacobian(mesh, elems):
    """Inverse Jacobian (ne, ngp, d, d) and the measure w det J vol_scale (ne, ngp)
    of the isoparametric map (the geometry interpolated like u)."""
    xi, w = gauss_rule(mesh.elem)
    _, dN = shape_functions(mesh.elem, xi)
    X = mesh.coords()[mesh.conn[elems]]                          # (ne, nen, d)
    J = np.einsum("eai,qaj->eqij", X, dN)                        # dx_i/dxi_j
    detJ = np.linalg.det(J)
    Jinv = np.linalg.inv(J)                                      # dxi_j/dx_i = Jinv[j, i]
    return Jinv, w[None, :] * detJ * mesh.vol_scale[elems][:, None]


def geometry(mesh, elems):
    """Physical shape derivatives dN/dx (ne, ngp, nen, d) and dV (ne, ngp)."""
    xi, _ = gauss_rule(mesh.elem)
    _, dN = shape_functions(mesh.elem, xi)
    Jinv, dV = _jacobian(mesh, elems)
    return np.einsum("qaj,eqji->eqai", dN, Jinv), dV


def ebar_geometry(mesh, elems):
    """Micro-equivalent-strain shape functions (ngp, nve) and their physical
    derivatives (ne, ngp, nve, d) at the Gauss points."""
    xi, _ = gauss_rule(mesh.elem)
    Ne, dNe = ebar_shape_functions(mesh.elem, xi)
    Jinv, _ = _jacobian(mesh, elems)
    return Ne, np.einsum("qaj,eqji->eqai", dNe, Jinv)


def element_terms(mesh, mat, u, kappa_hist, elems=None):
    """Element tangent blocks, residual blocks and Gauss-point fields.

    u: nodal dofs [ndof] (interleaved, may be complex for complex-step checks);
    kappa_hist: committed history [nel*ngp] (real).
    Returns a dict of arrays over the selected elements.
    """
    if elems is None:
        elems = np.arange(mesh.nel)
    elems = np.asarray(elems)
    d, nen, nd = mesh.dim, mesh.nen, mesh.nd
    nve = ebar_nodes(mesh.elem)
    dNdx, dV = geometry(mesh, elems)
    N, dNdx_e = ebar_geometry(mesh, elems)                       # (ngp, nve), (ne, ngp, nve, d)
    B = strain_displacement(dNdx)                                # (ne, ngp, nv, nen*d)

    U = np.asarray(u).reshape(mesh.nnode, nd)[mesh.conn[elems]]  # (ne, nen, nd)
    ue = U[:, :, :d].reshape(len(elems), nen * d)
    ee = U[:, :nve, d]                                           # (ne, nve): vertex nodes

    C = cm.elasticity_matrix(d, mat.E, mat.nu)
    Ce = mesh.e_scale[elems][:, None, None] * C                  # (ne, nv, nv)

    eps = np.einsum("eqvk,ek->eqv", B, ue)                       # strain
    eps_eq, deq = cm.equivalent_strain(eps, d, mat.nu, mat.k, mat.evm_variant)
    ebar = np.einsum("qa,ea->eq", N, ee)                         # micro-equivalent strain at GP
    gbar = np.einsum("eqai,ea->eqi", dNdx_e, ee)                 # its gradient
    kh = np.asarray(kappa_hist).reshape(mesh.nel, mesh.ngp)[elems]
    kappa, chi = cm.history(kh, ebar)
    D, dD = cm.damage(kappa, mat.kappa0, mat.alpha, mat.beta)
    g, dg = cm.interaction(D, mat.R, mat.eta)
    Ceps = np.einsum("evw,eqw->eqv", Ce, eps)
    sigma = (1.0 - D)[..., None] * Ceps
    h, c = mat.h, mat.c
    h_stress = int(getattr(mat, "h_stress", 0))
    if h_stress:
        sigma = sigma + (h * (eps_eq - ebar))[..., None] * deq

    ru = np.einsum("eqvk,eqv,eq->ek", B, sigma, dV)
    re = (np.einsum("qa,eq->ea", N, h * (ebar - eps_eq) * dV)
          + np.einsum("eqai,eqi,eq->ea", dNdx_e, gbar, g * h * c * dV))

    Kuu = np.einsum("eqvk,evw,eqwl,eq->ekl", B, Ce, B, (1.0 - D) * dV)
    Kue = -np.einsum("eqvk,eqv,qb,eq->ekb", B, Ceps, N, dD * chi * dV)
    if h_stress:
        Hq = cm.equivalent_strain_hessian(eps, d, mat.nu, mat.k, mat.evm_variant)
        Mq = (np.einsum("eqv,eqw->eqvw", deq, deq) + (eps_eq - ebar)[..., None, None] * Hq) * (h * dV)[..., None, None]
        Kuu = Kuu + np.einsum("eqvk,eqvw,eqwl->ekl", B, Mq, B)
        Kue = Kue - np.einsum("eqvk,eqv,qb,eq->ekb", B, deq, N, h * dV)
    Keu = -np.einsum("qa,eqv,eqvk,eq->eak", N, deq, B, h * dV)
    Kee = (np.einsum("qa,qb,eq->eab", N, N, h * dV)
           + np.einsum("eqai,eqbi,eq->eab", dNdx_e, dNdx_e, g * h * c * dV)
           + np.einsum("eqai,eqi,qb,eq->eab", dNdx_e, gbar, N, h * c * dg * dD * chi * dV))
    return dict(Kuu=Kuu, Kue=Kue, Keu=Keu, Kee=Kee, ru=ru, re=re,
                eps=eps, eps_eq=eps_eq, ebar=ebar, gbar=gbar, kappa=kappa, chi=chi,
                D=D, g=g, Ceps=Ceps, dV=dV)


def local_dofs(mesh, elems):
    """Global dof numbers of the element blocks: u part (ne, nen*d), e part
    (ne, nve): the micro-equivalent strain of the vertex nodes."""
    conn = mesh.conn[np.asarray(elems)].astype(np.int64)
    d, nd = mesh.dim, mesh.nd
    gu = (nd * conn[:, :, None] + np.arange(d)[None, None, :]).reshape(conn.shape[0], -1)
    ge = nd * conn[:, :ebar_nodes(mesh.elem)] + d
    return gu, ge


def unused_dofs(mesh):
    """Micro-equivalent-strain dofs that no element interpolates (those of the
    non-vertex nodes of mixed-order meshes): they take part in no equation."""
    carried = np.zeros(mesh.nnode, dtype=bool)
    carried[mesh.conn[:, :ebar_nodes(mesh.elem)].ravel()] = True
    return (mesh.nd * np.nonzero(~carried)[0] + mesh.dim).astype(np.int64)


def element_matrix(terms):
    """Element tangent in block order [u dofs; e dofs] (the paper's k_local)."""
    top = np.concatenate([terms["Kuu"], terms["Kue"]], axis=2)
    bot = np.concatenate([terms["Keu"], terms["Kee"]], axis=2)
    return np.concatenate([top, bot], axis=1), np.concatenate([terms["ru"], terms["re"]], axis=1)


def gp_ebar(mesh, u, elems=None):
    """Micro-equivalent strain at every Gauss point, (ne, ngp)."""
    if elems is None:
        elems = np.arange(mesh.nel)
    xi, _ = gauss_rule(mesh.elem)
    N, _ = ebar_shape_functions(mesh.elem, xi)
    ee = np.asarray(u).reshape(mesh.nnode, mesh.nd)[mesh.conn[elems][:, :ebar_nodes(mesh.elem)], mesh.dim]
    return np.einsum("qa,ea->eq", N, ee)
