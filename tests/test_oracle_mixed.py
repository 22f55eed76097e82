"""Pins for the mixed-order elements of the CPU oracle (Sec. 2.2: quadratic u
with linear micro-equivalent strain; the paper's 1D bar and 2D specimens).

  M1  shape functions: Kronecker property at the nodes, and exact
      reproduction of every monomial of the element's space (values and
      gradients) -- quadratic for u, linear for the micro-equivalent strain
  M2  3-point and 3x3 Gauss rules integrate polynomials of degree <= 5 per
      direction exactly
  M3  element measure: straight-edged elements give the polygon area; a
      mid-side node moved off its edge adds the parabolic segment 2/3 L s
  M4  patch test on a distorted mesh (linear u, constant eps_eq) and
      rigid-body motions: zero residual
  M5  tangent (Eq. 11a-d) = complex-step Jacobian of the residual, both
      stress variants, at random damaged states with loading and unloading
  M6  elastic closed forms: uniform bar reaction E A u / L, plane-strain
      uniaxial stress; stored energy (Eq. 1) = external work = 1/2 sigma eps V
  M7  dof structure: the micro-equivalent strain of non-vertex nodes has
      empty rows and columns and is held at zero; a linear-u field gives the
      same micro-strain residual as on the linear mesh of the vertex nodes
  M8  the paper's bar: its Fig. 10 parameters, the closed-form compliance
      of the elastic branch, and no damage before the defect's local strain
      reaches kappa0 (maximum principle of the micro-strain equation)
"""
import numpy as np
import pytest

import lgdm_inputs as li
from lgdm_inputs.meshes import L2, Q4, L3, Q9
from oracle import assembly as asm
from oracle import constitutive as cm
from oracle import element as el
from oracle import newton as nw

MAT = li.Material()


def _monomials(d, deg):
    """Exponent tuples of the tensor space of degree ``deg`` per direction."""
    if d == 1:
        return [(i,) for i in range(deg + 1)]
    return [(i, j) for i in range(deg + 1) for j in range(deg + 1)]


def _eval(exps, X):
    return np.prod([X[:, k] ** exps[k] for k in range(X.shape[1])], axis=0)


def _grad(exps, X):
    out = np.zeros(X.shape)
    for k in range(X.shape[1]):
        if exps[k] == 0:
            continue
        e = list(exps)
        e[k] -= 1
        out[:, k] = exps[k] * _eval(e, X)
    return out


@pytest.mark.parametrize("elem,deg", [(L3, 2), (Q9, 2), (L2, 1), (Q4, 1)])
def test_m1_shape_functions_reproduce_their_space(elem, deg):
    ref = el.reference_nodes(elem)
    N, dN = el.shape_functions(elem, ref)
    np.testing.assert_allclose(N, np.eye(ref.shape[0]), atol=1e-15)
    rng = np.random.default_rng(1)
    xi = rng.uniform(-1, 1, size=(7, ref.shape[1]))
    N, dN = el.shape_functions(elem, xi)
    for exps in _monomials(ref.shape[1], deg):
        np.testing.assert_allclose(N @ _eval(exps, ref), _eval(exps, xi), atol=1e-14)
        np.testing.assert_allclose(np.einsum("pak,a->pk", dN, _eval(exps, ref)), _grad(exps, xi), atol=1e-13)
    if deg == 2:     # the space is exactly quadratic: a cubic is not reproduced
        cub = (3,) + (0,) * (ref.shape[1] - 1)
        assert np.abs(N @ _eval(cub, ref) - _eval(cub, xi)).max() > 1e-3


@pytest.mark.parametrize("elem,lin", [(L3, L2), (Q9, Q4)])
def test_m1_ebar_shape_functions_are_the_vertex_element(elem, lin):
    xi, _ = el.gauss_rule(elem)
    Ne, dNe = el.ebar_shape_functions(elem, xi)
    assert Ne.shape[1] == el.ebar_nodes(elem) == el.reference_nodes(lin).shape[0]
    vert = el.reference_nodes(elem)[: Ne.shape[1]]
    np.testing.assert_array_equal(vert, el.reference_nodes(lin))
    for exps in _monomials(xi.shape[1], 1):
        np.testing.assert_allclose(Ne @ _eval(exps, vert), _eval(exps, xi), atol=1e-15)


@pytest.mark.parametrize("elem", [L3, Q9])
def test_m2_gauss_rules_exact_to_degree_five(elem):
    xi, w = el.gauss_rule(elem)
    d = xi.shape[1]
    assert len(w) == 3 ** d
    exact1 = lambda k: 0.0 if k % 2 else 2.0 / (k + 1)
    for exps in _monomials(d, 5):
        got = np.sum(w * _eval(exps, xi))
        assert abs(got - np.prod([exact1(k) for k in exps])) <= 1e-14
    assert abs(np.sum(w * _eval((6,) + (0,) * (d - 1), xi)) - 2.0 ** d / 7.0) > 1e-3   # degree 6 is not


def test_m3_element_measure():
    m = li.plate_q9(1, 1, 2.0, 1.0)
    X = np.array([[0.0, 0.0], [2.0, 0.2], [2.3, 1.4], [-0.2, 1.0]])    # a general quadrilateral
    ref = el.reference_nodes(Q9)
    N1, _ = el.shape_functions(Q4, ref)                              # straight edges, bilinear centre
    P = N1 @ X
    m.x[m.conn[0]] = P[:, 0]
    m.y[m.conn[0]] = P[:, 1]
    poly = 0.5 * abs(np.sum(X[:, 0] * np.roll(X[:, 1], -1) - np.roll(X[:, 0], -1) * X[:, 1]))
    _, dV = el.geometry(m, [0])
    assert abs(dV.sum() - poly) <= 1e-13 * poly
    # bow the bottom edge outwards by s at its mid-side node: + 2/3 L s
    s = 0.05
    L = np.hypot(*(X[1] - X[0]))
    nrm = np.array([X[1, 1] - X[0, 1], X[0, 0] - X[1, 0]]) / L      # outward for a counter-clockwise element
    m.x[m.conn[0, 4]] += s * nrm[0]
    m.y[m.conn[0, 4]] += s * nrm[1]
    _, dV = el.geometry(m, [0])
    assert abs(dV.sum() - (poly + 2.0 / 3.0 * L * s)) <= 1e-13 * poly
    # 1D: the bar's length times its section, middle node anywhere inside
    b = li.bar_l3(2, 4.0, 3.0)
    b.x[1] += 0.3
    _, dV = el.geometry(b, [0, 1])
    assert abs(dV.sum() - 12.0) <= 1e-13


def _distorted_q9(nx=3, ny=3):
    m = li.plate_q9(nx, ny, float(nx), float(ny))
    inner = (m.x > 0) & (m.x < nx) & (m.y > 0) & (m.y < ny)
    m.x[inner] += 0.12 * np.sin(2.1 * m.y[inner] + m.x[inner])
    m.y[inner] += 0.09 * np.cos(1.7 * m.x[inner])
    return m, inner


def test_m4_patch_test_and_rigid_body():
    m, inner = _distorted_q9()
    mat = li.Material(**{**MAT.__dict__})
    mat.kappa0 = 1.0                             # elastic
    rng = np.random.default_rng(2)
    G = rng.normal(size=(2, 2)) * 1e-4
    X = m.coords()
    U = np.zeros((m.nnode, 3))
    U[:, :2] = X @ G.T + rng.normal(size=2) * 1e-3
    eq, _ = cm.equivalent_strain(np.array([G[0, 0], G[1, 1], G[0, 1] + G[1, 0]]), 2, mat.nu, mat.k)
    U[:, 2] = eq
    U[el.unused_dofs(m) // 3, 2] = 0.0           # not interpolated: any value
    kh = np.full(m.nel * m.ngp, mat.kappa0)
    _, r = asm.assemble(m, mat, U.ravel(), kh)
    R = r.reshape(m.nnode, 3)
    assert np.abs(R[inner, :2]).max() < 1e-12 * mat.E * 1e-4
    assert np.abs(R[:, 2]).max() < 1e-12 * mat.h * 1e-4
    # rigid-body motion, bar and plate
    U[:, :2] = np.array([1e-3, -2e-3]) + 1e-3 * np.stack([-X[:, 1], X[:, 0]], 1)
    U[:, 2] = 0.0
    _, r = asm.assemble(m, MAT, U.ravel(), kh)
    assert np.abs(r).max() < 1e-12 * MAT.E * 1e-3
    b = li.bar_l3(3, 3.0, 2.0)
    ub = np.zeros(b.ndof)
    ub[0::2] = 1e-3
    _, r = asm.assemble(b, li.Material(nu=0.0, k=1.0), ub, np.full(b.nel * b.ngp, 1e-4))
    assert np.abs(r).max() < 1e-12 * MAT.E * 1e-3


def _mixed_meshes():
    b = li.bar_l3(4, 4.0, 10.0)
    b.x[1::2] += 0.1 * np.sin(np.arange(4))      # middle nodes off centre
    yield b
    q = li.plate_q9(2, 2, 2.0, 2.0)
    q.x = q.x + 0.1 * q.y ** 2
    q.y = q.y + 0.05 * np.sin(2 * q.x)
    q.e_scale[1] = 1e-6
    yield q


def _complex_step_jacobian(mesh, mat, u, kh):
    K, _ = asm.assemble(mesh, mat, u, kh)
    K = K.toarray()
    h = 1e-30
    J = np.empty_like(K)
    for j in range(mesh.ndof):
        uc = u.astype(complex)
        uc[j] += 1j * h
        _, rc = asm.assemble(mesh, mat, uc, kh, with_tangent=False)
        J[:, j] = rc.imag / h
    return K, J


@pytest.mark.parametrize("mi", [0, 1])
@pytest.mark.parametrize("h_stress", [0, 1])
def test_m5_tangent_is_complex_step_jacobian(mi, h_stress):
    mesh = list(_mixed_meshes())[mi]
    base = MAT if mesh.dim > 1 else li.Material(nu=0.0, k=1.0)
    mat = li.Material(**{**base.__dict__, "h_stress": h_stress})
    if h_stress:
        mat.h = 1e-3 * mat.E                     # make the h-terms visible against E
    u, kh = li.random_state(mesh, seed=30 + mi, kappa0=mat.kappa0)
    K, J = _complex_step_jacobian(mesh, mat, u, kh)
    t = el.element_terms(mesh, mat, u, kh)
    assert 0 < t["chi"].sum() < t["chi"].size and np.any(t["D"] > 0)
    is_e = (np.arange(mesh.ndof) % mesh.nd) == mesh.dim
    for rm, cmask in ((~is_e, ~is_e), (~is_e, is_e), (is_e, ~is_e), (is_e, is_e)):
        a, b = K[np.ix_(rm, cmask)], J[np.ix_(rm, cmask)]
        scale = np.abs(b).max()
        assert scale > 0.0
        assert np.abs(a - b).max() <= 1e-10 * scale


def test_m6_elastic_closed_forms():
    # uniform bar of quadratic elements, middle nodes off centre: R = E A u / L
    p = li.bar_problem(n=10, weak_factor=1.0, order=2)
    p.mesh.x[1::2] += 0.2 * np.cos(np.arange(10))
    out = nw.run(p, n_steps=3)
    E, A, L = p.material.E, 10.0, 100.0
    np.testing.assert_allclose(out["reaction"], E * A * out["load"] / L, rtol=1e-12)
    closed = 0.5 * E * A * L * (out["load"] / L) ** 2
    np.testing.assert_allclose(out["psi"], closed, rtol=1e-12)
    lp, rp = np.concatenate([[0.0], out["load"]]), np.concatenate([[0.0], out["reaction"]])
    w = np.cumsum(0.5 * (rp[1:] + rp[:-1]) * np.diff(lp))
    np.testing.assert_allclose(w, closed, rtol=1e-12)
    # plane strain, uniaxial stress in y on a distorted 9-node mesh:
    # reaction = E/(1-nu^2) eps_yy W, Psi = 1/2 E/(1-nu^2) eps_yy^2 V
    m, _ = _distorted_q9(4, 3)
    X = m.coords()
    bottom, top = np.nonzero(X[:, 1] == 0.0)[0], np.nonzero(X[:, 1] == 3.0)[0]
    left = np.nonzero((X[:, 0] == 0.0) & (X[:, 1] > 0.0))[0]
    bcs = li.BCs(np.concatenate([li.node_dofs(m, bottom, 1), li.node_dofs(m, left, 0),
                                 li.node_dofs(m, top, 1)]).astype(np.int32),
                 np.concatenate([np.zeros(len(bottom)), np.zeros(len(left)), np.ones(len(top))]))
    mat = li.Material(**{**MAT.__dict__})
    mat.kappa0 = 1.0
    p2 = li.Problem("uniax_q9", m, mat, bcs, u_max=3e-4, n_steps=3)
    out = nw.run(p2)
    eyy = out["load"] / 3.0
    Ep = mat.E / (1 - mat.nu ** 2)
    np.testing.assert_allclose(out["reaction"], Ep * eyy * 4.0, rtol=1e-12)
    np.testing.assert_allclose(out["psi"], 0.5 * Ep * eyy ** 2 * 12.0, rtol=1e-12)


def test_m7_dof_structure():
    m, _ = _distorted_q9(3, 2)
    unused = el.unused_dofs(m)
    assert len(unused) == (7 * 5) - (4 * 3)
    u, kh = li.random_state(m, seed=5, kappa0=MAT.kappa0)
    K, r = asm.assemble(m, MAT, u, kh)
    K = K.tocsr()
    assert abs(K[unused]).max() == 0.0 and abs(K[:, unused]).max() == 0.0 and np.all(r[unused] == 0.0)
    Kb, rb = asm.apply_dirichlet(K, r, np.zeros(0, np.int64), m)
    np.testing.assert_array_equal(Kb[unused][:, unused].toarray(), np.eye(len(unused)))
    b = li.bar_l3(5, 5.0, 1.0)
    np.testing.assert_array_equal(el.unused_dofs(b), 2 * (2 * np.arange(5) + 1) + 1)
    # On a rectangular mesh, with u linear and a uniform history above every
    # micro-strain (no loading point: D and g uniform), every micro-strain
    # integrand is of degree <= 2 per direction, which the 2x2 rule already
    # integrates exactly: the micro-strain rows of the 9-node mesh at its
    # vertices equal those of the 4-node mesh of the same vertices.
    q9 = li.plate_q9(3, 2, 3.0, 2.0)
    q4 = li.plate_q4(3, 2, 3.0, 2.0)
    G = np.array([[2e-4, 5e-5], [-3e-5, 1e-4]])
    rng = np.random.default_rng(8)
    ebar4 = rng.uniform(0.0, 3e-4, q4.nnode)
    vid = {(round(x, 9), round(y, 9)): k for k, (x, y) in enumerate(zip(q9.x, q9.y))}
    vmap = np.array([vid[(round(x, 9), round(y, 9))] for x, y in zip(q4.x, q4.y)])
    U9 = np.zeros((q9.nnode, 3))
    U9[:, :2] = q9.coords() @ G.T
    U9[vmap, 2] = ebar4
    U4 = np.zeros((q4.nnode, 3))
    U4[:, :2] = q4.coords() @ G.T
    U4[:, 2] = ebar4
    kh = 5e-4
    _, r9 = asm.assemble(q9, MAT, U9.ravel(), np.full(q9.nel * q9.ngp, kh))
    _, r4 = asm.assemble(q4, MAT, U4.ravel(), np.full(q4.nel * q4.ngp, kh))
    e9, e4 = r9.reshape(-1, 3)[vmap, 2], r4.reshape(-1, 3)[:, 2]
    assert np.abs(e4).max() > 0.0
    np.testing.assert_allclose(e9, e4, rtol=0, atol=1e-13 * np.abs(e4).max())


def test_m8_paper_bar_elastic_branch_and_parameters():
    """The paper's bar (Sec. 3.1, Fig. 10 table): before damage the reaction
    is the load over the closed-form compliance of a 100 mm bar of section
    10 with the 2 mm defect at 0.9 of it, 98/(10 E) + 2/(9 E), E = 1 GPa.
    The micro-equivalent strain solves a screened-Poisson problem driven by
    the local strain, so it never exceeds the largest local strain: no Gauss
    point's history leaves kappa0 before the defect's local strain reaches
    it (load = kappa0 * 9 E * compliance)."""
    p = li.paper_bar_problem(500, 1000)
    m = p.material
    assert (m.E, m.kappa0, m.c, m.alpha, m.beta, m.R, m.eta) == (1000.0, 1e-4, 10.0, 0.99, 25.0, 0.005, 5.0)
    assert m.h == 1e-9 * m.E and p.mesh.nel == 500 and p.n_steps == 1000 and p.u_max == 0.02
    comp = 98.0 / (m.E * 10.0) + 2.0 / (m.E * 9.0)
    out = nw.run(p, n_steps=5, energy=False)
    np.testing.assert_allclose(out["reaction"], out["load"] / comp, rtol=1e-12)
    onset = m.kappa0 * 9.0 * m.E * comp
    k = int(np.floor(onset / p.load(1)))                 # last step before the local onset
    st, _ = nw.advance(p, nw.initial_state(p), p.load(k))
    assert np.all(st.kappa_hist == m.kappa0)
    np.testing.assert_allclose(nw.reaction_at(p, st), p.load(k) / comp, rtol=1e-12)
