"""Pins for the CPU oracle: what the paper and the mathematics fix, without GPU.

Each test names the pin it implements:
  P1  interaction function g(D) (Eq. A.4): g(0)=1, g(1)=R, g'<0, g' exact
  P2  damage law (Eq. A.1): D(kappa0)=0, continuity, 0<=D<1, monotone, D' exact
  P3  equivalent strain (Eq. A.3): invariance, principal-strain form, uniaxial
      stress gives the axial strain, gradient exact
  P4  elastic closed forms: 1D bar, 2D plane-strain and 3D uniaxial stress
  P4b micro-equivalent strain in a uniform bar equals the local one; around a
      weak element it decays with the closed-form ratio of the discrete
      Helmholtz recurrence and conserves its integral
  P5  patch tests on distorted meshes (linear u, constant eps_eq)
  P6  rigid-body motions give zero residual
  P7  tangent (Eq. 11a-d) = complex-step Jacobian of the residual (Eq. 11e-f);
      central finite differences as a second check
  P8  history and damage irreversible and bounded over committed steps
  P10 sparse assembly = brute-force dense sum of element blocks; dof map
  P11 dissipated energy non-negative and non-decreasing
  P11b stored energy (Eq. 1) in closed form: in homogeneous elastic states
      (uniform bar, 2D plane-strain and 3D uniaxial stress) it equals
      1/2 sigma:eps V and the external work of the reaction
  P11c stored energy derivatives: with the history frozen (no loading point)
      d Psi / d ebar is the micro-strain residual (Eq. 11f) and, with h = 0,
      d Psi / d u is the displacement residual (Eq. 11e)
  P12 increment halving: a forced halving commits the midpoint and equals
      the two sub-steps taken explicitly, each from its committed state
  P13 tangent structure: K_uu symmetric, K_ue = 0 without loading points
  P14 damaged-region volume: sum of dV over the Gauss points with D above a
      threshold equals the volume of the elements built to carry that damage
  P15 Eq. 2-literal stress (h-term in sigma): the Hessian of Eq. A.3 equals
      the complex-step derivative of its gradient; the full tangent equals
      the complex-step Jacobian of the residual; the residual is then the
      exact gradient of Eq. 1 (frozen history), the h-term included
"""
import dataclasses

import numpy as np
import pytest

import lgdm_inputs as li
from lgdm_inputs.meshes import L2, Q4, H8
from oracle import assembly as asm
from oracle import constitutive as cm
from oracle import element as el
from oracle import newton as nw

MAT = li.Material()                    # the plate/beam parameters of the configurations


# ---------------------------------------------------------------- P1, P2
def test_p1_interaction_function():
    for R, eta in [(0.005, 5.0), (0.05, 3.0), (0.2, 8.0)]:
        g0, _ = cm.interaction(np.array(0.0), R, eta)
        g1, _ = cm.interaction(np.array(1.0), R, eta)
        assert abs(g0 - 1.0) < 1e-15 and abs(g1 - R) < 1e-15
        D = np.linspace(0.0, 1.0, 101)
        _, dg = cm.interaction(D, R, eta)
        assert np.all(dg < 0.0)
        h = 1e-30
        gc, _ = cm.interaction(D + 1j * h, R, eta)
        np.testing.assert_allclose(gc.imag / h, dg, rtol=1e-14)


def test_p2_damage_law():
    k0, a, b = 1e-4, 0.99, 300.0
    D0, dD0 = cm.damage(np.array([k0, 0.5 * k0]), k0, a, b)
    assert np.all(D0 == 0.0) and np.all(dD0 == 0.0)
    Dr, _ = cm.damage(np.array(k0 * (1 + 1e-12)), k0, a, b)
    assert 0.0 <= Dr < 1e-9                               # continuous at the threshold
    kap = k0 * np.logspace(0, 4, 400)[1:]
    D, dD = cm.damage(kap, k0, a, b)
    assert np.all(D >= 0.0) and np.all(D < 1.0) and np.all(np.diff(D) > 0.0)
    assert D[-1] > 0.99                                   # tends to 1 for large kappa
    h = 1e-30 * k0
    Dc, _ = cm.damage(kap + 1j * h, k0, a, b)
    np.testing.assert_allclose(Dc.imag / h, dD, rtol=1e-13)


# ---------------------------------------------------------------- P3
def _voigt_to_tensor(v, dim):
    if dim == 2:
        exx, eyy, gxy = v
        return np.array([[exx, gxy / 2, 0.0], [gxy / 2, eyy, 0.0], [0.0, 0.0, 0.0]])
    exx, eyy, ezz, gyz, gxz, gxy = v
    return np.array([[exx, gxy / 2, gxz / 2], [gxy / 2, eyy, gyz / 2], [gxz / 2, gyz / 2, ezz]])


def _tensor_to_voigt3(t):
    return np.array([t[0, 0], t[1, 1], t[2, 2], 2 * t[1, 2], 2 * t[0, 2], 2 * t[0, 1]])


def _evm_principal(t, nu, k):
    """de Vree form written from principal strains (independent of Voigt shear)."""
    p = np.linalg.eigvalsh(t)
    I1 = p.sum()
    J2 = ((p[0] - p[1]) ** 2 + (p[1] - p[2]) ** 2 + (p[2] - p[0]) ** 2) / 6.0
    A = (k - 1) / (1 - 2 * nu)
    return A * I1 / (2 * k) + np.sqrt(A**2 * I1**2 + 12 * k * J2 / (1 + nu) ** 2) / (2 * k)


def test_p3_equivalent_strain_closed_forms():
    rng = np.random.default_rng(0)
    nu, k = 0.2, 10.0
    for _ in range(20):
        e1 = rng.uniform(1e-5, 1e-3)
        R, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        t = R @ np.diag([e1, -nu * e1, -nu * e1]) @ R.T       # rotated uniaxial stress
        eq, _ = cm.equivalent_strain(_tensor_to_voigt3(t), 3, nu, k)
        assert abs(eq - e1) <= 1e-13 * e1
    for dim in (2, 3):
        nv = 3 if dim == 2 else 6
        for _ in range(20):
            v = rng.normal(size=nv) * 1e-4
            eq, _ = cm.equivalent_strain(v, dim, nu, k)
            ref = _evm_principal(_voigt_to_tensor(v, dim), nu, k)
            assert abs(eq - ref) <= 1e-12 * abs(ref)
    # pure volumetric plane strain exx = eyy = e: I1 = 2e, J2 = e^2/3
    e = 2e-4
    eq, _ = cm.equivalent_strain(np.array([e, e, 0.0]), 2, nu, k)
    A = (k - 1) / (1 - 2 * nu)
    ref = A * 2 * e / (2 * k) + np.sqrt(A**2 * 4 * e**2 + 12 * k * e**2 / 3 / (1 + nu) ** 2) / (2 * k)
    assert abs(eq - ref) < 1e-15
    # zero strain: no square-root singularity
    eq0, d0 = cm.equivalent_strain(np.zeros(6), 3, nu, k)
    assert eq0 == 0.0 and np.all(np.isfinite(d0))


def test_p3_equivalent_strain_gradient():
    rng = np.random.default_rng(1)
    for dim, nv in [(2, 3), (3, 6)]:
        for variant in (0, 1):
            v = rng.normal(size=nv) * 1e-4
            _, d = cm.equivalent_strain(v, dim, 0.2, 10.0, variant)
            h = 1e-30
            for j in range(nv):
                vc = v.astype(complex)
                vc[j] += 1j * h
                eqc, _ = cm.equivalent_strain(vc, dim, 0.2, 10.0, variant)
                assert abs(eqc.imag / h - d[j]) <= 1e-12 * np.abs(d).max()


# ---------------------------------------------------------------- P4
def test_p4_elastic_bar_closed_form():
    p = li.bar_problem()
    out = nw.run(p, n_steps=5, energy=False)
    E = p.material.E
    compliance = 99.0 / (E * 10.0) + 1.0 / (E * 9.0)
    np.testing.assert_allclose(out["reaction"], out["load"] / compliance, rtol=1e-12)


def _no_damage(mat):
    mat = li.Material(**{**mat.__dict__})
    mat.kappa0 = 1.0
    return mat


def test_p4_uniaxial_stress_plane_strain_and_3d():
    # 2D: rollers at the bottom (u_y = 0, one node u_x = 0), top u_y = load.
    m = li.plate_q4(4, 3, 4.0, 3.0)
    inner = (m.x > 0) & (m.x < 4.0) & (m.y > 0) & (m.y < 3.0)
    m.x[inner] += 0.15 * np.sin(3 * m.y[inner])     # distorted interior, straight edges
    bottom, top = np.arange(5), 15 + np.arange(5)
    bcs = li.BCs(np.concatenate([li.node_dofs(m, bottom, 1), li.node_dofs(m, [0], 0),
                                 li.node_dofs(m, top, 1)]),
                 np.concatenate([np.zeros(5), [0.0], np.ones(5)]))
    mat = _no_damage(MAT)
    p = li.Problem("uniax2d", m, mat, bcs, u_max=3e-4, n_steps=1)
    out = nw.run(p, energy=False)
    eyy = 3e-4 / 3.0
    np.testing.assert_allclose(out["reaction"][0], mat.E / (1 - mat.nu**2) * eyy * 4.0, rtol=1e-12)
    # 3D: rollers on x=0, y=0, z=0 faces; top face u_z = load.
    m3 = li.beam_h8(3, 2, 2, 3.0, 2.0, 2.0)
    X = m3.coords()
    f = lambda mask: np.nonzero(mask)[0]
    bcs3 = li.BCs(np.concatenate([li.node_dofs(m3, f(X[:, 0] == 0), 0), li.node_dofs(m3, f(X[:, 1] == 0), 1),
                                  li.node_dofs(m3, f(X[:, 2] == 0), 2), li.node_dofs(m3, f(X[:, 2] == 2.0), 2)]),
                  np.concatenate([np.zeros(int((X[:, 0] == 0).sum() + (X[:, 1] == 0).sum() + (X[:, 2] == 0).sum())),
                                  np.ones(int((X[:, 2] == 2.0).sum()))]))
    p3 = li.Problem("uniax3d", m3, mat, bcs3, u_max=4e-4, n_steps=1)
    out3 = nw.run(p3, energy=False)
    np.testing.assert_allclose(out3["reaction"][0], mat.E * 2e-4 * 6.0, rtol=1e-12)


def test_p4b_micro_strain_uniform_and_weak_bar():
    # uniform bar: ebar equals the local strain at every node
    p = li.bar_problem(weak_factor=1.0)
    out = nw.run(p, n_steps=1, energy=False)
    U = out["state"].u.reshape(-1, 2)
    eps = np.diff(U[:, 0]) / 1.0
    np.testing.assert_allclose(U[:, 1], eps[0], rtol=1e-12)
    # weak bar before damage: decay ratio of the discrete Helmholtz recurrence
    p = li.bar_problem()
    out = nw.run(p, n_steps=1, energy=False)
    U = out["state"].u.reshape(-1, 2)
    eps = np.diff(U[:, 0])
    es, ew = eps[0], eps[50]
    np.testing.assert_allclose(ew / es, 10.0 / 9.0, rtol=1e-12)
    c, dx = p.material.c, 1.0
    s = (2 * dx / 3 + 2 * c / dx) / (c / dx - dx / 6)
    rho = (s - np.sqrt(s * s - 4)) / 2
    delta = U[:, 1] - es
    np.testing.assert_allclose(delta[54:66] / delta[53:65], rho, rtol=1e-9)
    np.testing.assert_allclose(delta[47:35:-1] / delta[48:36:-1], rho, rtol=1e-9)
    # locally symmetric about the weak element's centre x = 50.5 (ends are ~50 mm away)
    np.testing.assert_allclose(delta[51:71], delta[50:30:-1], rtol=1e-9)
    assert np.all(U[:, 1] < ew) and np.all(U[:, 1] > es)
    # integral conservation: sum_a r_e,a = int h A (ebar - eps_eq) dx = 0 at equilibrium
    t = el.element_terms(p.mesh, p.material, out["state"].u, out["state"].kappa_hist)
    total = np.sum(t["dV"] * (t["ebar"] - t["eps_eq"]))
    assert abs(total) < 1e-12 * es * 1000.0


# ---------------------------------------------------------------- P5, P6
def _distorted_patch(elem):
    if elem == Q4:
        m = li.plate_q4(2, 2, 2.0, 2.0)
        m.x[4] += 0.23
        m.y[4] -= 0.17
        m.x[1] += 0.1
        m.y[3] += 0.08
        return m
    m = li.beam_h8(2, 2, 2, 2.0, 2.0, 2.0)
    centre = 13                                   # node (1,1,1)
    m.x[centre] += 0.2
    m.y[centre] -= 0.15
    m.z[centre] += 0.1
    m.x[4] += 0.07
    m.z[10] -= 0.05
    return m


@pytest.mark.parametrize("elem", [Q4, H8])
def test_p5_patch_test(elem):
    m = _distorted_patch(elem)
    d = m.dim
    mat = _no_damage(MAT)
    rng = np.random.default_rng(2)
    G = rng.normal(size=(d, d)) * 1e-4
    X = m.coords()
    U = np.zeros((m.nnode, m.nd))
    U[:, :d] = X @ G.T + rng.normal(size=d) * 1e-3
    strain = G + G.T
    voigt = (np.array([G[0, 0], G[1, 1], strain[0, 1]]) if d == 2 else
             np.array([G[0, 0], G[1, 1], G[2, 2], strain[1, 2], strain[0, 2], strain[0, 1]]))
    eq, _ = cm.equivalent_strain(voigt, d, mat.nu, mat.k)
    U[:, d] = eq
    kh = np.full(m.nel * m.ngp, mat.kappa0)
    _, r = asm.assemble(m, mat, U.ravel(), kh)
    R = r.reshape(m.nnode, m.nd)
    interior = 4 if elem == Q4 else 13
    scale = mat.E * 1e-4
    assert np.abs(R[interior, :d]).max() < 1e-12 * scale
    assert np.abs(R[:, d]).max() < 1e-12 * mat.h * 1e-4


@pytest.mark.parametrize("elem", [L2, Q4, H8])
def test_p6_rigid_body(elem):
    m = li.bar_l2(3, 3.0, 2.0) if elem == L2 else _distorted_patch(elem)
    d = m.dim
    X = m.coords()
    U = np.zeros((m.nnode, m.nd))
    t = np.array([1e-3, -2e-3, 5e-4])[:d]
    if d == 1:
        U[:, 0] = t[0]
    elif d == 2:
        U[:, :2] = t + 1e-3 * np.stack([-X[:, 1], X[:, 0]], 1)
    else:
        w = np.array([1e-3, -2e-3, 1.5e-3])
        U[:, :3] = t + np.cross(w, X)
    kh = np.full(m.nel * m.ngp, MAT.kappa0)
    _, r = asm.assemble(m, MAT, U.ravel(), kh)
    assert np.abs(r).max() < 1e-12 * MAT.E * 1e-3


# ---------------------------------------------------------------- P7
def _small_meshes():
    yield li.bar_l2(4, 4.0, 10.0)
    q = li.plate_q4(3, 2, 3.0, 2.0)
    q.x = q.x + 0.1 * q.y ** 2
    q.e_scale[1] = 1e-6
    yield q
    h = li.beam_h8(2, 2, 1, 2.0, 2.0, 1.0)
    h.z = h.z + 0.05 * h.x
    yield h


def _blocks(mesh, K):
    is_e = (np.arange(mesh.ndof) % mesh.nd) == mesh.dim
    iu, ie = np.nonzero(~is_e)[0], np.nonzero(is_e)[0]
    return {"uu": K[np.ix_(iu, iu)], "ue": K[np.ix_(iu, ie)], "eu": K[np.ix_(ie, iu)], "ee": K[np.ix_(ie, ie)]}


@pytest.mark.parametrize("mi", [0, 1, 2])
def test_p7_tangent_is_complex_step_jacobian(mi):
    mesh = list(_small_meshes())[mi]
    mat = MAT if mesh.dim > 1 else li.Material(nu=0.0, k=1.0)
    u, kh = li.random_state(mesh, seed=10 + mi, kappa0=mat.kappa0)
    K, r = asm.assemble(mesh, mat, u, kh)
    K = K.toarray()
    h = 1e-30
    J = np.empty_like(K)
    for j in range(mesh.ndof):
        uc = u.astype(complex)
        uc[j] += 1j * h
        _, rc = asm.assemble(mesh, mat, uc, kh, with_tangent=False)
        J[:, j] = rc.imag / h
    t = el.element_terms(mesh, mat, u, kh)
    assert 0 < t["chi"].sum() < t["chi"].size and np.any(t["D"] > 0)   # mixed loading/unloading
    bk, bj = _blocks(mesh, K), _blocks(mesh, J)
    for name in bk:
        scale = np.abs(bj[name]).max()
        if scale == 0.0:
            assert np.abs(bk[name]).max() == 0.0
            continue
        assert np.abs(bk[name] - bj[name]).max() <= 1e-10 * scale, name
    # central finite differences as a second, cruder check
    j = 1
    du = 1e-7 * max(np.abs(u).max(), 1e-4)
    up, um = u.copy(), u.copy()
    up[j] += du
    um[j] -= du
    _, rp = asm.assemble(mesh, mat, up, kh, with_tangent=False)
    _, rm = asm.assemble(mesh, mat, um, kh, with_tangent=False)
    fd = (rp - rm) / (2 * du)
    assert np.abs(fd - K[:, j]).max() <= 1e-5 * np.abs(K[:, j]).max()


# ---------------------------------------------------------------- P10
def test_p10_assembly_against_dense_brute_force():
    q = li.plate_q4(2, 1, 2.0, 1.0)
    gu, ge = el.local_dofs(q, [0])
    # hand-expanded map of element 0 (nodes 0, 1, 4, 3; three dofs per node)
    assert list(gu[0]) == [0, 1, 3, 4, 12, 13, 9, 10] and list(ge[0]) == [2, 5, 14, 11]
    for mesh in list(_small_meshes()) + [q]:
        mat = MAT if mesh.dim > 1 else li.Material(nu=0.0, k=1.0)
        u, kh = li.random_state(mesh, seed=3, kappa0=mat.kappa0)
        K, r = asm.assemble(mesh, mat, u, kh)
        t = el.element_terms(mesh, mat, u, kh)
        Ke, rl = el.element_matrix(t)
        gu, ge = el.local_dofs(mesh, np.arange(mesh.nel))
        gl = np.concatenate([gu, ge], axis=1)
        Kd = np.zeros((mesh.ndof, mesh.ndof))
        rd = np.zeros(mesh.ndof)
        for e in range(mesh.nel):
            for i in range(gl.shape[1]):
                rd[gl[e, i]] += rl[e, i]
                for j in range(gl.shape[1]):
                    Kd[gl[e, i], gl[e, j]] += Ke[e, i, j]
        assert np.abs(K.toarray() - Kd).max() <= 1e-15 * np.abs(Kd).max()
        assert np.abs(r - rd).max() <= 1e-15 * np.abs(rd).max()


# ---------------------------------------------------------------- P8, P11
@pytest.fixture(scope="module")
def bar_run():
    p = li.bar_problem()
    state = nw.initial_state(p)
    hist, Ds, reac, loads, psis = [], [], [], [], []
    for n in range(1, p.n_steps + 1):
        state, _ = nw.advance(p, state, p.load(n))
        hist.append(state.kappa_hist.copy())
        Ds.append(cm.damage(state.kappa_hist, p.material.kappa0, p.material.alpha, p.material.beta)[0])
        reac.append(nw.reaction_at(p, state))
        loads.append(state.load)
        psis.append(nw.free_energy(p, state))
    return p, np.array(hist), np.array(Ds), np.array(reac), np.array(loads), np.array(psis)


def test_p8_history_and_damage_irreversible(bar_run):
    p, hist, Ds, *_ = bar_run
    assert np.all(np.diff(hist, axis=0) >= 0.0)
    assert np.all(np.diff(Ds, axis=0) >= 0.0)
    assert np.all(Ds >= 0.0) and np.all(Ds < 1.0)
    assert np.all(Ds[hist == p.material.kappa0] == 0.0)
    assert Ds[-1].max() > 0.9                      # the bar does localise and soften


def test_p11_dissipated_energy(bar_run):
    p, _, _, reac, loads, psi = bar_run
    lp = np.concatenate([[0.0], loads])
    rp = np.concatenate([[0.0], reac])
    w_ext = np.cumsum(0.5 * (rp[1:] + rp[:-1]) * np.diff(lp))
    Ed = w_ext - psi
    scale = w_ext[-1]
    assert np.all(Ed >= -1e-6 * scale)
    assert np.all(np.diff(Ed) >= -1e-6 * scale)
    assert Ed[-1] > 0.5 * scale                    # most of the work is dissipated after failure


# ---------------------------------------------------------------- P13
@pytest.mark.parametrize("mi", [1, 2])
def test_p13_tangent_structure(mi):
    mesh = list(_small_meshes())[mi]
    u, kh = li.random_state(mesh, seed=5, kappa0=MAT.kappa0)
    K, _ = asm.assemble(mesh, MAT, u, kh)
    b = _blocks(mesh, K.toarray())
    assert np.abs(b["uu"] - b["uu"].T).max() <= 1e-14 * np.abs(b["uu"]).max()
    kh_un = np.full_like(kh, 10 * np.abs(u).max())                 # every point unloading
    K2, _ = asm.assemble(mesh, MAT, u, kh_un)
    b2 = _blocks(mesh, K2.toarray())
    assert np.abs(b2["ue"]).max() == 0.0
    assert np.abs(b2["ee"] - b2["ee"].T).max() <= 1e-14 * np.abs(b2["ee"]).max()


def test_secant_tangent_same_residual_and_root():
    """The secant tangent (loading indicator chi = 0, i.e. the D'(kappa) terms
    of Eq. 11b and 11d dropped) changes the Jacobian only: with the history
    raised to the trial value max(kappa_hist, ebar) chi vanishes while kappa,
    D and therefore the residual stay the same.  Iterating with it converges
    (linearly) to the root exact Newton finds, here on a notched plate in its
    first, damaging load step."""
    p = li.sen_plate_problem(12, 12, n_steps=100)
    m, mat = p.mesh, p.material
    st = nw.initial_state(p)
    u0 = st.u.copy()
    u0[p.bcs.dir_dof] = p.bcs.dir_scale * p.load(1)
    isd = (np.arange(m.ndof) % m.nd) == m.dim

    def system(u, secant):
        kh = np.maximum(st.kappa_hist, el.gp_ebar(m, u).ravel()) if secant else st.kappa_hist
        K, r = asm.assemble(m, mat, u, kh)
        return asm.apply_dirichlet(K, r, p.bcs.dir_dof), r

    def solve(secant):
        import scipy.sparse.linalg as spla
        u = u0.copy()
        for k in range(40):
            (Kb, rb), _ = system(u, secant)
            du = spla.spsolve(Kb.tocsc(), -rb)
            u += du
            if (np.linalg.norm(du[~isd]) <= 1e-12 * np.linalg.norm(u[~isd])
                    and np.linalg.norm(du[isd]) <= 1e-12 * np.linalg.norm(u[isd])):
                return u, k + 1
        raise AssertionError("no convergence")

    # same residual, different tangent, at a damaging trial state
    (_, _), r_c = system(u0 * 1.0, False)
    (_, _), r_s = system(u0 * 1.0, True)
    np.testing.assert_array_equal(r_c, r_s)
    u_n, it_n = solve(False)
    u_s, it_s = solve(True)
    D, _ = cm.damage(np.maximum(st.kappa_hist, el.gp_ebar(m, u_n).ravel()), mat.kappa0, mat.alpha, mat.beta)
    assert D.max() > 0.0 and np.count_nonzero(D) > 0       # the step damages the notch tip
    assert it_s > it_n                                     # linear against quadratic convergence
    assert np.abs(u_s - u_n).max() <= 1e-9 * np.abs(u_n).max()


# ---------------------------------------------------------------- P11b, P11c
def _trapezoid_work(loads, reactions):
    lp = np.concatenate([[0.0], loads])
    rp = np.concatenate([[0.0], reactions])
    return np.cumsum(0.5 * (rp[1:] + rp[:-1]) * np.diff(lp))


def test_p11b_stored_energy_closed_forms():
    """Homogeneous elastic states: the micro-strain equals the (uniform) local
    equivalent strain, so the h-terms of Eq. 1 vanish and Psi = 1/2 sigma eps V
    exactly; the response is linear, so the trapezoid external work of the
    reaction is exact and equals Psi too."""
    # uniform bar: Psi = 1/2 E A L eps^2
    p = li.bar_problem(weak_factor=1.0, n_steps=200)
    out = nw.run(p, n_steps=3)
    eps = out["load"] / 100.0
    closed = 0.5 * p.material.E * 10.0 * 100.0 * eps ** 2
    np.testing.assert_allclose(out["psi"], closed, rtol=1e-12)
    np.testing.assert_allclose(_trapezoid_work(out["load"], out["reaction"]), closed, rtol=1e-12)
    # plane strain, uniaxial stress (distorted interior): Psi = 1/2 E/(1-nu^2) eps_yy^2 V
    m = li.plate_q4(4, 3, 4.0, 3.0)
    inner = (m.x > 0) & (m.x < 4.0) & (m.y > 0) & (m.y < 3.0)
    m.x[inner] += 0.15 * np.sin(3 * m.y[inner])
    bottom, top = np.arange(5), 15 + np.arange(5)
    left = np.arange(4) * 5
    bcs = li.BCs(np.concatenate([li.node_dofs(m, bottom, 1), li.node_dofs(m, left, 0),
                                 li.node_dofs(m, top, 1)]),
                 np.concatenate([np.zeros(5), np.zeros(4), np.ones(5)]))
    mat = _no_damage(MAT)
    p2 = li.Problem("uniax2d", m, mat, bcs, u_max=3e-4, n_steps=3)
    out = nw.run(p2)
    eyy = out["load"] / 3.0
    closed = 0.5 * mat.E / (1 - mat.nu ** 2) * eyy ** 2 * 12.0
    np.testing.assert_allclose(out["psi"], closed, rtol=1e-12)
    np.testing.assert_allclose(_trapezoid_work(out["load"], out["reaction"]), closed, rtol=1e-12)
    # 3D uniaxial stress: Psi = 1/2 E eps_zz^2 V
    m3 = li.beam_h8(3, 2, 2, 3.0, 2.0, 2.0)
    X = m3.coords()
    f = lambda mask: np.nonzero(mask)[0]
    groups = [(f(X[:, 0] == 0), 0, 0.0), (f(X[:, 1] == 0), 1, 0.0), (f(X[:, 2] == 0), 2, 0.0),
              (f(X[:, 2] == 2.0), 2, 1.0)]
    bcs3 = li.BCs(np.concatenate([li.node_dofs(m3, n, c) for n, c, _ in groups]),
                  np.concatenate([np.full(len(n), v) for n, _, v in groups]))
    p3 = li.Problem("uniax3d", m3, mat, bcs3, u_max=4e-4, n_steps=3)
    out = nw.run(p3)
    ezz = out["load"] / 2.0
    closed = 0.5 * mat.E * ezz ** 2 * 12.0
    np.testing.assert_allclose(out["psi"], closed, rtol=1e-12)
    np.testing.assert_allclose(_trapezoid_work(out["load"], out["reaction"]), closed, rtol=1e-12)


@pytest.mark.parametrize("mi", [0, 1, 2])
def test_p11c_stored_energy_gradient_is_residual(mi):
    """With kappa_hist above every micro-strain (chi = 0) D and g are fixed, so
    Eq. 1 is a function of u and ebar whose partial derivatives are the
    residuals: d Psi / d ebar_a = r_e[a] (the N h (ebar - eps_eq) and
    g h c grad(ebar) terms, Eq. 11f) and, with h = 0, d Psi / d u = r_u
    (the (1 - D) C eps term, Eq. 11e).  Complex-step derivatives."""
    mesh = list(_small_meshes())[mi]
    base = MAT if mesh.dim > 1 else li.Material(nu=0.0, k=1.0)
    u, kh = li.random_state(mesh, seed=40 + mi, kappa0=base.kappa0)
    ebar = el.gp_ebar(mesh, u).ravel()
    kh = np.maximum(kh, ebar + 0.1 * base.kappa0)               # no loading point
    assert np.any(kh > base.kappa0)                             # damaged points present
    is_e = (np.arange(mesh.ndof) % mesh.nd) == mesh.dim
    for mat, dofs, part in ((base, np.nonzero(is_e)[0], "e"),
                            (dataclasses.replace(base, h=0.0), np.nonzero(~is_e)[0], "u")):
        prob = li.Problem("p11c", mesh, mat, li.BCs(np.zeros(0, np.int32), np.zeros(0)), 1.0, 1)
        _, r = asm.assemble(mesh, mat, u, kh, with_tangent=False)
        hstep = 1e-30
        grad = np.empty(len(dofs))
        for k, j in enumerate(dofs):
            uc = u.astype(complex)
            uc[j] += 1j * hstep
            grad[k] = nw.free_energy(prob, nw.State(uc, kh)).imag / hstep
        ref = r[dofs]
        assert np.abs(ref).max() > 0.0
        assert np.abs(grad - ref).max() <= 1e-10 * np.abs(ref).max(), part


# ---------------------------------------------------------------- P12
def test_p12_forced_halving_equals_explicit_substeps():
    """Plate 10 x 10, 30 load steps: step 5 needs 24 Newton iterations from the
    committed state of step 4.  With max_newton = 16 the full increment fails
    and is halved once; the result must be the midpoint step committed and
    then the target step, each started from the committed state before it."""
    p = li.sen_plate_problem(10, 10, n_steps=30)
    st = nw.initial_state(p)
    for n in range(1, 5):
        st, _ = nw.advance(p, st, p.load(n))
    q = dataclasses.replace(p, max_newton=16)
    halved, its = nw.advance(q, st, q.load(5))
    assert len(its) == 3 and its[0] == 16 and max(its[1:]) < 16     # one failure, two sub-steps
    mid = 0.5 * (p.load(4) + p.load(5))
    u1, _ = nw.newton(q, st, mid)
    s1 = nw.commit(q, st, u1, mid)
    u2, _ = nw.newton(q, s1, q.load(5))
    s2 = nw.commit(q, s1, u2, q.load(5))
    assert halved.load == q.load(5)
    np.testing.assert_allclose(halved.u, s2.u, rtol=0, atol=1e-12 * np.abs(s2.u).max())
    np.testing.assert_allclose(halved.kappa_hist, s2.kappa_hist, rtol=1e-12)
    assert np.any(s1.kappa_hist > st.kappa_hist)                   # the midpoint commit moved the history
    # the unhalved step needs 24 iterations; its state differs from the halved
    # one because the committed midpoint raised the history (Eq. A.2) at
    # points that unload afterwards: the response is path dependent
    _, its_full = nw.advance(p, st, p.load(5))
    assert its_full == [24]


# ---------------------------------------------------------------- P14
def test_p14_damaged_volume():
    """Plate 6 x 4 on 60 x 40 mm with skewed interior nodes: the history of
    the Gauss points of a chosen set of elements is put where D > 0.9 and
    every other point below; the damaged volume is the area of that set
    (the shoelace area of each element), and 0 or the whole area at the
    extreme thresholds."""
    m = li.plate_q4(6, 4, 60.0, 40.0)
    inner = (m.x > 0) & (m.x < 60.0) & (m.y > 0) & (m.y < 40.0)
    m.x[inner] += 2.0 * np.sin(m.y[inner])
    mat = MAT
    p = li.Problem("p14", m, mat, li.BCs(np.zeros(0, np.int32), np.zeros(0)), 1.0, 1)
    chosen = np.array([2, 3, 9, 14, 15, 20])
    kh = np.full((m.nel, m.ngp), 1.5 * mat.kappa0)                # D small
    kh[chosen] = 200.0 * mat.kappa0                                # D > 0.9
    D, _ = cm.damage(kh, mat.kappa0, mat.alpha, mat.beta)
    assert D[chosen].min() > 0.9 and np.delete(D, chosen, axis=0).max() < 0.9
    st = nw.State(np.zeros(m.ndof), kh.ravel())
    X = m.coords()

    def area(e):
        xy = X[m.conn[e]]
        return 0.5 * abs(np.dot(xy[:, 0], np.roll(xy[:, 1], -1)) - np.dot(xy[:, 1], np.roll(xy[:, 0], -1)))

    np.testing.assert_allclose(nw.damaged_volume(p, st, 0.9), sum(area(e) for e in chosen), rtol=1e-13)
    np.testing.assert_allclose(nw.damaged_volume(p, st, 0.0), 2400.0, rtol=1e-13)
    assert nw.damaged_volume(p, st, 0.999999) == 0.0


# ---------------------------------------------------------------- P15
@pytest.mark.parametrize("dim,variant", [(2, 0), (3, 0), (3, 1)])
def test_p15_equivalent_strain_hessian(dim, variant):
    rng = np.random.default_rng(7 + dim + variant)
    nv = 3 if dim == 2 else 6
    for _ in range(5):
        v = rng.normal(size=nv) * 1e-4
        H = cm.equivalent_strain_hessian(v, dim, 0.2, 10.0, variant)
        hs = 1e-30
        for j in range(nv):
            vc = v.astype(complex)
            vc[j] += 1j * hs
            _, dc = cm.equivalent_strain(vc, dim, 0.2, 10.0, variant)
            assert np.abs(dc.imag / hs - H[:, j]).max() <= 1e-9 * np.abs(H).max()
        assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()


def _h_material(dim):
    base = MAT if dim > 1 else li.Material(nu=0.0, k=1.0)
    return dataclasses.replace(base, h=0.05 * base.E, h_stress=1)


@pytest.mark.parametrize("mi", [0, 1, 2])
def test_p15_literal_stress_tangent_is_complex_step_jacobian(mi):
    mesh = list(_small_meshes())[mi]
    mat = _h_material(mesh.dim)
    u, kh = li.random_state(mesh, seed=60 + mi, kappa0=mat.kappa0)
    K, r = asm.assemble(mesh, mat, u, kh)
    K = K.toarray()
    hs = 1e-30
    J = np.empty_like(K)
    for j in range(mesh.ndof):
        uc = u.astype(complex)
        uc[j] += 1j * hs
        _, rc = asm.assemble(mesh, mat, uc, kh, with_tangent=False)
        J[:, j] = rc.imag / hs
    bk, bj = _blocks(mesh, K), _blocks(mesh, J)
    for name in bk:
        scale = np.abs(bj[name]).max()
        assert scale > 0.0
        assert np.abs(bk[name] - bj[name]).max() <= 1e-10 * scale, name
    # the variant changes the displacement blocks and the residual
    K0, r0 = asm.assemble(mesh, dataclasses.replace(mat, h_stress=0), u, kh)
    b0 = _blocks(mesh, K0.toarray())
    assert np.abs(b0["uu"] - bk["uu"]).max() > 1e-3 * np.abs(bk["uu"]).max()
    assert np.abs(r0 - r).max() > 1e-3 * np.abs(r).max()


@pytest.mark.parametrize("mi", [1, 2])
def test_p15_literal_stress_residual_is_energy_gradient(mi):
    """With the h-term in the stress, the coupled residual is the exact
    gradient of Eq. 1 at a frozen history (no loading point): d Psi / d u =
    r_u and d Psi / d ebar = r_e, with h far from negligible."""
    mesh = list(_small_meshes())[mi]
    mat = _h_material(mesh.dim)
    u, kh = li.random_state(mesh, seed=70 + mi, kappa0=mat.kappa0)
    ebar = el.gp_ebar(mesh, u).ravel()
    kh = np.maximum(kh, ebar + 0.1 * mat.kappa0)
    prob = li.Problem("p15", mesh, mat, li.BCs(np.zeros(0, np.int32), np.zeros(0)), 1.0, 1)
    _, r = asm.assemble(mesh, mat, u, kh, with_tangent=False)
    hs = 1e-30
    grad = np.empty(mesh.ndof)
    for j in range(mesh.ndof):
        uc = u.astype(complex)
        uc[j] += 1j * hs
        grad[j] = nw.free_energy(prob, nw.State(uc, kh)).imag / hs
    assert np.abs(grad - r).max() <= 1e-10 * np.abs(r).max()
