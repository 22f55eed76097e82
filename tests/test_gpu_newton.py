"""GPU Krylov solve, Newton iterations and load stepping against the oracle.

Load-displacement curves (Algorithm 2 with the history commit of Eq. A.2)
must match the oracle to 1e-6 relative of the peak load: the 1D bar in full
(100 elements, 200 steps), reduced notched plate and notched beam.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import lgdm_inputs as li
from _parity import gpu_csr, oracle_system
from oracle import newton as nw

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sim(problem, **kw):
    from paper_2301_06503_gb300 import Sim
    return Sim(problem.mesh, problem.material, problem.bcs, **kw)


@pytest.mark.parametrize("blocks", [0, 1, 5])
def test_krylov_solution_matches_direct_solve(blocks):
    """Undamaged state (well conditioned): solution equals the direct solve."""
    p = li.sen_plate_problem(17, 11)
    u, _ = li.random_state(p.mesh, seed=21, kappa0=p.material.kappa0, strain=2e-5)
    kh = np.full(p.mesh.nel * p.mesh.ngp, 1.0)      # far above every micro-strain: no damage
    s = _sim(p, krylov_rtol=1e-12, krylov_blocks=blocks)
    s.set_state(u, kh)
    s.assemble()
    it, rel = s.solve()
    assert rel <= 1e-12 and it > 0
    x = s.field("delta")
    Kref, rref, _ = oracle_system(p.mesh, p.material, p.bcs, u, kh)
    xref = spla.spsolve(Kref.tocsc(), rref)
    assert np.abs(x - xref).max() <= 1e-9 * np.abs(xref).max()
    conv = s.update()
    assert not conv
    np.testing.assert_allclose(s.field("u"), u + x, rtol=0, atol=1e-15 * np.abs(u).max())
    s.close()


def test_krylov_true_residual_damaged_state():
    """Random damaged state (condition number ~1e11): the true residual is small."""
    p = li.sen_plate_problem(17, 11)
    u, kh = li.random_state(p.mesh, seed=21, kappa0=p.material.kappa0)
    s = _sim(p, krylov_rtol=1e-12, krylov_blocks=3)
    s.set_state(u, kh)
    s.assemble()
    it, rel = s.solve()
    assert rel <= 1e-9                   # the reported residual is the true one: b - K x
    x = s.field("delta")
    Kref, rref, _ = oracle_system(p.mesh, p.material, p.bcs, u, kh)
    true = np.linalg.norm(Kref @ x - rref) / np.linalg.norm(rref)
    assert true <= 1e-9, true
    s.close()


def test_krylov_fp32_tangent_solve():
    """Float matrix, preconditioner and SpMV; FP64 vectors and inner products."""
    p = li.sen_plate_problem(17, 11)
    u, _ = li.random_state(p.mesh, seed=22, kappa0=p.material.kappa0, strain=2e-5)
    kh = np.full(p.mesh.nel * p.mesh.ngp, 1.0)
    s = _sim(p, krylov_rtol=1e-6, krylov_blocks=4, precision="fp32")
    s.set_state(u, kh)
    s.assemble()
    it, rel = s.solve()
    assert rel <= 1e-5                    # true residual; float SpMV bounds what is attainable
    x = s.field("delta")
    Kref, rref, _ = oracle_system(p.mesh, p.material, p.bcs, u, kh)
    true = np.linalg.norm(Kref @ x - rref) / np.linalg.norm(rref)
    assert true <= 1e-5, true
    s.close()


@pytest.mark.parametrize("m", [16, 64])
def test_gmres_solution_matches_direct_solve(m):
    p = li.sen_plate_problem(17, 11)
    u, _ = li.random_state(p.mesh, seed=23, kappa0=p.material.kappa0, strain=2e-5)
    kh = np.full(p.mesh.nel * p.mesh.ngp, 1.0)
    s = _sim(p, krylov="gmres", gmres_m=m, krylov_rtol=1e-11, krylov_blocks=4)
    s.set_state(u, kh)
    s.assemble()
    it, rel = s.solve()
    assert rel <= 1e-11 and it > 0
    x = s.field("delta")
    Kref, rref, _ = oracle_system(p.mesh, p.material, p.bcs, u, kh)
    xref = spla.spsolve(Kref.tocsc(), rref)
    assert np.abs(x - xref).max() <= 1e-8 * np.abs(xref).max()
    s.close()


def test_gmres_damaged_state_true_residual():
    """On the cond ~1e11 random state the small least-squares update of GMRES
    is itself ill-conditioned; the solver must never return an iterate whose
    true residual exceeds the best one it has seen, and it reports that true
    residual."""
    p = li.sen_plate_problem(17, 11)
    u, kh = li.random_state(p.mesh, seed=21, kappa0=p.material.kappa0)
    s = _sim(p, krylov="gmres", gmres_m=128, krylov_rtol=1e-6, krylov_blocks=3, max_krylov=4000)
    s.set_state(u, kh)
    s.assemble()
    it, rel = s.solve()
    x = s.field("delta")
    Kref, rref, _ = oracle_system(p.mesh, p.material, p.bcs, u, kh)
    true = np.linalg.norm(Kref @ x - rref) / np.linalg.norm(rref)
    assert true <= 1.0 + 1e-12 and abs(true - rel) <= 1e-3 * true + 1e-12, (true, rel)
    s.close()


def test_plate_harsh_increments_with_fallback():
    """24 x 24 plate with 40 load steps (increments 12x those of the full
    workload): BiCGSTAB breaks down after damage onset and GMRES continues.
    Parity up to and including the peak (step 4); past it the coarse
    increments let exact and inexact Newton settle on different branches of
    the softening response, so only completion is checked there."""
    p = li.sen_plate_problem(24, 24, n_steps=40)
    ref, reac, its, _ = _curve_check(p, 4)
    assert reac.argmax() >= 2
    s = _sim(p)
    reac2, _ = s.run([p.load(n) for n in range(1, 13)])
    s.close()
    assert np.all(np.isfinite(reac2)) and reac2[-1] < reac2.max()


def _curve_check(p, n_steps, tol=1e-6, **kw):
    ref = nw.run(p, n_steps=n_steps, energy=False)
    s = _sim(p, **kw)
    reac, its = s.run([p.load(n) for n in range(1, n_steps + 1)])
    kh = s.field("kappa_hist")
    s.close()
    scale = np.abs(ref["reaction"]).max()
    err = np.abs(reac - ref["reaction"]).max() / scale
    assert err <= tol, (err, np.argmax(np.abs(reac - ref["reaction"])))
    return ref, reac, its, kh


def test_bar_full_curve():
    p = li.bar_problem()
    ref, reac, its, kh = _curve_check(p, p.n_steps)
    assert reac.max() > 10.0 and reac[-1] < 0.5 * reac.max()     # peak and softening reached
    # an inexact linear solve may cost one more Newton iteration per step
    assert np.all(its >= ref["newton_iters"] - 1) and its.sum() <= 1.5 * ref["newton_iters"].sum()
    np.testing.assert_allclose(kh, ref["state"].kappa_hist, rtol=1e-6)


def test_plate_reduced_curve():
    """24 x 24 notched plate, load increments of the full-size workload's order."""
    p = li.sen_plate_problem(24, 24, n_steps=200)
    ref, reac, its, _ = _curve_check(p, 40)
    assert reac.argmax() < 39                                       # past the peak


def test_beam_reduced_curve():
    p = li.tpb_beam_problem(20, 4, 6, 200.0, 40.0, 40.0, n_steps=30)
    _curve_check(p, 30)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_literal_h_stress_plate_curve(precision):
    """Eq. 2-literal stress on a 16 x 16 notched plate with h = 1e-3 E (large
    enough for the h-term to move the curve by about 1 %), 16 load steps of a
    240-step schedule (damaging, no halving): the curve matches the oracle's
    run of the same variant."""
    import dataclasses
    base = li.sen_plate_problem(16, 16, n_steps=240)
    mat = dataclasses.replace(base.material, h=1e-3 * base.material.E, h_stress=1)
    p = dataclasses.replace(base, material=mat)
    ref0 = nw.run(dataclasses.replace(p, material=dataclasses.replace(mat, h_stress=0)), n_steps=16, energy=False)
    ref, reac, its, kh = _curve_check(p, 16, precision=precision)
    assert np.abs(ref["reaction"] - ref0["reaction"]).max() > 1e-4 * np.abs(ref["reaction"]).max()
    np.testing.assert_allclose(kh, ref["state"].kappa_hist, rtol=1e-6)


def test_bar_curve_fp32_tangent():
    """Inexact Newton with the float tangent converges to the FP64 solution."""
    p = li.bar_problem()
    _curve_check(p, p.n_steps, tol=1e-6, precision="fp32")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


from _parity import ACCURACY, accuracy as _accuracy  # noqa: E402


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_full_size_plate_prefix_against_oracle(precision):
    """200 x 200 notched plate (the benchmark workload), the oracle's first 30
    load steps (damage from step 1, peak at step 27) stored by
    tests/golden/make_golden.py."""
    path = os.path.join(GOLDEN, "sen_plate_prefix.json")
    if not os.path.exists(path):
        pytest.skip("oracle golden not generated")
    g = json.load(open(path))
    p = li.sen_plate_problem()
    s = _sim(p, precision=precision)
    reac, its = s.run(g["load"])
    psi, dmg = s.energy(), s.field("damage")
    s.close()
    err = _accuracy(p, g, reac, psi, dmg)
    print(f"\naccuracy {precision} plate 200x200, 30 steps:", {k: f"{v:.2e}" for k, v in err.items()})
    for k, v in err.items():
        assert v <= ACCURACY[precision][k], (k, v)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_beam_reduced_accuracy_against_stored_oracle(precision):
    """Notched beam in three-point bending at 40 x 8 x 8 hexahedra (the 3D
    workload's geometry and material on a coarser mesh), the oracle's first 90
    of 300 load steps (peak at step 28, softening to 83 N): curve, peak load,
    dissipated energy and the final damage field (Eq. 11a-f in 3D)."""
    g = json.load(open(os.path.join(GOLDEN, "tpb_beam_40x8x8_90.json")))
    p = li.tpb_beam_problem(40, 8, 8)
    s = _sim(p, precision=precision)
    reac, its = s.run(g["load"])
    psi, dmg = s.energy(), s.field("damage")
    s.close()
    err = _accuracy(p, g, reac, psi, dmg)
    print(f"\naccuracy {precision} beam 40x8x8, 90 steps:", {k: f"{v:.2e}" for k, v in err.items()})
    for k, v in err.items():
        assert v <= ACCURACY[precision][k], (k, v)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_bar_accuracy_against_stored_oracle(precision):
    """1D bar, all 200 steps (peak and softening): peak load, dissipated
    energy and the final damage field against the stored oracle run."""
    g = json.load(open(os.path.join(GOLDEN, "bar1d.json")))
    p = li.bar_problem()
    s = _sim(p, precision=precision)
    reac, _ = s.run(g["load"])
    psi, dmg = s.energy(), s.field("damage")
    s.close()
    err = _accuracy(p, g, reac, psi, dmg)
    print(f"\naccuracy {precision} bar, 200 steps:", {k: f"{v:.2e}" for k, v in err.items()})
    for k, v in err.items():
        assert v <= ACCURACY[precision][k], (k, v)


def test_bar_curve_against_stored_oracle():
    g = json.load(open(os.path.join(GOLDEN, "bar1d.json")))
    p = li.bar_problem()
    s = _sim(p)
    reac, _ = s.run(g["load"])
    s.close()
    ref = np.asarray(g["reaction"])
    assert np.abs(reac - ref).max() <= 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("precond", ["block", "multigrid"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_secant_fallback_hard_member_against_oracle(precision, precond):
    """Plate 8 of the 256-plate batch (200 x 200), first load step: from the
    fourth Newton iteration on, the consistent tangent defeats the node-block
    Jacobi-preconditioned BiCGSTAB and GMRES; the step continues with the
    secant tangent and must reach the oracle's converged state (the oracle
    solves every tangent directly), alone and inside a batch, bitwise.  The
    multigrid preconditioner solves the consistent tangent itself; the
    converged state is the same."""
    from paper_2301_06503_gb300 import Batch, Sim
    g = json.load(open(os.path.join(GOLDEN, "batch_plate8_step1.json")))
    p = li.batch_plate_problems()[8]
    st = torch.cuda.Stream()
    s = Sim(p.mesh, p.material, p.bcs, stream=st, precision=precision, precond=precond)
    reac, its = s.run(g["load"])
    psi, dmg = s.energy(), s.field("damage")
    c = s.counters()
    s.close()
    if precond == "block":
        assert c["secant_iters"] > 0                 # the fallback was taken
    err = _accuracy(p, g, reac, psi, dmg)
    print(f"\nsecant fallback {precision} plate 8: newton {int(its[0])} secant {c['secant_iters']}",
          {k: f"{v:.2e}" for k, v in err.items()})
    for k in ("curve", "peak", "damage"):            # one step: no dissipation to speak of yet
        assert err[k] <= ACCURACY[precision][k], (k, err[k])
    # the same member inside a batch with two small plates: bitwise equal
    small = [li.sen_plate_problem(10, 10, n_steps=300, material=p.material),
             li.sen_plate_problem(16, 16, n_steps=300)]
    sims = [Sim(q.mesh, q.material, q.bcs, stream=st, precision=precision, precond=precond) for q in [p] + small]
    b = Batch(sims)
    b.run_step([q.load(1) for q in [p] + small])
    r_batch = sims[0].reaction()
    b.close()
    for x in sims:
        x.close()
    assert r_batch == reac[0]
