"""Failure detection, increment halving, checkpoint/resume and the committed-
state outputs of the library, against the CPU oracle.

The failures are made on the host or through bounded device waits: a NaN
refused by the host-side check, a NaN written into the device state by the
library's injection hook, iteration limits that Newton cannot meet, and a grid
barrier that waits for a block that is never launched (each wait gives up
after a 1 ms limit and the launch returns).  No test faults the GPU.
"""
import dataclasses
import json
import os
import time

import numpy as np
import pytest

import lgdm_inputs as li
from _parity import oracle_system
from oracle import newton as nw

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NOT_CONVERGED, NONFINITE, TIMEOUT = 4, 5, 6
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _sim(problem, **kw):
    from paper_2301_06503_gb300 import Sim
    return Sim(problem.mesh, problem.material, problem.bcs, **kw)


def _status(excinfo):
    return excinfo.value.status


def test_set_state_rejects_nonfinite_on_host():
    from paper_2301_06503_gb300._lib import LgdmError
    p = li.sen_plate_problem(9, 7)
    u, kh = li.random_state(p.mesh, seed=3, kappa0=p.material.kappa0)
    s = _sim(p)
    s.set_state(u, kh)
    bad = u.copy()
    bad[5] = np.nan
    with pytest.raises(LgdmError) as ei:
        s.set_state(bad, None)
    assert _status(ei) == NONFINITE
    kbad = kh.copy()
    kbad[-1] = np.inf
    with pytest.raises(LgdmError) as ei:
        s.set_state(None, kbad)
    assert _status(ei) == NONFINITE
    np.testing.assert_array_equal(s.field("u"), u)               # state untouched
    np.testing.assert_array_equal(s.field("kappa_hist"), kh)
    s.close()


def test_nan_in_device_state_is_reported_then_halving_recovers():
    """A NaN in the device dofs makes the solve's right-hand side non-finite:
    lgdm_newton_step returns LGDM_ERR_NONFINITE.  lgdm_run_step treats it like
    a diverged iteration: it halves the increment from the clean committed
    state and completes the step (elastic bar: the halved step reaches the
    same state as the oracle's unhalved one)."""
    from paper_2301_06503_gb300._lib import LgdmError, FAULT_NAN_STATE
    p = li.bar_problem()
    s = _sim(p)
    s.begin_step(p.load(1))
    s.inject_fault(FAULT_NAN_STATE)
    with pytest.raises(LgdmError) as ei:
        s.newton_step()
    assert _status(ei) == NONFINITE
    s.reset_state()
    s.run_step(p.load(1))
    s.run_step(p.load(2))
    s.inject_fault(FAULT_NAN_STATE)
    s.run_step(p.load(3))
    assert s.counters()["halvings"] == 1
    ref = nw.run(p, n_steps=3, energy=False)
    assert abs(s.reaction() - ref["reaction"][-1]) <= 1e-10 * abs(ref["reaction"][-1])
    s.close()


def test_newton_limits_give_not_converged_and_keep_committed_state():
    """max_newton = 1 and no halving on the first, damaging step of a notched
    plate: Newton cannot meet its test in one iteration, the call returns
    LGDM_ERR_NOT_CONVERGED and the dofs are back at the committed state."""
    from paper_2301_06503_gb300._lib import LgdmError
    p = li.sen_plate_problem(10, 10, n_steps=30)
    s = _sim(p, max_newton=1, max_halvings=0)
    with pytest.raises(LgdmError) as ei:
        s.run_step(p.load(1))
    assert _status(ei) == NOT_CONVERGED
    assert np.all(s.field("u") == 0.0)
    assert np.all(s.field("kappa_hist") == p.material.kappa0)
    s.close()


def test_grid_barrier_timeout_is_reported_and_context_stays_usable():
    """The injected launch waits at its first grid barrier for one block more
    than it launched; every wait gives up after wait_limit_s = 1 ms, the
    launch returns, lgdm_solve reports LGDM_ERR_TIMEOUT.  The next solve on
    the same context is correct."""
    import scipy.sparse.linalg as spla
    from paper_2301_06503_gb300._lib import LgdmError, FAULT_BARRIER_TIMEOUT
    p = li.sen_plate_problem(17, 11)
    u, _ = li.random_state(p.mesh, seed=21, kappa0=p.material.kappa0, strain=2e-5)
    kh = np.full(p.mesh.nel * p.mesh.ngp, 1.0)
    s = _sim(p, krylov_rtol=1e-12, krylov_blocks=4, wait_limit_s=1e-3)
    s.set_state(u, kh)
    s.assemble()
    s.inject_fault(FAULT_BARRIER_TIMEOUT)
    t0 = time.perf_counter()
    with pytest.raises(LgdmError) as ei:
        s.solve()
    assert _status(ei) == TIMEOUT
    assert time.perf_counter() - t0 < 1.0
    assert s.last_solve()[1] == 4
    it, rel = s.solve()
    assert rel <= 1e-12 and it > 0
    Kref, rref, _ = oracle_system(p.mesh, p.material, p.bcs, u, kh)
    xref = spla.spsolve(Kref.tocsc(), rref)
    assert np.abs(s.field("delta") - xref).max() <= 1e-9 * np.abs(xref).max()
    s.close()


def test_forced_halving_matches_oracle():
    """Plate 10 x 10, 30 load steps.  Load step 5 (damaging) is forced to halve
    once: its first Newton iteration meets an injected NaN, which the load-step
    driver treats like divergence.  The library then commits the midpoint and
    the target from the committed state before each; the oracle takes the
    same two sub-steps explicitly (Newton iteration counts of the two sides
    differ with the inexact linear solves, so an iteration cap could not force
    the same halving on both).  Curve, history and the external work (one
    curve point for the halved step) match."""
    from paper_2301_06503_gb300._lib import FAULT_NAN_STATE
    p = li.sen_plate_problem(10, 10, n_steps=30)
    st = nw.initial_state(p)
    ref = []
    for n in range(1, 5):
        st, _ = nw.advance(p, st, p.load(n))
        ref.append(nw.reaction_at(p, st))
    mid = 0.5 * (p.load(4) + p.load(5))
    u1, _ = nw.newton(p, st, mid)
    s1 = nw.commit(p, st, u1, mid)
    u2, _ = nw.newton(p, s1, p.load(5))
    s2 = nw.commit(p, s1, u2, p.load(5))
    ref.append(nw.reaction_at(p, s2))
    s = _sim(p)
    reac, _ = s.run([p.load(n) for n in range(1, 5)])
    s.inject_fault(FAULT_NAN_STATE)
    s.run_step(p.load(5))
    reac = np.append(reac, s.reaction())
    c = s.counters()
    kh = s.field("kappa_hist")
    _, w_ext, _ = s.committed()
    s.close()
    assert c["halvings"] == 1
    ref = np.asarray(ref)
    assert np.abs(reac - ref).max() <= 1e-6 * np.abs(ref).max()
    np.testing.assert_allclose(kh, s2.kappa_hist, rtol=1e-6)
    loads = np.array([p.load(n) for n in range(0, 6)])
    rp = np.concatenate([[0.0], ref])
    w_ref = np.sum(0.5 * (rp[1:] + rp[:-1]) * np.diff(loads))
    assert abs(w_ext - w_ref) <= 1e-6 * abs(w_ref)


def test_checkpoint_resume_is_exact():
    """Checkpoint after 70 load steps of the bar (past the peak), continue 20
    steps; a new simulation restored from the checkpoint continues the same
    20 steps bitwise (curve, dofs, history, external work)."""
    p = li.bar_problem()
    s = _sim(p)
    s.run([p.load(n) for n in range(1, 71)])
    ck = s.checkpoint()
    ra, _ = s.run([p.load(n) for n in range(71, 91)])
    ua, ka, ca = s.field("u"), s.field("kappa_hist"), s.committed()
    s.close()
    t = _sim(p)
    t.restore(ck)
    assert t.committed() == (ck["load"], ck["external_work"], ck["reaction"])
    rb, _ = t.run([p.load(n) for n in range(71, 91)])
    assert np.array_equal(ra, rb)
    assert np.array_equal(ua, t.field("u")) and np.array_equal(ka, t.field("kappa_hist"))
    assert t.committed() == ca
    t.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_library_energy_bookkeeping_matches_oracle(precision):
    """External work and dissipated energy kept by the library at the end
    point of every load step (R17) against the stored oracle run of the bar (200 steps)."""
    g = json.load(open(os.path.join(GOLDEN, "bar1d.json")))
    p = li.bar_problem()
    s = _sim(p, precision=precision)
    s.run(g["load"])
    load, w_ext, reac = s.committed()
    ed, psi = s.dissipated_energy()
    s.close()
    assert load == g["load"][-1]
    w_ref = g["dissipated"][-1] + g["psi"][-1]
    assert abs(w_ext - w_ref) <= 1e-6 * abs(w_ref)
    assert abs(ed - g["dissipated"][-1]) <= 1e-6 * abs(g["dissipated"][-1])
    assert abs(psi - g["psi"][-1]) <= 1e-6 * abs(w_ref)


@pytest.mark.parametrize("name", ["plate", "beam"])
def test_damaged_volume_matches_oracle(name):
    """Volume of the Gauss points above damage thresholds at a random
    history, on distorted meshes: same points selected on both sides (the
    thresholds sit away from every damage value), volumes to 1e-12."""
    from oracle import constitutive as cm
    p = (li.sen_plate_problem(13, 7) if name == "plate" else li.tpb_beam_problem(6, 5, 4, 6.0, 5.0, 4.0))
    if name == "plate":
        p.mesh.x = p.mesh.x + 0.3 * np.sin(p.mesh.y)
    else:
        p.mesh.z = p.mesh.z + 0.1 * np.cos(p.mesh.x)
    rng = np.random.default_rng(11)
    kh = p.material.kappa0 * np.exp(rng.uniform(0.0, np.log(300.0), p.mesh.nel * p.mesh.ngp))
    D, _ = cm.damage(kh, p.material.kappa0, p.material.alpha, p.material.beta)
    s = _sim(p)
    s.set_state(None, kh)
    state = nw.State(np.zeros(p.mesh.ndof), kh)
    for thr in (0.0, 0.1, 0.5, 0.9, 0.97):
        assert np.abs(D - thr).min() > 1e-9
        ref = nw.damaged_volume(p, state, thr)
        got = s.damaged_volume(thr)
        assert abs(got - ref) <= 1e-12 * max(abs(ref), 1.0), (thr, got, ref)
    s.close()
