"""Batched execution: uneven meshes in one persistent element launch, grouped
Krylov solves, a CUDA graph per Newton step.

Every member's results must be bitwise those of the same simulation run
alone (same options), whatever the mix, the tuning or the graph setting.
"""
import numpy as np
import pytest

import lgdm_inputs as li

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problems():
    rng = np.random.default_rng(5)
    out = []
    for n in (9, 14, 21, 12):
        mat = li.Material(kappa0=rng.uniform(0.8e-4, 1.5e-4), beta=rng.uniform(200, 500),
                          eta=rng.uniform(3, 8), c=rng.uniform(0.5, 4.0))
        out.append(li.sen_plate_problem(n, n, notch_frac=rng.uniform(0.2, 0.6), n_steps=60, material=mat))
    out.append(li.tpb_beam_problem(12, 3, 4, 120.0, 30.0, 40.0, n_steps=40))
    return out


def _alone(p, steps, **kw):
    from paper_2301_06503_gb300 import Sim
    s = Sim(p.mesh, p.material, p.bcs, stream=torch.cuda.Stream(), **kw)
    reac, its = s.run([p.load(n) for n in range(1, steps + 1)])
    u = s.field("u")
    kh = s.field("kappa_hist")
    s.close()
    return reac, its, u, kh


@pytest.mark.parametrize("graph", [True, False])
def test_batch_members_equal_alone_bitwise(graph):
    from paper_2301_06503_gb300 import Batch, Sim
    probs = _problems()
    steps = 8
    stream = torch.cuda.Stream()                 # capture needs a created stream
    sims = [Sim(p.mesh, p.material, p.bcs, stream=stream) for p in probs]
    b = Batch(sims)
    b.set_tuning(block_threads=64, grid_factor=1, graph=graph)
    reac = np.zeros((steps, len(probs)))
    for n in range(1, steps + 1):
        its, st = b.run_step([p.load(n) for p in probs])
        assert np.all(st == 0)
        reac[n - 1] = [s.reaction() for s in sims]
    fields = [(s.field("u"), s.field("kappa_hist")) for s in sims]
    tuning = b.tuning()
    note = b._lib.lgdm_batch_last_error(b.h)
    b.close()
    for s in sims:
        s.close()
    if graph:
        assert tuning["graph"] in (1, 2), note
    for j, p in enumerate(probs):
        r1, _, u1, k1 = _alone(p, steps)
        assert np.array_equal(reac[:, j], r1), j
        assert np.array_equal(fields[j][0], u1) and np.array_equal(fields[j][1], k1), j


def test_batch_subset_and_autotune():
    """A member sitting out a step (NaN load) and the autotuner's choice leave
    the other members' results unchanged."""
    from paper_2301_06503_gb300 import Batch, Sim
    probs = _problems()[:3]
    stream = torch.cuda.Stream()
    sims = [Sim(p.mesh, p.material, p.bcs, stream=stream) for p in probs]
    b = Batch(sims)
    choice = b.autotune()
    assert choice["block_threads"] in (64, 128, 256) and 1 <= choice["grid_factor"] <= 8
    for s in sims:
        s.reset_state()
    loads1 = [probs[0].load(1), float("nan"), probs[2].load(1)]
    b.run_step(loads1)
    b.run_step([p.load(k) for p, k in zip(probs, (2, 1, 2))])
    got = [s.reaction() for s in sims]
    b.close()
    for s in sims:
        s.close()
    for j, steps in ((0, 2), (1, 1), (2, 2)):
        r1, *_ = _alone(probs[j], steps)
        assert got[j] == r1[-1], j


def test_batch_fp32_tangent_members():
    from paper_2301_06503_gb300 import Batch, Sim
    probs = _problems()[:2]
    stream = torch.cuda.Stream()
    sims = [Sim(p.mesh, p.material, p.bcs, precision="fp32", stream=stream) for p in probs]
    b = Batch(sims)
    for n in range(1, 5):
        b.run_step([p.load(n) for p in probs])
    got = [s.reaction() for s in sims]
    b.close()
    for s in sims:
        s.close()
    for j, p in enumerate(probs):
        r1, *_ = _alone(p, 4, precision="fp32")
        assert got[j] == r1[-1]


def test_batch_mixing_stress_variants_equals_alone():
    """A batch whose members use both stress forms (one element kernel per
    element type and variant): every member bitwise equal to itself alone."""
    import dataclasses
    from paper_2301_06503_gb300 import Batch, Sim
    probs = _problems()[:3]
    probs[1] = dataclasses.replace(probs[1], material=dataclasses.replace(probs[1].material, h=1e-3 * 20000.0,
                                                                          h_stress=1))
    stream = torch.cuda.Stream()
    sims = [Sim(p.mesh, p.material, p.bcs, stream=stream) for p in probs]
    b = Batch(sims)
    steps = 4
    reac = np.zeros((steps, len(probs)))
    for n in range(1, steps + 1):
        its, st = b.run_step([p.load(n) for p in probs])
        assert np.all(st == 0)
        reac[n - 1] = [s.reaction() for s in sims]
    b.close()
    for s in sims:
        s.close()
    for j, p in enumerate(probs):
        r1, _, _, _ = _alone(p, steps)
        assert np.array_equal(reac[:, j], r1), j
