"""The seeded inputs have the sizes and structure of the benchmark
configurations: element, node and dof counts, notches, load schedules,
the batch draw and the serving trace (host only)."""
import numpy as np

import lgdm_inputs as li


def test_bar_plate_beam_sizes():
    b = li.bar_problem()
    assert (b.mesh.nel, b.mesh.nnode, b.mesh.ndof, b.n_steps) == (100, 101, 202, 200)
    assert abs(b.load(b.n_steps) - 0.02) < 1e-15
    p = li.sen_plate_problem()
    assert (p.mesh.nel, p.mesh.nnode, p.mesh.ndof, p.n_steps) == (40000, 40401, 121203, 500)
    assert abs(p.load(p.n_steps) - 0.1) < 1e-15
    assert np.count_nonzero(p.mesh.e_scale < 1.0) == 100          # the 50 mm notch row
    t = li.tpb_beam_problem()
    assert (t.mesh.nel, t.mesh.nnode, t.mesh.ndof, t.n_steps) == (320000, 337881, 1351524, 300)
    assert np.count_nonzero(t.mesh.e_scale < 1.0) == 20 * 40       # one column, 20 layers deep, full width


def test_batch_draw_is_seeded_and_in_range():
    a = li.batch_plate_problems()
    b = li.batch_plate_problems()
    assert len(a) == 256
    n = np.array([int(round(np.sqrt(p.mesh.nel))) for p in a])
    assert n.min() >= 20 and n.max() <= 300
    assert [p.mesh.nel for p in a] == [p.mesh.nel for p in b]      # same seed, same draw
    for p in a[:32]:
        m = p.material
        assert 0.8e-4 <= m.kappa0 <= 1.5e-4 and 200 <= m.beta <= 500 and 3 <= m.eta <= 8 and 0.5 <= m.c <= 4


def test_serving_trace_mix_and_arrivals():
    tr = li.serving_trace()
    assert len(tr) == 400
    arr = np.array([r.arrival for r in tr])
    assert np.all(np.diff(arr) > 0)
    assert 10.0 < arr[-1] < 30.0                                   # Poisson at 20/s: about 20 s
    plates = sum(1 for r in tr if r.problem.mesh.elem == 2)
    assert 0.6 < plates / len(tr) < 0.8                            # 70 % plates
    beams = [r.problem.mesh for r in tr if r.problem.mesh.elem == 3]
    assert min(m.nel for m in beams) >= 40 * 8 * 8 and max(m.nel for m in beams) <= 160 * 32 * 32
