"""Continuous-batching server: admission by device-memory budget, resident
state, interleaved load steps, slot reuse; each result bitwise equal to the
same request run alone."""
import json
import os

import numpy as np
import pytest

import lgdm_inputs as li

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _jobs(n_steps=6):
    from paper_2301_06503_gb300.serve import Job
    # the trace's own schedule (300 increments); a job serves its first n_steps
    trace = li.serving_trace(seed=4, count=80, rate=20.0, n_steps=300)
    # the smallest plates and beams of the trace's mix keep the test short
    plates = sorted([r for r in trace if r.problem.mesh.elem == 2], key=lambda r: r.problem.mesh.nel)[:4]
    beams = sorted([r for r in trace if r.problem.mesh.elem == 3], key=lambda r: r.problem.mesh.nel)[:2]
    small = sorted(plates + beams, key=lambda r: r.arrival)
    return [Job(i, r.problem, 0.0, n_steps) for i, r in enumerate(small)]


def _alone(job, precision):
    from paper_2301_06503_gb300 import Sim
    p = job.problem
    s = Sim(p.mesh, p.material, p.bcs, stream=torch.cuda.Stream(), precision=precision)
    r, _ = s.run([p.load(n) for n in range(1, job.n_steps + 1)])
    s.close()
    return r


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_served_results_equal_alone(precision):
    from paper_2301_06503_gb300.serve import Server
    jobs = _jobs()
    srv = Server(budget_bytes=8 << 30, max_resident=3, precision=precision,    # 6 jobs, 3 slots: reuse
                 log=lambda m: print(m, flush=True))
    rep = srv.run(jobs)
    assert rep["completed"] == len(jobs) and rep["failed"] == 0
    assert srv.ticks > jobs[0].n_steps                                        # slots were reused
    for j in jobs:
        assert np.array_equal(np.asarray(j.reactions), _alone(j, precision)), j.rid


def test_admission_respects_budget():
    from paper_2301_06503_gb300.serve import Server
    from paper_2301_06503_gb300.sim import workspace_bytes
    jobs = _jobs(n_steps=3)
    big = max(workspace_bytes(j.problem.mesh, precision="fp32") for j in jobs)
    srv = Server(budget_bytes=int(2.2 * big), max_resident=16, precision="fp32")
    rep = srv.run(jobs)
    assert rep["completed"] == len(jobs)
    assert rep["peak_resident_bytes"] <= rep["budget_bytes"]
    with pytest.raises(ValueError):
        Server(budget_bytes=big // 2, precision="fp32").submit(jobs[np.argmax([j.problem.mesh.nel for j in jobs])])


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_served_plate_and_beam_against_oracle(precision):
    """Requests 14 (56 x 56 notched plate, 30 load steps) and 7 (42 x 8 x 8
    notched beam, 40 load steps) of the seeded trace, served together with two
    other trace requests by the continuous-batching server, against the
    oracle's stored runs of the same requests: curve, peak load, dissipated
    energy (kept by the library) and the final damage field."""
    from paper_2301_06503_gb300.serve import Job, Server
    from _parity import ACCURACY, accuracy
    trace = li.serving_trace()
    cases = {14: ("trace_plate_r14_30.json", 30), 7: ("trace_beam_r7_40.json", 40)}
    for k, (f, _) in cases.items():
        if not os.path.exists(os.path.join(GOLDEN, f)):
            pytest.skip(f"oracle run {f} not stored")
    jobs = [Job(k, trace[k].problem, 0.0, n) for k, (_, n) in cases.items()]
    jobs += [Job(k, trace[k].problem, 0.0, 4) for k in (16, 17)]      # two small plates join the mix
    srv = Server(budget_bytes=8 << 30, max_resident=3, precision=precision, keep_fields=True)
    rep = srv.run(jobs)
    assert rep["completed"] == len(jobs) and rep["failed"] == 0
    for j in jobs[:2]:
        g = json.load(open(os.path.join(GOLDEN, cases[j.rid][0])))
        err = accuracy(j.problem, g, j.reactions, j.psi, j.damage, dissipated=j.dissipated)
        print(f"\nserved {precision} request {j.rid}:", {k: f"{v:.2e}" for k, v in err.items()})
        for k, v in err.items():
            assert v <= ACCURACY[precision][k], (j.rid, k, v)
