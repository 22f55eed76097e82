"""Host-side logic that needs no GPU: the replica timing aggregation of the
benchmark over two gloo ranks, and the serving scheduler (admission by
device-memory budget, slots, interleaved ticks, retirement) driven with a
stand-in for the simulation library."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, units = bench.job_totals(1.0 + rank, 10 * (rank + 1), world, "cpu")
    out.put((rank, t, units))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_totals_two_gloo_ranks():
    """value = units of all ranks / the slowest rank's time."""
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, t, units in res:
        assert t == 2.0 and units == 30.0


def test_replica_totals_single_rank():
    import bench
    assert bench.job_totals(3.5, 7, 1, "cpu") == (3.5, 7.0)


# ------------------------------------------------------------------ serving
class _FakeSim:
    """Stand-in for a resident simulation: no device work.  A load step
    converges at its second Newton iteration; the reaction after step n is n;
    the stored energy is 0.25; a mesh with ``fails_at = n`` diverges in load
    step n and its load-step driver then reports non-convergence."""
    live = 0

    def __init__(self, mesh, material, bcs, **kw):
        _FakeSim.live += 1
        self.mesh, self.steps, self.iters = mesh, 0, 0
        self.load, self.load_commit, self.w_ext = 0.0, 0.0, 0.0

    def begin_step(self, load):
        self.load, self.iters = load, 0

    def _commit(self):
        r_old = float(self.steps)
        self.steps += 1
        self.w_ext += 0.5 * (r_old + self.steps) * (self.load - self.load_commit)
        self.load_commit = self.load

    def commit(self):
        self._commit()

    def run_step(self, load):
        from paper_2301_06503_gb300._lib import LgdmError
        if getattr(self.mesh, "fails_at", None) == self.steps + 1:
            raise LgdmError(4, "no convergence")
        self.begin_step(load)
        self._commit()
        return 2

    def reaction(self):
        return float(self.steps)

    def counters(self):
        return {"krylov_iters": 10 * self.steps}

    def committed(self):
        return self.load_commit, self.w_ext, float(self.steps)

    def dissipated_energy(self):
        return self.w_ext - 0.25, 0.25

    def close(self):
        _FakeSim.live -= 1


class _FakeBatch:
    made = []

    def __init__(self, sims):
        self.sims = list(sims)
        _FakeBatch.made.append(len(self.sims))

    def autotune(self):
        return {"block_threads": 128, "grid_factor": 2, "assembly_ms": 0.0}

    def set_tuning(self, *a):
        pass

    def newton_step(self, active=None):
        conv = []
        for s in self.sims:
            s.iters += 1
            if getattr(s.mesh, "fails_at", None) == s.steps + 1:
                conv.append(-1)
            else:
                conv.append(1 if s.iters >= 2 else 0)
        return np.asarray(conv, np.int32), np.full(len(self.sims), 5, np.int32)

    def close(self):
        pass


class _Mesh:
    def __init__(self, nbytes, fails_at=None):
        self.nbytes, self.fails_at = nbytes, fails_at


class _Problem:
    def __init__(self, nbytes, fails_at=None):
        self.mesh, self.material, self.bcs = _Mesh(nbytes, fails_at), None, None

    def load(self, n):
        return 0.001 * n


@pytest.fixture
def serve(monkeypatch):
    from paper_2301_06503_gb300 import serve as sv
    monkeypatch.setattr(sv, "Sim", _FakeSim)
    monkeypatch.setattr(sv, "Batch", _FakeBatch)
    monkeypatch.setattr(sv, "workspace_bytes", lambda mesh, **kw: mesh.nbytes)
    _FakeBatch.made.clear()
    _FakeSim.live = 0
    return sv


def test_server_budget_slots_and_reuse(serve):
    sizes = [40, 30, 50, 20, 60, 10]
    jobs = [serve.Job(i, _Problem(b), 0.0, n_steps=3 + i % 2) for i, b in enumerate(sizes)]
    srv = serve.Server(budget_bytes=100, max_resident=3, stream=object(), autotune=True)
    rep = srv.run(jobs)
    assert rep["completed"] == len(jobs) and rep["failed"] == 0
    assert rep["peak_resident_bytes"] <= 100
    assert max(_FakeBatch.made) <= 3                  # never more residents than slots
    assert len(_FakeBatch.made) > 1                   # the batch was rebuilt as slots freed
    assert _FakeSim.live == 0                         # every admitted simulation was closed
    for j in jobs:
        assert j.step == j.n_steps and j.reactions == [float(k) for k in range(1, j.n_steps + 1)]
    # admission in arrival order: a job is admitted no earlier than the one before it
    admits = [j.admit for j in sorted(jobs, key=lambda j: j.rid)]
    assert all(a <= b for a, b in zip(admits, admits[1:]))
    # per-request log: reactions 1, 2, 3 at loads 1, 2, 3 mm-thousandths
    rec = srv.records()
    assert [r["rid"] for r in rec] == list(range(len(jobs)))
    r0 = rec[0]
    assert r0["load_steps"] == 3 and r0["peak_load"] == 3.0 and r0["krylov_iters"] == 30
    assert r0["newton_iters"] == 6                   # two batched Newton iterations per load step
    w_ext = 0.001 * (0.5 * (0 + 1) + 0.5 * (1 + 2) + 0.5 * (2 + 3))
    assert abs(r0["external_work"] - w_ext) <= 1e-15
    assert abs(r0["dissipated_energy"] - (w_ext - 0.25)) <= 1e-15
    # arrivals join between Newton iterations: two ticks per load step
    assert srv.ticks >= 2 * max(j.n_steps for j in jobs)


def test_server_retires_a_failed_request(serve):
    jobs = [serve.Job(0, _Problem(10, fails_at=2), 0.0, n_steps=5),
            serve.Job(1, _Problem(10), 0.0, n_steps=5)]
    srv = serve.Server(budget_bytes=100, max_resident=4, stream=object(), autotune=False)
    rep = srv.run(jobs)
    assert rep["completed"] == 1 and rep["failed"] == 1
    assert jobs[0].step == 1 and jobs[1].step == 5     # the failure came in load step 2
    assert jobs[0].status == 4 and jobs[0].reactions == [1.0]
    assert _FakeSim.live == 0


def test_server_refuses_a_request_larger_than_the_budget(serve):
    srv = serve.Server(budget_bytes=50, stream=object())
    with pytest.raises(ValueError):
        srv.submit(serve.Job(0, _Problem(51), 0.0, n_steps=1))


# ------------------------------------------------------------------ bench line
def _plate_stats(newton=30, kiters=34250):
    import lgdm_inputs as li
    m = li.sen_plate_problem().mesh
    return m, {"gp": newton * m.nel * m.ngp, "newton": newton, "elem_integrations": newton * m.nel,
               "krylov_iters": kiters, "halvings": 0, "launches": 175,
               "phase_ms": {"element": 6.0, "gather": 1.64, "precond": 0.43, "krylov": 1898.6,
                            "commit": 0.15, "begin_step": 0.05},
               "phase_n": {"element": newton, "gather": newton, "precond": newton, "krylov": 2 * newton,
                           "commit": 5, "begin_step": 5},
               "elements": m.nel, "elem": m.elem, "nnode": m.nnode, "nel": m.nel, "nd": m.nd,
               "nnz": 3250809, "npairs": 361201,
               "members": [(m.nnode, m.nd, 3250809, 361201, kiters, [(40401, 361201), (4489, 39601), (64, 484)])]}


def test_bench_line_contract_and_rooflines():
    """The JSON line built from a run's counters and phase times: contract
    keys, throughput, and the roofline arithmetic of both kernels."""
    import argparse
    import bench
    from paper_2301_06503_gb300 import roofline
    m, st = _plate_stats()
    args = argparse.Namespace(precision="fp64", steps=5, warmup=3, mode="loadstep")
    pk = {"hbm_gbs": 6788.3, "hbm_src": "measured", "fp64_tflops": 1.25, "fp32_tflops": 75.0}
    step_ms = [381.6] * 5
    line = bench.summarize(args, "sen_plate_q4_200x200", 1, [m], st, step_ms, sum(step_ms) / 1e3, st["gp"], 1, pk,
                           {"value": 1.0, "unit": "GP/s", "h2d_bytes_per_step": 1, "d2h_bytes_per_step": 1},
                           None, {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []})
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
              "gpu_launches", "clocks"):
        assert k in line
    # the metric: Gauss points over element + gather time; the whole step beside it
    assert abs(line["value"] - st["gp"] / ((6.0 + 1.64) * 1e-3)) <= 1e-9 * line["value"]
    assert line["whole_step"]["value"] == st["gp"] / (sum(step_ms) / 1e3)
    assert abs(line["ms_per_step"] - 381.6) < 1e-9
    res_f, tan_f = roofline.element_flops(m.elem)
    el = line["roofline_element"]
    assert el["bound"] == "alu" and abs(el["achieved"] - m.nel * (res_f + tan_f) / 0.2e-3 / 1e12) < 1e-9
    assert abs(el["frac"] - el["achieved"] / 1.25) < 1e-12
    kr = line["roofline_krylov"]
    fl, by, f32 = roofline.krylov_iteration(m.nnode, m.nd, 3250809, 361201, 8,
                                            [(40401, 361201), (4489, 39601), (64, 484)])
    fj, _, _ = roofline.krylov_iteration(m.nnode, m.nd, 3250809, 361201, 8)
    assert fl > 2 * fj and f32 == 0                         # two V-cycles cost more than two Jacobi applies
    # float pairs (FP32 tangent): the 2 SpMVs and the 2 finest residuals move to the
    # FP32 pipe, the total algorithmic flops stay the same
    fl2, by2, f2 = roofline.krylov_iteration(m.nnode, m.nd, 3250809, 361201, 8,
                                             [(40401, 361201), (4489, 39601), (64, 484)], float_pairs=True)
    assert fl2 + f2 == fl and f2 == 4 * 2 * 3250809 and by2 > by
    t_fl, t_by = fl / 1.25e12, by / 6788.3e9                # the slower of the two at its peak binds
    if t_by > t_fl:
        assert kr["bound"] == "hbm"
        assert abs(kr["achieved"] - by * st["krylov_iters"] / (1898.6e-3) / 1e9) < 1e-6
    else:
        assert kr["bound"] == "alu"
        assert abs(kr["achieved"] - fl * st["krylov_iters"] / (1898.6e-3) / 1e12) < 1e-9
    assert abs(kr["frac"] - kr["achieved"] / kr["peak"]) < 1e-12
    assert line["roofline"] is kr                           # the solve dominates this step


def test_bench_line_fp32_element_bound():
    """FP32 tangent: the element roofline takes the slowest of the FP64
    residual path, the FP32 tangent path and the bytes."""
    import argparse
    import bench
    m, st = _plate_stats()
    args = argparse.Namespace(precision="fp32", steps=2, warmup=3, mode="newton")
    pk = {"hbm_gbs": 6788.3, "hbm_src": "measured", "fp64_tflops": 1.25, "fp32_tflops": 75.0}
    line = bench.summarize(args, "x", 1, [m], st, [10.0, 10.0], 0.02, st["gp"], 1, pk, None, None, None)
    el = line["roofline_element"]
    assert el["bound"] == "alu" and el["peak"] == 1.25 and line["dtype"] == "f32-tangent/f64"


def test_paper_workloads_and_mixed_order_work_model():
    """The paper's problems as bench workloads (their largest printed meshes)
    and the element work model of the mixed-order elements: the micro-strain
    terms of a 9-node quad count on its 4 vertices only, so it costs less
    than a 9-node equal-order count and more than a 4-node quad."""
    import argparse
    import bench
    from paper_2301_06503_gb300 import roofline
    probs, label = bench.workload("paper_plate")
    assert label == "paper_sen_plate_q9_120x120" and probs[0].mesh.nel == 14400 and probs[0].mesh.nen == 9
    probs, label = bench.workload("paper_slab")
    assert label == "paper_sen_slab_h8_100x100x5" and probs[0].mesh.nel == 50000
    probs, label = bench.workload("paper_bar")
    assert label == "paper_bar_l3_1000" and probs[0].mesh.nel == 1000 and probs[0].mesh.nen == 3
    for w in ("paper_plate", "paper_slab"):
        (q,) = bench._problem_list(w, 1)                # the oracle's bounded sample: same elements
        assert q.mesh.elem == bench.workload(w)[0][0].mesh.elem and q.mesh.nel < 14400
    r9, t9 = roofline.element_flops(5)
    r4, t4 = roofline.element_flops(2)
    assert r9 + t9 > 2 * (r4 + t4)
    # a 9-node element with every node carrying the micro-strain would cost more
    d, n, v, ne = roofline._DIMS[5]
    roofline._DIMS[5] = (d, n, v, n)
    try:
        full = sum(roofline.element_flops(5))
    finally:
        roofline._DIMS[5] = (d, n, v, ne)
    assert full > r9 + t9
    # the bench line of a 9-node run: the element roofline uses that count
    m = bench.workload("paper_plate")[0][0].mesh
    st = {"gp": 2 * m.nel * m.ngp, "newton": 2, "elem_integrations": 2 * m.nel, "krylov_iters": 300,
          "halvings": 0, "launches": 40,
          "phase_ms": {"element": 1.3, "gather": 0.2, "precond": 1.0, "krylov": 100.0, "commit": 0.1,
                       "begin_step": 0.01},
          "phase_n": {"element": 2, "gather": 2, "precond": 2, "krylov": 4, "commit": 1, "begin_step": 1},
          "elements": m.nel, "elem": m.elem, "nnode": m.nnode, "nel": m.nel, "nd": m.nd,
          "nnz": 9 * 25 * m.nnode, "npairs": 25 * m.nnode,
          "members": [(m.nnode, m.nd, 9 * 25 * m.nnode, 25 * m.nnode, 300, [(m.nnode, 25 * m.nnode), (900, 8100)])]}
    args = argparse.Namespace(precision="fp64", steps=1, warmup=3, mode="loadstep")
    pk = {"hbm_gbs": 6788.3, "hbm_src": "measured", "fp64_tflops": 1.25, "fp32_tflops": 75.0}
    line = bench.summarize(args, "paper_sen_plate_q9_120x120", 1, [m], st, [100.0], 0.1, st["gp"], 1, pk,
                           None, None, None)
    el = line["roofline_element"]
    assert abs(el["achieved"] - m.nel * (r9 + t9) / 0.65e-3 / 1e12) < 1e-9
