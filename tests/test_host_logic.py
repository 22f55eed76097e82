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
    """Stand-in for a resident simulation: no device work."""
    live = 0

    def __init__(self, mesh, material, bcs, **kw):
        _FakeSim.live += 1
        self.mesh, self.steps = mesh, 0

    def reaction(self):
        return float(self.steps)

    def counters(self):
        return {"krylov_iters": 10 * self.steps}

    def energy(self):
        return 0.25

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

    def run_step(self, loads):
        for s in self.sims:
            s.steps += 1
        fail = [1 if getattr(s.mesh, "fails_at", None) == s.steps else 0 for s in self.sims]
        return np.full(len(self.sims), 3, np.int32), np.asarray(fail, np.int32) * 4

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
    w_ext = 0.001 * (0.5 * (0 + 1) + 0.5 * (1 + 2) + 0.5 * (2 + 3))
    assert abs(r0["dissipated_energy"] - (w_ext - 0.25)) <= 1e-15


def test_server_retires_a_failed_request(serve):
    jobs = [serve.Job(0, _Problem(10, fails_at=2), 0.0, n_steps=5),
            serve.Job(1, _Problem(10), 0.0, n_steps=5)]
    srv = serve.Server(budget_bytes=100, max_resident=4, stream=object(), autotune=False)
    rep = srv.run(jobs)
    assert rep["completed"] == 1 and rep["failed"] == 1
    assert jobs[0].step == 2 and jobs[1].step == 5
    assert _FakeSim.live == 0


def test_server_refuses_a_request_larger_than_the_budget(serve):
    srv = serve.Server(budget_bytes=50, stream=object())
    with pytest.raises(ValueError):
        srv.submit(serve.Job(0, _Problem(51), 0.0, n_steps=1))
