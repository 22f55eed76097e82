"""Continuous-batching server for LGDM simulations.

Requests (a problem: mesh, material, Dirichlet list, load schedule) arrive
over time.  Each scheduler tick:

1. admits queued requests, in arrival order, while the device-memory budget
   (the sum of the resident simulations' workspaces) and the slot count
   allow; an admitted simulation keeps its mesh, CSR pattern and history
   resident until it finishes;
2. advances every resident simulation by one load step together: a batch
   over the residents runs the Newton iterations of all of them in the same
   launches (persistent element kernel, grouped solves), each simulation at
   its own load value;
3. retires the simulations whose last load step is done (their slot and
   memory are reused by the next admission).

A request's result is bitwise the same whether it ran alone or among others
(the batch guarantees it), so serving changes only latency and throughput.
The scheduler is host code; all arithmetic of the method runs in the
library's kernels.
"""
import time
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import torch

from .batch import Batch
from .sim import Sim, workspace_bytes


@dataclass
class Job:
    rid: int
    problem: object
    arrival: float                  # seconds after the trace start
    n_steps: int
    admit: Optional[float] = None
    finish: Optional[float] = None
    step: int = 0
    sim: Optional[Sim] = None
    bytes: int = 0
    reactions: List[float] = field(default_factory=list)
    newton_iters: int = 0
    krylov_iters: int = 0
    psi: Optional[float] = None             # stored energy (Eq. 1) at the last committed state
    status: int = 0

    @property
    def time_to_solution(self):
        return None if self.finish is None else self.finish - self.arrival

    @property
    def service_time(self):
        return None if self.finish is None else self.finish - self.admit

    def record(self) -> dict:
        """One line of the per-request log: times, iteration counts, peak load
        and dissipated energy (external work by the trapezoid rule over the
        served load steps minus the stored energy)."""
        loads = [0.0] + [self.problem.load(n) for n in range(1, len(self.reactions) + 1)]
        reac = [0.0] + list(self.reactions)
        w_ext = sum(0.5 * (reac[k] + reac[k - 1]) * (loads[k] - loads[k - 1]) for k in range(1, len(reac)))
        return {"rid": self.rid, "arrival": self.arrival, "admit": self.admit, "finish": self.finish,
                "status": self.status, "load_steps": self.step, "newton_iters": self.newton_iters,
                "krylov_iters": self.krylov_iters,
                "peak_load": max(self.reactions) if self.reactions else None,
                "dissipated_energy": (w_ext - self.psi) if self.psi is not None else None}


class Server:
    def __init__(self, budget_bytes: int, max_resident: int = 64, precision: str = "fp32",
                 stream: Optional[torch.cuda.Stream] = None, autotune: bool = True, log=None, **sim_opts):
        self.budget = int(budget_bytes)
        self.max_resident = max_resident
        self.precision = precision
        self.sim_opts = sim_opts
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.autotune = autotune
        self.queue: List[Job] = []
        self.resident: List[Job] = []
        self.done: List[Job] = []
        self.used = 0
        self.peak_used = 0
        self.batch: Optional[Batch] = None
        self.ticks = 0
        self.tuning = None
        self.log = log
        self._t0 = time.perf_counter()

    # ------------------------------------------------------------------ admission
    def submit(self, job: Job):
        job.bytes = workspace_bytes(job.problem.mesh, precision=self.precision, **self.sim_opts)
        if job.bytes > self.budget:
            raise ValueError(f"request {job.rid} needs {job.bytes} bytes, more than the whole budget")
        self.queue.append(job)

    def _admit(self, now: float) -> bool:
        changed = False
        while self.queue and len(self.resident) < self.max_resident:
            job = self.queue[0]
            if job.arrival > now or self.used + job.bytes > self.budget:
                break
            self.queue.pop(0)
            p = job.problem
            job.sim = Sim(p.mesh, p.material, p.bcs, stream=self.stream, precision=self.precision, **self.sim_opts)
            job.admit = now
            self.used += job.bytes
            self.peak_used = max(self.peak_used, self.used)
            self.resident.append(job)
            changed = True
        return changed

    def _retire(self, now: float):
        keep = []
        for job in self.resident:
            if job.step >= job.n_steps or job.status != 0:
                job.finish = now
                job.krylov_iters = job.sim.counters()["krylov_iters"]
                if job.status == 0:
                    job.psi = job.sim.energy()
                job.sim.close()
                job.sim = None
                self.used -= job.bytes
                self.done.append(job)
            else:
                keep.append(job)
        changed = len(keep) != len(self.resident)
        self.resident = keep
        return changed

    def _rebuild(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        if self.resident:
            self.batch = Batch([j.sim for j in self.resident])
            if self.autotune and self.tuning is None:
                self.tuning = self.batch.autotune()
                # the autotuner assembled on the current states; restore nothing:
                # assembly does not change the state
            elif self.tuning is not None:
                self.batch.set_tuning(self.tuning["block_threads"], self.tuning["grid_factor"], True)

    # ------------------------------------------------------------------ ticks
    def tick(self, now: float):
        changed = self._admit(now)
        if changed or (self.batch is None and self.resident):
            self._rebuild()
        if not self.resident:
            return
        loads = [j.problem.load(j.step + 1) for j in self.resident]
        its, status = self.batch.run_step(loads)
        for j, it, st in zip(self.resident, its, status):
            j.newton_iters += int(it)
            j.status = int(st)
            j.step += 1
            j.reactions.append(j.sim.reaction())
        self.ticks += 1
        if self.log is not None:
            self.log(f"tick {self.ticks} t={self._clock():.2f}s resident={len(self.resident)} "
                     f"queued={len(self.queue)} done={len(self.done)} newton={list(map(int, its))}")
        if self._retire(self._clock()):
            self._rebuild()

    def _clock(self):
        return time.perf_counter() - self._t0

    def run(self, jobs: List[Job], time_limit: Optional[float] = None):
        """Serve a trace in real time: a job is admissible once its arrival time has passed."""
        for j in sorted(jobs, key=lambda j: j.arrival):
            self.submit(j)
        self._t0 = time.perf_counter()
        while self.queue or self.resident:
            now = self._clock()
            if not self.resident and self.queue and self.queue[0].arrival > now:
                time.sleep(min(self.queue[0].arrival - now, 0.05))
                continue
            self.tick(now)
            if time_limit is not None and self._clock() > time_limit:
                break
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        return self.report(self._clock())

    def report(self, wall: float):
        tts = np.array([j.time_to_solution for j in self.done if j.status == 0])
        svc = np.array([j.service_time for j in self.done if j.status == 0])
        ok = len(tts)
        return {
            "completed": ok, "failed": sum(1 for j in self.done if j.status != 0),
            "wall_s": wall, "sims_per_hour": 3600.0 * ok / wall if wall > 0 else 0.0,
            "p50_time_to_solution_s": float(np.percentile(tts, 50)) if ok else None,
            "p99_time_to_solution_s": float(np.percentile(tts, 99)) if ok else None,
            "p50_service_s": float(np.percentile(svc, 50)) if ok else None,
            "p99_service_s": float(np.percentile(svc, 99)) if ok else None,
            "ticks": self.ticks, "peak_resident_bytes": self.peak_used, "budget_bytes": self.budget,
        }

    def records(self) -> List[dict]:
        """Per-request log of the finished requests, in request order."""
        return [j.record() for j in sorted(self.done, key=lambda j: j.rid)]


def run_one_at_a_time(jobs: List[Job], precision: str = "fp64", stream=None, **sim_opts):
    """The plain form: requests served one after the other, each alone."""
    stream = stream if stream is not None else torch.cuda.Stream()
    jobs = sorted(jobs, key=lambda j: j.arrival)
    t0 = time.perf_counter()
    for job in jobs:
        now = time.perf_counter() - t0
        if job.arrival > now:
            time.sleep(job.arrival - now)
        job.admit = time.perf_counter() - t0
        p = job.problem
        s = Sim(p.mesh, p.material, p.bcs, stream=stream, precision=precision, **sim_opts)
        for n in range(1, job.n_steps + 1):
            try:
                job.newton_iters += s.run_step(p.load(n))
            except Exception:
                job.status = 4
                break
            job.reactions.append(s.reaction())
            job.step = n
        s.close()
        job.finish = time.perf_counter() - t0
    wall = time.perf_counter() - t0
    tts = np.array([j.time_to_solution for j in jobs if j.status == 0])
    svc = np.array([j.service_time for j in jobs if j.status == 0])
    ok = len(tts)
    return {"completed": ok, "failed": len(jobs) - ok, "wall_s": wall,
            "sims_per_hour": 3600.0 * ok / wall if wall > 0 else 0.0,
            "p50_time_to_solution_s": float(np.percentile(tts, 50)) if ok else None,
            "p99_time_to_solution_s": float(np.percentile(tts, 99)) if ok else None,
            "p50_service_s": float(np.percentile(svc, 50)) if ok else None,
            "p99_service_s": float(np.percentile(svc, 99)) if ok else None}
