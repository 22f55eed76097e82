"""Continuous-batching server for LGDM simulations.

Requests (a problem: mesh, material, Dirichlet list, load schedule) arrive
over time.  Each scheduler tick:

1. admits queued requests, in arrival order, while the device-memory budget
   (the sum of the resident simulations' workspaces) and the slot count
   allow; an admitted simulation keeps its mesh, CSR pattern and history
   resident until it finishes;
2. runs ONE batched Newton iteration for every resident simulation: each
   resident that is not inside a load step begins its next one, then a batch
   over all residents assembles, solves and updates them in the same launches
   (persistent element kernel, grouped solves), each at its own load value;
3. commits every resident whose Newton test passed (the library keeps its
   reaction, external work and history), and hands a resident that used up
   its Newton iterations to the library's own load-step driver (increment
   halving from its committed state);
4. retires the simulations whose last load step is done; their slots and
   memory go to the next admission.

New requests therefore join between Newton iterations, not between load
steps.  The batch is rebuilt when the membership changes (its descriptors and
launch sizes depend on the members); the autotuned tile sizes are kept.  A
request's result is bitwise the same whether it ran alone or among others (a
batch member computes exactly what it computes alone), so serving changes
only latency and throughput.  The scheduler is host code; all arithmetic of
the method runs in the library's kernels.
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
    dissipated: Optional[float] = None      # external work minus stored energy, from the library
    external_work: Optional[float] = None
    damage: Optional[np.ndarray] = None     # final committed damage field (kept on request)
    status: int = 0
    in_step: bool = False                   # inside a load step (Newton iterations running)
    step_iters: int = 0                     # Newton iterations of the current load step

    @property
    def time_to_solution(self):
        return None if self.finish is None else self.finish - self.arrival

    @property
    def service_time(self):
        return None if self.finish is None else self.finish - self.admit

    def record(self) -> dict:
        """One line of the per-request log: times, iteration counts, peak load,
        external work and dissipated energy (both kept by the library at every
        commit)."""
        return {"rid": self.rid, "arrival": self.arrival, "admit": self.admit, "finish": self.finish,
                "status": self.status, "load_steps": self.step, "newton_iters": self.newton_iters,
                "krylov_iters": self.krylov_iters,
                "peak_load": max(self.reactions) if self.reactions else None,
                "external_work": self.external_work, "stored_energy": self.psi,
                "dissipated_energy": self.dissipated}


class Server:
    def __init__(self, budget_bytes: int, max_resident: int = 64, precision: str = "fp32",
                 stream: Optional[torch.cuda.Stream] = None, autotune: bool = True, log=None,
                 keep_fields: bool = False, **sim_opts):
        self.keep_fields = keep_fields
        self.max_newton = int(sim_opts.get("max_newton", 50))
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
        self.rebuilds = 0
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
                    job.dissipated, job.psi = job.sim.dissipated_energy()
                    job.external_work = job.sim.committed()[1]
                    if self.keep_fields:
                        job.damage = job.sim.field("damage")
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
        self.rebuilds += 1
        if self.resident:
            self.batch = Batch([j.sim for j in self.resident])
            if self.autotune and self.tuning is None:
                self.tuning = self.batch.autotune()
                # the autotuner assembled on the current states; restore nothing:
                # assembly does not change the state
            elif self.tuning is not None:
                self.batch.set_tuning(self.tuning["block_threads"], self.tuning["grid_factor"], True)

    # ------------------------------------------------------------------ ticks
    def _finish_step(self, j: Job):
        j.step += 1
        j.in_step = False
        j.reactions.append(j.sim.reaction())

    def tick(self, now: float):
        """Admit, one batched Newton iteration of every resident, commit, retire."""
        from ._lib import LgdmError
        changed = self._admit(now)
        if changed or (self.batch is None and self.resident):
            self._rebuild()
        if not self.resident:
            return
        for j in self.resident:
            if not j.in_step:
                j.sim.begin_step(j.problem.load(j.step + 1))
                j.in_step = True
                j.step_iters = 0
        conv, kits = self.batch.newton_step()
        for j, c, kit in zip(self.resident, conv, kits):
            j.step_iters += 1
            j.newton_iters += 1
            if c == 1:
                j.sim.commit()
                self._finish_step(j)
            elif c == -1 or j.step_iters >= self.max_newton:
                # diverged or out of Newton iterations: the library's load-step
                # driver halves the increment from the committed state
                try:
                    j.newton_iters += j.sim.run_step(j.problem.load(j.step + 1))
                    self._finish_step(j)
                except LgdmError as e:
                    j.status = int(e.status)
        self.ticks += 1
        if self.log is not None:
            self.log(f"tick {self.ticks} t={self._clock():.2f}s resident={len(self.resident)} "
                     f"queued={len(self.queue)} done={len(self.done)} steps={[j.step for j in self.resident]}")
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
            "ticks": self.ticks, "batch_rebuilds": self.rebuilds, "peak_resident_bytes": self.peak_used,
            "budget_bytes": self.budget,
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
        if job.status == 0:
            job.dissipated, job.psi = s.dissipated_energy()
            job.external_work = s.committed()[1]
        job.krylov_iters = s.counters()["krylov_iters"]
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
