#!/usr/bin/env python
"""Throughput of the LGDM hot path on GB300.

Default workload: the batch of 256 notched plates (20..300 four-node quads
per edge, seeded draw; 4.84M elements, 19.4M Gauss points, 14.6M dofs) with
the FP32 tangent and FP64 residual, in one batch: persistent element kernel,
batched gather and preconditioner set-up, grouped multigrid-preconditioned
BiCGSTAB solves, the batched update, autotuned tiles.  A timed step is one
batched Newton iteration of every member at load increment 1 from its
initial state (device-side reset, Dirichlet predictor, assembly, multigrid
set-up, solve, update and convergence test).

The metric counts Gauss-point integrations with assembly per second: the
Gauss points integrated in the timed region over the CUDA-event time of the
element-integration and CSR-gather (with Dirichlet rows) launches in it.
The line also gives the whole step's rate (same Gauss points over the whole
step time), the rooflines of the element and Krylov kernels, the oracle on
the host cores (one core and all cores) and an end-to-end figure through the
public API from pinned host buffers (state in, damage field and reaction
out).  Inputs are resident in HBM when the timed region starts; L2 is flushed
(256 MB write) before each step and the batch's state is far larger than L2.

Other workloads (--workload): plate (the 200 x 200 notched plate), bar (100
two-node elements), beam (200 x 40 x 40 hexahedra, 1.35M dofs), and the
paper's own problems at their largest printed meshes: paper_bar (1000
three-node quadratic elements), paper_plate (the 2D notched specimen, 120 x
120 nine-node elements), paper_slab (the 3D notched specimen, 100 x 100 x 5
hexahedra); for them a step solves load increment 1 (Newton to convergence)
unless --mode newton.
--precision fp64 assembles and applies everything in FP64.

--serving runs the request-serving comparison instead and prints its own
JSON line: the first --requests requests of the seeded Poisson trace (70 %
plates, 30 % beams, 20 requests/s), each simulation --serve-steps load
increments of its 300-increment schedule, served (i) by the continuous-
batching server with the FP32 tangent and (ii) one at a time in FP64;
simulations/hour, p50/p99 time-to-solution and service time, and the
largest difference between the two forms' load-displacement curves.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank runs an independent replica (weak scaling).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gauss-pt integrations+assembly/s"
UNIT = "GP/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32"],
                    help="fp32: FP32 tangent, FP64 residual (default for the batch); fp64 (default otherwise)")
    ap.add_argument("--workload", default="batch",
                    choices=["plate", "bar", "beam", "batch", "paper_bar", "paper_plate", "paper_slab"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default=None, choices=["loadstep", "newton"],
                    help="loadstep: a step is a converged load increment (default for one simulation); "
                         "newton: one Newton iteration, assemble + solve + update (default for the batch)")
    ap.add_argument("--batch-count", type=int, default=256,
                    help="simulations of the batch workload (the first ones of the seeded 256-plate draw)")
    ap.add_argument("--serving", action="store_true")
    ap.add_argument("--requests", type=int, default=16)
    ap.add_argument("--serve-steps", type=int, default=10)
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--max-resident", type=int, default=64)
    ap.add_argument("--max-krylov", type=int, default=5000,
                    help="BiCGSTAB iteration cap (profiling captures use a small cap)")
    ap.add_argument("--serve-max-newton", type=int, default=25,
                    help="Newton iterations per attempt in the serving comparison (both forms)")
    ap.add_argument("--serve-max-halvings", type=int, default=2,
                    help="increment halvings per load step in the serving comparison (both forms)")
    return ap.parse_args()


def workload(name):
    import lgdm_inputs as li
    if name == "plate":
        return [li.sen_plate_problem()], "sen_plate_q4_200x200"
    if name == "bar":
        return [li.bar_problem()], "bar_l2_100"
    if name == "beam":
        return [li.tpb_beam_problem()], "tpb_beam_h8_200x40x40"
    if name == "paper_bar":
        return [li.paper_bar_problem(1000)], "paper_bar_l3_1000"
    if name == "paper_plate":
        return [li.paper_sen_plate_problem(120)], "paper_sen_plate_q9_120x120"
    if name == "paper_slab":
        return [li.paper_sen_slab_problem(100)], "paper_sen_slab_h8_100x100x5"
    return li.batch_plate_problems(), "batch_plates_q4_20to300"


def mg_levels(sz):
    """[(nodes, node pairs)] of the multigrid levels of a simulation (empty without)."""
    return [(int(sz.mg_nnode[k]), int(sz.mg_npairs[k])) for k in range(int(sz.mg_levels))]


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi samples during the timed region (200 ms period)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[5 + k] and "Not" not in r[5 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm, src = 6800.0, "fallback"
    if os.path.exists(path):
        try:
            hbm, src = float(json.load(open(path))["hbm_gbs"]), "measured"
        except (ValueError, KeyError):
            pass
    # FP64 / FP32 pipe peaks: nominal GB300 figures (1.25 and 75 TFLOP/s)
    return {"hbm_gbs": hbm, "hbm_src": src, "fp64_tflops": 1.25, "fp32_tflops": 75.0}


def traffic_for(kernel, workload):
    """DRAM bytes from a committed ncu summary, if the kernels are unchanged:
    per launch for the element kernel, per iteration for the Krylov kernel."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path))
        if rec.get("csrc_sha") != csrc_sha():
            return None
        return rec["kernels"].get(f"{kernel}@{workload}")
    except (ValueError, KeyError, AttributeError):
        return None


# the sources the profiled kernels are compiled from (host code lives in api.cu)
KERNEL_SOURCES = ("element.cu", "krylov.cu", "amg.cu", "lgdm_internal.cuh", "node_block.cuh")


def csrc_sha():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2301_06503_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def job_totals(t_s, units, world, device):
    """Whole-job time and work over the replicas: the slowest rank's timed
    seconds and the sum of every rank's units (Gauss points)."""
    if world <= 1:
        return t_s, float(units)
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t_s, float(units)], device=device, dtype=torch.float64)
    tmax = tt.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tt, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tt[1])


def _cores_used(cpu_s, wall_s):
    """Threads the oracle actually kept busy: process CPU time over wall time."""
    return max(1, int(round(cpu_s / wall_s))) if wall_s > 0 else 1


# the beam's oracle sample: a slab of 4 of its 200 element columns (same
# 1 mm hexahedra, material and notch depth), one assembly of which takes
# seconds on a host core instead of minutes
BEAM_SAMPLE = "a 4 x 40 x 40-hexahedra slab of the beam (same element size and material)"
# the same for the paper's 2D and 3D specimens: smaller meshes of the same
# elements and material (the oracle's cost per Gauss point does not depend on
# the element size)
SAMPLES = {"beam": BEAM_SAMPLE,
           "paper_plate": "the 30 x 30 mesh of the same specimen (same elements and material)",
           "paper_slab": "the 20 x 20 x 5 mesh of the same specimen (same elements and material)"}


def _problem_list(workload_name, count):
    """The problems of a workload's CPU sample, rebuilt from its seeded recipe
    (no arrays pass between processes)."""
    import lgdm_inputs as li
    if workload_name == "batch":
        return li.batch_plate_problems()[:count]
    if workload_name == "beam":
        return [li.tpb_beam_problem(4, 40, 40, 4.0, 40.0, 40.0)]
    if workload_name == "paper_plate":
        return [li.paper_sen_plate_problem(30)]
    if workload_name == "paper_slab":
        return [li.paper_sen_slab_problem(20)]
    return workload(workload_name)[0]


def _oracle_assembly(workload_name, count, first, stride, budget_s):
    """Time the oracle's assembly (element integration of every Gauss point,
    sparse assembly, Dirichlet rows) at load step 1 from the initial state,
    on problems first, first+stride, ... (cycling) until budget_s of wall
    time.  Returns (Gauss points, wall seconds, CPU seconds, assemblies)."""
    from oracle import assembly as asm
    from oracle import newton as nw
    probs = _problem_list(workload_name, count)
    gp = done = 0
    k = first
    c0, t0 = time.process_time(), time.perf_counter()
    while True:
        p = probs[k % len(probs)]
        st = nw.initial_state(p)
        u = st.u.copy()
        u[p.bcs.dir_dof] = p.bcs.dir_scale * p.load(1)
        K, r = asm.assemble(p.mesh, p.material, u, st.kappa_hist)
        asm.apply_dirichlet(K, r, p.bcs.dir_dof, p.mesh)
        gp += p.mesh.nel * p.mesh.ngp
        done += 1
        k += stride
        if time.perf_counter() - t0 > budget_s:
            break
    return gp, time.perf_counter() - t0, time.process_time() - c0, done


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(workload_name, count, label, budget_s=8.0):
    """The oracle as it stands, on the same metric: Gauss-point integrations
    with assembly per second.  One process (one core) and a pool of spawned
    processes over all host cores, each assembling different problems of the
    workload for about budget_s (a bounded sample)."""
    import multiprocessing as mp
    gp1, wall1, cpu1, n1 = _oracle_assembly(workload_name, count, 0, 1, budget_s)
    what = f"{label} ({SAMPLES[workload_name]})" if workload_name in SAMPLES else label
    one = {"value": gp1 / wall1, "unit": UNIT, "cores": _cores_used(cpu1, wall1), "kind": "oracle",
           "sample": f"{what}: {n1} oracle assemblies (numpy element integration, scipy sparse assembly, "
                     f"Dirichlet rows) at load step 1, {wall1:.1f} s wall"}
    ncores = _host_cores()
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(ncores) as pool:
        res = pool.starmap(_oracle_assembly, [(workload_name, count, w, ncores, budget_s) for w in range(ncores)])
    wall = time.perf_counter() - t0
    gp = sum(r[0] for r in res)
    span = max(r[1] for r in res)
    cpu = sum(r[2] for r in res)
    n = sum(r[3] for r in res)
    return {"value": gp / span, "unit": UNIT, "cores": _cores_used(cpu, span), "kind": "oracle",
            "sample": f"{what}: {n} oracle assemblies at load step 1 in {ncores} spawned processes (each "
                      f"assembling different problems for {budget_s:.0f} s; throughput = Gauss points / "
                      f"longest worker time {span:.1f} s; pool wall {wall:.1f} s with start-up)",
            "one_core": one}


def run_reference(args):
    """Reference arm: the CPU oracle on the same metric (Gauss-point
    integrations with assembly per second); a step is one oracle assembly of
    the next problem of the workload (bounded sample)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import assembly as asm
    from oracle import newton as nw
    probs, label = workload(args.workload)
    if args.workload == "batch":
        probs = probs[:args.batch_count]
        label = f"batch_{len(probs)}_plates_q4_20to300"
    sample = label
    if args.workload in SAMPLES:
        probs = _problem_list(args.workload, 1)
        sample = f"{label} ({SAMPLES[args.workload]})"
    k = [0]

    def step():
        p = probs[k[0] % len(probs)]
        k[0] += 1
        st = nw.initial_state(p)
        u = st.u.copy()
        u[p.bcs.dir_dof] = p.bcs.dir_scale * p.load(1)
        K, r = asm.assemble(p.mesh, p.material, u, st.kappa_hist)
        asm.apply_dirichlet(K, r, p.bcs.dir_dof, p.mesh)
        return p.mesh.nel * p.mesh.ngp

    for _ in range(args.warmup):
        step()
    k[0] = 0
    times, gp = [], 0
    c0 = time.process_time()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        gp += step()
        times.append(time.perf_counter() - t0)
    wall = sum(times)
    cores = _cores_used(time.process_time() - c0, wall)
    value = gp / wall
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": label, "step": "one oracle assembly (element integration, sparse assembly, "
                                                  "Dirichlet rows) of the next problem at load step 1",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{sample}: {args.steps} oracle assemblies, problems in order"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class SingleLeg:
    """One simulation; a step solves load increment 1 from the initial state."""

    def __init__(self, p, label, args):
        from paper_2301_06503_gb300 import Sim
        self.p, self.label, self.args = p, label, args
        self.sim = Sim(p.mesh, p.material, p.bcs, precision=args.precision, max_krylov=args.max_krylov)
        self.stream = self.sim.stream
        self.load = p.load(1)
        self.meshes = [p.mesh]

    def step(self):
        self.sim.reset_state()
        if self.args.mode == "newton":
            self.sim.begin_step(self.load)
            self.sim.newton_step()
        else:
            self.sim.run_step(self.load)

    def start_timing(self):
        self.sim.enable_timers(True)
        self.sim.timers(reset=True)
        self.c0 = self.sim.counters()

    def stop_timing(self):
        c1 = self.sim.counters()
        tm = self.sim.timers()
        m = self.p.mesh
        newton = c1["assemblies"] - self.c0["assemblies"]
        sz = self.sim.sizes
        return {"gp": newton * m.nel * m.ngp, "newton": newton, "elem_integrations": newton * m.nel,
                "krylov_iters": c1["krylov_iters"] - self.c0["krylov_iters"],
                "halvings": c1["halvings"] - self.c0["halvings"],
                "launches": c1["kernel_launches"] - self.c0["kernel_launches"],
                "phase_ms": {k: v[0] for k, v in tm.items()}, "phase_n": {k: v[1] for k, v in tm.items()},
                "elements": m.nel, "elem": m.elem, "nnode": int(sz.nnode), "nel": m.nel, "nd": int(sz.nd),
                "nnz": int(sz.nnz), "npairs": int(sz.npairs),
                "members": [(int(sz.nnode), int(sz.nd), int(sz.nnz), int(sz.npairs),
                             c1["krylov_iters"] - self.c0["krylov_iters"], mg_levels(sz))]}

    def e2e(self, reps):
        import torch
        m = self.p.mesh
        u0 = torch.zeros(m.ndof, dtype=torch.float64).pin_memory().numpy()
        kh0 = torch.full((m.nel * m.ngp,), self.p.material.kappa0, dtype=torch.float64).pin_memory().numpy()
        times, gp, dmg = [], 0, None
        for _ in range(reps):
            cn0 = self.sim.counters()["assemblies"]
            t0 = time.perf_counter()
            self.sim.set_state(u0, kh0)                      # state in (pinned host -> device)
            if self.args.mode == "newton":
                self.sim.begin_step(self.load)
                self.sim.newton_step()
            else:
                self.sim.run_step(self.load)
            dmg = self.sim.field("damage")                   # damage field out
            self.sim.reaction()                              # load-displacement point out
            times.append(time.perf_counter() - t0)
            gp += (self.sim.counters()["assemblies"] - cn0) * m.nel * m.ngp
        return {"value": gp / sum(times), "unit": UNIT, "h2d_bytes_per_step": int(u0.nbytes + kh0.nbytes),
                "d2h_bytes_per_step": int(dmg.nbytes + 8)}

    def close(self):
        self.sim.close()


class BatchLeg:
    """Many simulations in one batch (persistent element kernel, grouped
    solves, a CUDA graph per Newton step, autotuned tiles); a step solves
    load increment 1 of every member from its initial state."""

    def __init__(self, problems, label, args):
        import torch
        from paper_2301_06503_gb300 import Batch, Sim
        self.problems, self.label, self.args = problems, label, args
        self.stream = torch.cuda.Stream()
        self.sims = [Sim(p.mesh, p.material, p.bcs, stream=self.stream, precision=args.precision,
                         max_krylov=args.max_krylov) for p in problems]
        self.batch = Batch(self.sims)
        self.tuning = self.batch.autotune()
        self.loads = [p.load(1) for p in problems]
        self.meshes = [p.mesh for p in problems]

    def step(self):
        for s in self.sims:
            s.reset_state()
        if self.args.mode == "newton":
            for s, ld in zip(self.sims, self.loads):
                s.begin_step(ld)
            self.batch.newton_step()
        else:
            self.batch.run_step(self.loads)

    def start_timing(self):
        self.batch.enable_timers(True)
        self.batch.timers(reset=True)
        self.c0 = [s.counters() for s in self.sims]
        self.l0 = self.batch.launches()

    def stop_timing(self):
        c1 = [s.counters() for s in self.sims]
        tm = self.batch.timers()
        d = lambda k: sum(b[k] - a[k] for a, b in zip(self.c0, c1))
        gp = sum((b["assemblies"] - a["assemblies"]) * s.mesh.nel * s.mesh.ngp
                 for a, b, s in zip(self.c0, c1, self.problems))
        els = sum(p.mesh.nel for p in self.problems)
        return {"gp": gp, "newton": d("assemblies"), "krylov_iters": d("krylov_iters"), "halvings": d("halvings"),
                "elem_integrations": sum((b["assemblies"] - a["assemblies"]) * p.mesh.nel
                                         for a, b, p in zip(self.c0, c1, self.problems)),
                "launches": d("kernel_launches") + self.batch.launches() - self.l0,
                "phase_ms": {k: v[0] for k, v in tm.items()}, "phase_n": {k: v[1] for k, v in tm.items()},
                "elements": els, "elem": self.problems[0].mesh.elem,
                "nnode": sum(int(s.sizes.nnode) for s in self.sims), "nel": els,
                "nd": int(self.sims[0].sizes.nd), "nnz": sum(int(s.sizes.nnz) for s in self.sims),
                "npairs": sum(int(s.sizes.npairs) for s in self.sims), "tuning": self.tuning,
                "members": [(int(s.sizes.nnode), int(s.sizes.nd), int(s.sizes.nnz), int(s.sizes.npairs),
                             b["krylov_iters"] - a["krylov_iters"], mg_levels(s.sizes))
                            for s, a, b in zip(self.sims, self.c0, c1)]}

    def e2e(self, reps):
        import torch
        pinned = [(torch.zeros(p.mesh.ndof, dtype=torch.float64).pin_memory().numpy(),
                   torch.full((p.mesh.nel * p.mesh.ngp,), p.material.kappa0,
                              dtype=torch.float64).pin_memory().numpy()) for p in self.problems]
        times, gp, dbytes = [], 0, 0
        for _ in range(reps):
            cn0 = [s.counters()["assemblies"] for s in self.sims]
            t0 = time.perf_counter()
            for s, (u0, kh0) in zip(self.sims, pinned):
                s.set_state(u0, kh0)
            if self.args.mode == "newton":
                for s, ld in zip(self.sims, self.loads):
                    s.begin_step(ld)
                self.batch.newton_step()
            else:
                self.batch.run_step(self.loads)
            dbytes = 0
            for s in self.sims:
                dbytes += s.field("damage").nbytes + 8
                s.reaction()
            times.append(time.perf_counter() - t0)
            gp += sum((s.counters()["assemblies"] - a) * p.mesh.nel * p.mesh.ngp
                      for s, a, p in zip(self.sims, cn0, self.problems))
        return {"value": gp / sum(times), "unit": UNIT,
                "h2d_bytes_per_step": int(sum(u.nbytes + k.nbytes for u, k in pinned)),
                "d2h_bytes_per_step": int(dbytes)}

    def close(self):
        self.batch.close()
        for s in self.sims:
            s.close()


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2301_06503_gb300 import build
    if rank == 0:
        build()
    if world > 1:
        torch.distributed.barrier()
    build()
    probs, label = workload(args.workload)
    if args.workload == "batch":
        probs = probs[:args.batch_count]
        label = f"batch_{len(probs)}_plates_q4_20to300"
    leg = BatchLeg(probs, label, args) if args.workload == "batch" else SingleLeg(probs[0], label, args)
    stream = leg.stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            leg.step()
    leg.start_timing()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            leg.step()
            ends[k].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    st = leg.stop_timing()
    t_s = sum(step_ms) / 1e3
    t_job, gp_job = job_totals(t_s, st["gp"], world, "cuda")
    t_asm_job, _ = job_totals((st["phase_ms"]["element"] + st["phase_ms"]["gather"]) * 1e-3, 0, world, "cuda")
    e2e = leg.e2e(max(1, min(args.steps, 3))) if rank == 0 else None
    meshes = leg.meshes
    leg.close()
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, len(probs), label)
    line = summarize(args, label, len(probs), meshes, st, step_ms, t_job, gp_job, world, peaks(), e2e, cpu, ck,
                     t_asm_job)
    print(json.dumps(line), flush=True)


def summarize(args, label, n_sims, meshes, st, step_ms, t_job, gp_job, world, pk, e2e, cpu, ck, t_asm_job=None):
    """The JSON line of one timed run: throughput, rooflines of the element
    and Krylov kernels (work over the timed region's CUDA-event phase times),
    the assembly-only rate and the details."""
    from paper_2301_06503_gb300 import roofline
    fp32 = args.precision == "fp32"
    tb = 4 if fp32 else 8
    phase_ms, phase_n = st["phase_ms"], st["phase_n"]
    # Krylov work summed member by member: iterations x work per iteration
    kr_flops = kr_bytes = kr_f32 = 0
    for nnode, nd, nnz, npairs, its, levels in st["members"]:
        f1, b1, g1 = roofline.krylov_iteration(nnode, nd, nnz, npairs, tb, levels, float_pairs=fp32)
        kr_flops += f1 * its
        kr_bytes += b1 * its
        kr_f32 += g1 * its
    res_f, tan_f = roofline.element_flops(st["elem"])
    el_kernel = "batch_element_kernel"
    kr_kernel = "bicgstab_grouped_kernel"

    def roof(bound, work, ms, peak, kernel, note):
        if bound == "hbm":
            ach = work / (ms * 1e-3) / 1e9
            return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                    "traffic": traffic_for(kernel, label), "kernel": kernel, "peak_source": pk["hbm_src"],
                    "note": note}
        ach = work / (ms * 1e-3) / 1e12
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": traffic_for(kernel, label), "kernel": kernel,
                "peak_source": ("nominal FP64 pipe of GB300 (1.25 TFLOP/s; an FMA-chain probe measured 1.20)"
                                if peak == pk["fp64_tflops"] else "nominal FP32 pipe of GB300 (75 TFLOP/s)"),
                "note": note}

    # element kernel: every element integration of the timed region over the
    # summed element-launch time, per launch; FP64 pipe, FP32 pipe or bytes,
    # whichever takes longest at its peak
    n_el = max(phase_n["element"], 1)
    el_ms = phase_ms["element"] / n_el
    units = st["elem_integrations"] / n_el                 # elements per launch, on average
    el_bytes = roofline.assembly_bytes(st["elem"], st["nnode"], st["nel"], st["nnz"], tb) * units / st["nel"]
    if fp32:
        cands = {"alu": (units * res_f / (pk["fp64_tflops"] * 1e12), units * res_f, pk["fp64_tflops"]),
                 "alu_fp32": (units * tan_f / (pk["fp32_tflops"] * 1e12), units * tan_f, pk["fp32_tflops"]),
                 "hbm": (el_bytes / (pk["hbm_gbs"] * 1e9), el_bytes, pk["hbm_gbs"])}
    else:
        cands = {"alu": (units * (res_f + tan_f) / (pk["fp64_tflops"] * 1e12), units * (res_f + tan_f),
                         pk["fp64_tflops"]),
                 "hbm": (el_bytes / (pk["hbm_gbs"] * 1e9), el_bytes, pk["hbm_gbs"])}
    b_el = max(cands, key=lambda k: cands[k][0])
    roof_el = roof("hbm" if b_el == "hbm" else "alu", cands[b_el][1], el_ms, cands[b_el][2], el_kernel,
                   f"{units:.0f} element integrations per launch on average"
                   + ("; FP64 residual path on the FP64 pipe (the binding one of FP64 pipe, FP32 pipe, HBM)"
                      if fp32 else "; FP64 residual and tangent"))
    # Krylov kernel: the FP64 arithmetic, the FP32-pipe products (FP32
    # tangent) or the algorithmic bytes, whichever takes longer at its peak
    n_kr = max(phase_n["krylov"], 1)
    kr_ms = phase_ms["krylov"] / n_kr
    its_per_launch = st["krylov_iters"] / n_kr
    t_fl = kr_flops / (pk["fp64_tflops"] * 1e12)
    t_by = kr_bytes / (pk["hbm_gbs"] * 1e9)
    nit = max(st["krylov_iters"], 1)
    note_kr = (f"{its_per_launch:.0f} BiCGSTAB iterations per launch on average (solve and update launches), "
               f"{kr_flops / nit:.4g} FP64 flops, {kr_f32 / nit:.4g} FP32-pipe flops (float-pair SpMV) and "
               f"{kr_bytes / nit:.4g} algorithmic bytes per iteration")
    if t_by > t_fl:
        roof_kr = roof("hbm", kr_bytes / n_kr, kr_ms, pk["hbm_gbs"], kr_kernel, note_kr)
    else:
        roof_kr = roof("alu", kr_flops / n_kr, kr_ms, pk["fp64_tflops"], kr_kernel, note_kr)
    tr = traffic_for(kr_kernel, label)
    roof_kr["traffic"] = (tr * its_per_launch) if tr is not None else None
    roof_dom = roof_kr if phase_ms["krylov"] >= phase_ms["element"] else roof_el

    # the metric: Gauss points over the element-integration and
    # scatter (CSR gather with the Dirichlet rows) time inside the timed
    # region; replicas: every rank's points over the slowest rank's time
    if t_asm_job is None:
        t_asm_job = (phase_ms["element"] + phase_ms["gather"]) * 1e-3
    value = gp_job / t_asm_job if t_asm_job > 0 else None
    setup_ms = phase_ms.get("precond", 0.0)
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_job / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if not fp32 else "f32-tangent/f64",
        "data": "synthetic",
        "config": {"workload": label, "simulations": n_sims, "elements": st["elements"],
                   "gauss_points": sum(m.nel * m.ngp for m in meshes),
                   "ndof": sum(m.ndof for m in meshes), "precision": args.precision,
                   "step": ("one Newton iteration from the initial state" if args.mode == "newton" else
                            "load increment 1 from the initial state, Newton to convergence"),
                   "l2": "flushed (256 MB write) before every step", "parallelism": f"replicas x{world}"},
        "roofline": roof_dom, "roofline_element": roof_el, "roofline_krylov": roof_kr,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(st["launches"]), "clocks": ck,
        "value_definition": "Gauss points integrated in the timed region / the summed CUDA-event time of the "
                            "element-integration and CSR-gather (+ Dirichlet rows) launches in it",
        # the whole step: assembly, preconditioner set-up, Krylov solve and update
        "whole_step": {"value": gp_job / t_job, "unit": UNIT, "ms_per_step": 1e3 * t_job / args.steps,
                       "definition": "Gauss points integrated / device time of the whole steps"},
        "detail": {"newton_iters": st["newton"], "krylov_iters": st["krylov_iters"], "halvings": st["halvings"],
                   "phase_ms": phase_ms, "phase_launches": phase_n, "element_ms_per_launch": el_ms,
                   "preconditioner_setup_ms": setup_ms, "step_ms": step_ms,
                   **({"tuning": st["tuning"]} if "tuning" in st else {})},
    }


def run_serving(args):
    """Continuous-batching FP32-tangent serving against one-at-a-time FP64."""
    import numpy as np
    import torch
    import lgdm_inputs as li
    from paper_2301_06503_gb300 import build
    from paper_2301_06503_gb300.serve import Job, Server, run_one_at_a_time
    torch.cuda.set_device(0)
    build()
    trace = li.serving_trace(seed=4, count=400, rate=20.0, n_steps=300)[:args.requests]

    def jobs():
        return [Job(r.seed_index, r.problem, r.arrival, args.serve_steps) for r in trace]

    clocks = Clocks(0)
    clocks.start()
    opts = dict(max_newton=args.serve_max_newton, max_halvings=args.serve_max_halvings)
    srv = Server(budget_bytes=int(args.budget_gb * (1 << 30)), max_resident=args.max_resident, precision="fp32",
                 **opts)
    js = jobs()
    rep_b = srv.run(js)
    js1 = jobs()
    rep_1 = run_one_at_a_time(js1, precision="fp64", **opts)
    ck = clocks.stop()
    diff = []
    for a, b in zip(sorted(js, key=lambda j: j.rid), sorted(js1, key=lambda j: j.rid)):
        ra, rb = np.asarray(a.reactions), np.asarray(b.reactions)
        if len(ra) == len(rb) and len(rb):
            diff.append(float(np.abs(ra - rb).max() / max(np.abs(rb).max(), 1e-300)))
    line = {"metric": "simulations/hour (served)", "value": rep_b["sims_per_hour"], "unit": "sims/h",
            "higher_is_better": True, "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "serving_mix", "requests": len(trace),
                       "plates": sum(1 for r in trace if r.problem.mesh.elem == 2),
                       "beams": sum(1 for r in trace if r.problem.mesh.elem == 3),
                       "elements": [int(r.problem.mesh.nel) for r in trace],
                       "load_steps_per_sim": args.serve_steps, "schedule": "300 increments to the final load",
                       "arrivals": "Poisson 20/s, seed 4", "budget_gb": args.budget_gb,
                       "max_resident": args.max_resident, "max_newton": args.serve_max_newton,
                       "max_halvings": args.serve_max_halvings},
            "requests_detail": {"served_fp32": srv.records(), "one_at_a_time_fp64": [j.record() for j in js1]},
            "served_fp32_batched": rep_b, "one_at_a_time_fp64": rep_1,
            "speedup_sims_per_hour": rep_b["sims_per_hour"] / rep_1["sims_per_hour"] if rep_1["sims_per_hour"] else None,
            "curve_max_rel_diff_fp32_vs_fp64": max(diff) if diff else None,
            "tuning": srv.tuning, "clocks": ck}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.precision is None:
        args.precision = "fp32" if args.workload == "batch" else "fp64"
    if args.mode is None:
        args.mode = "newton" if args.workload == "batch" else "loadstep"
    if args.serving:
        run_serving(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
