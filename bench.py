#!/usr/bin/env python
"""Throughput of the LGDM hot path on GB300.

Workload: the notched plate (200 x 200 four-node quads, plane strain, 40k
elements, 160k Gauss points, 121k dofs).  A timed step solves one load
increment (0.1 mm / 500) from the initial state: device-side reset of the
state, the Dirichlet predictor, Newton iterations until convergence -- each
one element integration at every Gauss point, deterministic CSR assembly
with Dirichlet rows, node-block Jacobi set-up, and one persistent BiCGSTAB
launch with the fused update and convergence test -- then the history commit
and the reaction.  The metric counts Gauss-point integrations with assembly:
every Newton iteration integrates nel * ngp points.  Inputs are resident in
HBM when the timed region starts; L2 is flushed (256 MB write) before each
step.  The e2e figure drives the same step through the public API from
pinned host buffers (state in, damage field and reaction out).

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
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--workload", default="plate", choices=["plate", "bar", "beam"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="loadstep", choices=["loadstep", "newton"],
                    help="loadstep: a step is a converged load increment; newton: one Newton iteration "
                         "(assemble + solve + update), used for profiling captures")
    ap.add_argument("--max-krylov", type=int, default=5000,
                    help="BiCGSTAB iteration cap (profiling captures use a small cap)")
    return ap.parse_args()


def workload(name):
    import lgdm_inputs as li
    if name == "plate":
        return li.sen_plate_problem(), "sen_plate_q4_200x200"
    if name == "bar":
        return li.bar_problem(), "bar_l2_100"
    return li.tpb_beam_problem(), "tpb_beam_h8_200x40x40"


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


def traffic_for(kernel):
    """DRAM bytes per launch from a committed ncu summary, if the kernels are unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path))
        if rec.get("csrc_sha") != csrc_sha():
            return None
        return rec["kernels"].get(kernel)
    except (ValueError, KeyError):
        return None


def csrc_sha():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2301_06503_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def cpu_baseline(problem, label, newton_iters=2):
    """The oracle as it stands: the first Newton iterations of load step 1 (bounded sample)."""
    from oracle import assembly as asm
    from oracle import newton as nw
    import scipy.sparse.linalg as spla
    st = nw.initial_state(problem)
    u = st.u.copy()
    u[problem.bcs.dir_dof] = problem.bcs.dir_scale * problem.load(1)
    t0 = time.perf_counter()
    for _ in range(newton_iters):
        K, r = asm.assemble(problem.mesh, problem.material, u, st.kappa_hist)
        Kb, rb = asm.apply_dirichlet(K, r, problem.bcs.dir_dof)
        u += spla.spsolve(Kb.tocsc(), -rb)
    dt = time.perf_counter() - t0
    gp = newton_iters * problem.mesh.nel * problem.mesh.ngp
    return {"value": gp / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{label}: first {newton_iters} Newton iterations of load step 1 "
                      f"(numpy element integration + scipy SuperLU direct solve), {dt:.1f} s"}


def run_reference(args):
    """Reference arm: the CPU oracle, one Newton iteration per step (bounded sample)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import assembly as asm
    from oracle import newton as nw
    import numpy as np
    import scipy.sparse.linalg as spla
    p, label = workload(args.workload)
    st = nw.initial_state(p)
    u0 = st.u.copy()
    u0[p.bcs.dir_dof] = p.bcs.dir_scale * p.load(1)

    def step():
        K, r = asm.assemble(p.mesh, p.material, u0, st.kappa_hist)
        Kb, rb = asm.apply_dirichlet(K, r, p.bcs.dir_dof)
        du = spla.spsolve(Kb.tocsc(), -rb)
        return float(np.linalg.norm(du))

    for _ in range(args.warmup):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    gp = p.mesh.nel * p.mesh.ngp
    value = gp * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": label, "step": "one Newton iteration (assemble + direct solve) at load step 1",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{label}: {args.steps} Newton iterations at load step 1"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2301_06503_gb300 import Sim, build, roofline
    if rank == 0:
        build()
    if world > 1:
        torch.distributed.barrier()
    build()
    p, label = workload(args.workload)
    m = p.mesh
    sim = Sim(m, p.material, p.bcs, precision=args.precision, max_krylov=args.max_krylov)
    stream = sim.stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    load = p.load(1)

    if args.mode == "newton":
        def step():
            sim.reset_state()
            sim.begin_step(load)
            sim.newton_step()
            return 0.0
    else:
        def step():
            sim.reset_state()
            sim.run_step(load)
            return sim.reaction()

    for _ in range(args.warmup):
        step()
    sim.enable_timers(True)
    sim.timers(reset=True)
    c0 = sim.counters()
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
            step()
            ends[k].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    c1 = sim.counters()
    tm = sim.timers()
    newton = c1["assemblies"] - c0["assemblies"]
    gp = newton * m.nel * m.ngp
    t_s = sum(step_ms) / 1e3
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([t_s, float(gp)], device="cuda", dtype=torch.float64)
        tmax = tt.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(tt, op=dist.ReduceOp.SUM)
        t_job, gp_job = float(tmax[0]), float(tt[1])
    else:
        t_job, gp_job = t_s, float(gp)
    value = gp_job / t_job

    # ------------------------------------------------ roofline of the dominant kernel
    pk = peaks()
    tb = 4 if args.precision == "fp32" else 8
    sz = sim.sizes
    phase_ms = {k: v[0] for k, v in tm.items()}
    dom = max(("element", "krylov"), key=lambda k: phase_ms[k])
    kiters = c1["krylov_iters"] - c0["krylov_iters"]
    fl_k, by_k = roofline.krylov_iteration(int(sz.nnode), int(sz.nd), int(sz.nnz), int(sz.npairs), tb)
    res_f, tan_f = roofline.element_flops(m.elem)

    def roof_alu(flops_per_launch, ms_per_launch, peak_tf, kernel):
        ach = flops_per_launch / (ms_per_launch * 1e-3) / 1e12
        return {"bound": "alu", "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s", "frac": ach / peak_tf,
                "traffic": traffic_for(kernel), "kernel": kernel,
                "peak_source": "nominal FP64 pipe of GB300 (1.25 TFLOP/s); an FMA-chain probe measured 1.20"}

    def roof_hbm(bytes_per_launch, ms_per_launch, kernel):
        ach = bytes_per_launch / (ms_per_launch * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"], "traffic": traffic_for(kernel), "kernel": kernel,
                "peak_source": pk["hbm_src"]}

    el_ms = phase_ms["element"] / max(tm["element"][1], 1)
    el_flops = m.nel * (res_f + (tan_f if args.precision == "fp64" else 0))
    roof_el = roof_alu(el_flops, el_ms, pk["fp64_tflops"], "element_kernel")
    kr_ms = phase_ms["krylov"] / max(tm["krylov"][1], 1)
    kr_per_launch = kiters / max(tm["krylov"][1], 1)
    if args.precision == "fp64":
        roof_kr = roof_alu(fl_k * kr_per_launch, kr_ms, pk["fp64_tflops"], "bicgstab_kernel")
    else:
        roof_kr = roof_hbm(by_k * kr_per_launch, kr_ms, "bicgstab_kernel")
    roof = roof_kr if dom == "krylov" else roof_el

    # ------------------------------------------------ end to end through the public API
    e2e = None
    if rank == 0:
        u0 = torch.zeros(m.ndof, dtype=torch.float64).pin_memory().numpy()
        kh0 = torch.full((m.nel * m.ngp,), p.material.kappa0, dtype=torch.float64).pin_memory().numpy()
        e_times, e_gp = [], 0
        for k in range(max(1, min(args.steps, 5))):
            cn0 = sim.counters()["assemblies"]
            t0 = time.perf_counter()
            sim.set_state(u0, kh0)                           # state in (pinned host -> device)
            if args.mode == "newton":
                sim.begin_step(load)
                sim.newton_step()
            else:
                sim.run_step(load)
            dmg = sim.field("damage")                        # damage field out
            sim.reaction()                                   # load-displacement point out
            e_times.append(time.perf_counter() - t0)
            e_gp += (sim.counters()["assemblies"] - cn0) * m.nel * m.ngp
        e2e = {"value": e_gp / sum(e_times), "unit": UNIT, "h2d_bytes_per_step": int(u0.nbytes + kh0.nbytes),
               "d2h_bytes_per_step": int(dmg.nbytes + 8)}
    sim.close()

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(p, label)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_job / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32-tangent/f64",
        "data": "synthetic",
        "config": {"workload": label, "nel": m.nel, "gauss_points": m.nel * m.ngp, "ndof": m.ndof,
                   "precision": args.precision, "step": "load increment 1 of 500 from the initial state, Newton to convergence",
                   "l2": "flushed (256 MB write) before every step", "parallelism": f"replicas x{world}"},
        "roofline": roof, "roofline_element": roof_el, "roofline_krylov": roof_kr,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(c1["kernel_launches"] - c0["kernel_launches"]),
        "clocks": ck,
        "detail": {"newton_iters": newton, "krylov_iters": kiters, "halvings": c1["halvings"] - c0["halvings"],
                   "phase_ms": phase_ms, "phase_launches": {k: v[1] for k, v in tm.items()},
                   "element_ms_per_launch": el_ms, "assembly_gp_per_s": m.nel * m.ngp / (
                       (phase_ms["element"] + phase_ms["gather"] + phase_ms["precond"]) / max(tm["element"][1], 1) * 1e-3),
                   "step_ms": step_ms},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
