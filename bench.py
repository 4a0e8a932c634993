"""Benchmark of the DMRG superblock Davidson hot path on GB300.

A step is one complete Davidson solve (Algorithm 3 to ||r|| <= 1e-10: projections,
overlaps, small eigenproblem, residual, correction, Gram-Schmidt, restarts) of the
mid-chain superblock of a spin-1/2 Hubbard chain, t = 1, U = 4, half filling, L = 64,
m = 2048 (synthetic operators from the seeded warm-up generator, n = 3.6e6), with the plan
(operation records, device operator arena, diagonal) built once before timing.
The reported value is H*psi throughput over the whole solve: algorithmic projection
FLOPs of all projections of the step divided by the step time.  Default arithmetic: BF16x2
projections (two-term BF16 split, FP32 accumulation) with FP64-accurate anchors on the
tensor cores (FP64_TC), FP64 Davidson scalars; the returned energy is FP64-accurate.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--prec P]
  python bench.py --mode project [--prec P] [--workload NAME]   projections only (profiling)
  python bench.py --mode peaks                                  matmul peak probe

Under torchrun (N > 1) every rank solves its own replica of the workload (no data-path
collective; weak scaling), timed with a barrier and the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "hub_L64_m2048"
WORKLOAD_DESC = "Hubbard chain t=1 U=4 half filling L=64 m=2048, mid-chain LR superblock"
METRIC = "H*psi TFLOP/s over a full Davidson solve (tol 1e-10), Hubbard L=64 m=2048"


def workload_desc(name):
    from dmrg_inputs import warmup
    w = warmup.WORKLOADS[name]
    if w["model"] == "hubbard":
        fill = w.get("filling", 1.0)
        return (f"Hubbard chain t={w.get('t', 1.0):g} U={w.get('U', 4.0):g} "
                f"{'half' if fill == 1.0 else 'quarter' if fill == 0.5 else fill} filling "
                f"L={w['L']} m={w['m']}, mid-chain LR superblock")
    return f"Heisenberg chain J=1 L={w['L']} m={w['m']}, mid-chain LR superblock"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# measured on this machine's GB300 with torch.matmul 8192^3 (cuBLAS dgemm and TF32 GEMM;
# `python bench.py --mode peaks`)
FP64_DGEMM_TFLOPS = 1.10
TF32_TFLOPS = 1006.0
# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) of one low-precision
# projection of the default workload, summed over its launches (pack, the two tcgen05 GEMM
# stages, the split-K reduction when stage 2 splits), keyed by arithmetic and by the tile
# schedules of the two GEMM stages the capture ran with; the traffic of a run whose
# autotuner picked other schedules is not known and is reported as null
TC_TRAFFIC = {
    ("bf16x3", (6, 17)): 535.3e6,
    # BF16x2, captured with `bench.py --mode traffic --prec bf16x2 --scheds ...` under
    # `ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum`
    ("bf16x2", (6, 6)): 306.0e6, ("bf16x2", (6, 7)): 306.4e6, ("bf16x2", (6, 8)): 305.2e6,
    ("bf16x2", (6, 15)): 410.8e6, ("bf16x2", (6, 16)): 360.8e6, ("bf16x2", (6, 17)): 362.4e6,
    ("bf16x2", (7, 6)): 303.8e6, ("bf16x2", (7, 7)): 302.6e6, ("bf16x2", (7, 8)): 302.9e6,
    ("bf16x2", (7, 15)): 408.8e6, ("bf16x2", (7, 16)): 357.4e6, ("bf16x2", (7, 17)): 358.7e6,
    ("bf16x2", (8, 6)): 304.2e6, ("bf16x2", (8, 7)): 302.8e6, ("bf16x2", (8, 8)): 303.6e6,
    ("bf16x2", (8, 15)): 409.8e6, ("bf16x2", (8, 16)): 360.5e6, ("bf16x2", (8, 17)): 358.5e6,
}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, device=None) -> float:
    """The slowest rank's time (weak scaling: every rank solves its own replica)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed divided by the max time."""
    return units_per_rank * world / seconds


def cpu_oracle_projection_sample(sb, x, budget_s=15.0):
    """Time the FP64 oracle's projection (Eq. 11 in NumPy) on the host cores; also returns
    its result, the reference for the projection errors of the GPU arithmetics."""
    from oracle import projection as oproj
    flops = oproj.flop_count(sb)["flops"]
    t0 = time.perf_counter()
    reps = 0
    while True:
        y = oproj.project_blocks(sb, x)
        reps += 1
        if time.perf_counter() - t0 >= budget_s or reps >= 20:
            break
    dt = (time.perf_counter() - t0) / reps
    return flops / dt / 1e12, reps, dt, y


_SINGLE_THREAD_SAMPLE = """
import sys, time
from dmrg_inputs import superblock, warmup
from oracle import projection as oproj
sb = superblock.load_npz(sys.argv[1])
x = warmup.start_vector(sb.n, 0)
budget = float(sys.argv[2])
oproj.project_blocks(sb, x)
t0 = time.perf_counter()
reps = 0
while True:
    oproj.project_blocks(sb, x)
    reps += 1
    if time.perf_counter() - t0 >= budget or reps >= 5:
        break
print((time.perf_counter() - t0) / reps, reps)
"""


def cpu_oracle_single_thread(sb, budget_s=5.0):
    """The same oracle projection with the host BLAS held to one thread: in a subprocess,
    since the thread count of a BLAS that is already loaded cannot be changed portably.
    Returns (TFLOP/s, projections timed, seconds each) or None if the subprocess fails."""
    import tempfile
    from dmrg_inputs import superblock
    from oracle import projection as oproj
    flops = oproj.flop_count(sb)["flops"]
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        with tempfile.TemporaryDirectory() as d:
            path = os.path.join(d, "superblock.npz")
            superblock.save_npz(sb, path)
            r = subprocess.run([sys.executable, "-c", _SINGLE_THREAD_SAMPLE, path, str(budget_s)],
                               env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
        dt, reps = r.stdout.split()[-2:]
        return flops / float(dt) / 1e12, int(reps), float(dt)
    except Exception:
        return None


def workload_config(name, n, flops, ws):
    """The `config` object of a bench line: what defines the workload and its timing, the
    same in both arms (run-specific facts go to the line's `run` object)."""
    return {"workload": name, "desc": workload_desc(name), "n": n,
            "flops_per_projection": flops, "tol": 1e-10, "parallelism": f"replicas x{ws}",
            "l2": f"solve working set (V, W: 2 x 20 x {8 * n / 1e6:.0f} MB) > L2; "
                  "L2 flushed between projection timings"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    from dmrg_inputs import warmup
    from oracle import projection as oproj
    sb = warmup.workload(WORKLOAD)
    x = warmup.start_vector(sb.n, 0)
    flops = oproj.flop_count(sb)["flops"]
    for _ in range(args.warmup):
        oproj.project_blocks(sb, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oproj.project_blocks(sb, x)
    dt = (time.perf_counter() - t0) / args.steps
    val = flops / dt / 1e12
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(WORKLOAD, sb.n, flops, ws),
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": f"each step = one FP64 oracle projection (Eq. 11, NumPy) "
                                   f"of the {WORKLOAD} superblock"},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_peaks():
    """torch.matmul 8192^3 in float64, float32 (SIMT), TF32 and BF16: best of N CUDA-event
    timings.  Used for the FP64 and TF32 roofline denominators."""
    import torch
    torch.cuda.set_device(0)
    out = {}
    for name, dtype, tf32, n, reps in (("fp64", torch.float64, False, 8192, 3),
                                       ("fp32_simt", torch.float32, False, 8192, 5),
                                       ("tf32", torch.float32, True, 8192, 10),
                                       ("bf16", torch.bfloat16, False, 8192, 10)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device="cuda", dtype=dtype)
        b = torch.randn(n, n, device="cuda", dtype=dtype)
        for _ in range(2):
            a @ b
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        out[name] = 2 * n ** 3 / best / 1e12
        del a, b
    print(json.dumps({"mode": "peaks", "unit": "TFLOP/s", **out}), flush=True)


def run_project(args):
    """Projections only, in one precision, on one workload (the launch used for ncu)."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from dmrg_inputs import warmup
    from paper_1309_5571_gb300 import Plan
    prec = "bf16x2" if args.prec == "auto" else args.prec
    sb = warmup.workload_l11r(args.workload) if args.strategy == "l11r" else warmup.workload(args.workload)
    x = torch.from_numpy(warmup.start_vector(sb.n, 0)).cuda()
    y = torch.empty_like(x)
    plan = Plan(sb, prec=prec, graphs=not args.no_graphs)
    if prec in ("bf16x3", "bf16x2", "tf32"):
        if args.sched:   # pinned tile schedules: no autotuning launches before the timed ones
            s1, s2 = (int(v) for v in args.sched.split(","))
            plan.set_tile_schedule(s1, s2, prec=prec)
        else:
            plan.autotune(prec)
    for _ in range(args.warmup):
        plan.project(x, y, prec=prec)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()   # profiler range = the timed projections only
    e0.record()
    for _ in range(args.steps):
        plan.project(x, y, prec=prec)
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    t = e0.elapsed_time(e1) / 1e3 / args.steps
    print(json.dumps({"mode": "project", "workload": args.workload, "strategy": args.strategy,
                      "prec": prec, "n": sb.n, "records": plan.stats["records"],
                      "flops": plan.stats["flops"],
                      "ms": t * 1e3, "tflops": plan.stats["flops"] / t / 1e12,
                      "graphs": not args.no_graphs,
                      "tc_schedule": plan.get_stats()["tc_schedule"]}), flush=True)


def run_traffic(args):
    """One projection per listed tile schedule, each alone inside the CUDA profiler range,
    for `ncu --profile-from-start off --metrics dram__bytes_read.sum,dram__bytes_write.sum`:
    the DRAM traffic of the projection's launches under each schedule (the source of the
    TC_TRAFFIC table).  Prints the schedules in capture order."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from dmrg_inputs import warmup
    from paper_1309_5571_gb300 import Plan
    prec = "bf16x2" if args.prec == "auto" else args.prec
    sb = warmup.workload(args.workload)
    x = torch.from_numpy(warmup.start_vector(sb.n, 0)).cuda()
    y = torch.empty_like(x)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    plan = Plan(sb, prec=prec, graphs=False)
    order = []
    for spec in args.scheds.split(":"):
        s1, s2 = (int(v) for v in spec.split(","))
        plan.set_tile_schedule(s1, s2, prec=prec)
        for _ in range(2):
            plan.project(x, y, prec=prec)
        flush.zero_()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        plan.project(x, y, prec=prec)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        order.append([s1, s2])
    print(json.dumps({"mode": "traffic", "workload": args.workload, "prec": prec,
                      "schedules_in_capture_order": order}), flush=True)


def run_batched(args):
    """Uneven batch of independent Heisenberg superblocks (L = 100, m drawn from
    {256, 512, 1024, 2048} with seed 1234): one batched solve versus the same solves one
    after the other."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from dmrg_inputs import warmup
    from paper_1309_5571_gb300 import Plan, solve_batched
    prec = "bf16x2" if args.prec == "auto" else args.prec
    sbs, ms, x0s = warmup.batched_workload(count=args.batch)
    # one plan (and scratch) per problem
    plist = [Plan(sb, prec=prec, anchor_prec=args.anchor) for sb in sbs]
    xs = [torch.from_numpy(x).cuda() for x in x0s]
    flops = sum(p.stats["flops"] for p in plist)
    solve_batched(plist, xs, raise_on_nonconvergence=False)  # warm-up (operand images)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    outs, infos = solve_batched(plist, xs, raise_on_nonconvergence=False)
    torch.cuda.synchronize()
    t_b = time.perf_counter() - t0
    t0 = time.perf_counter()
    for p, x in zip(plist, xs):
        p.solve(x, raise_on_nonconvergence=False)
    torch.cuda.synchronize()
    t_s = time.perf_counter() - t0
    proj = sum(i["projections"] + i["fp64_projections"] for i in infos)
    print(json.dumps({"mode": "batched", "problems": len(plist), "m": sorted(set(ms)),
                      "m_counts": {int(m): ms.count(m) for m in sorted(set(ms))},
                      "prec": prec, "anchor": args.anchor, "batched_s": t_b, "sequential_s": t_s,
                      "speedup": t_s / t_b, "all_converged": all(i["converged"] for i in infos),
                      "projections": proj,
                      "hpsi_tflops_batched": sum(i["projections"] + i["fp64_projections"]
                                                 for i in infos) and
                      sum((i["projections"] + i["fp64_projections"]) * p.stats["flops"]
                          for i, p in zip(infos, plist)) / t_b / 1e12}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--prec", default="auto", choices=["auto", "fp64", "tf32", "bf16x3", "bf16x2", "fp64tc"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-l11r", action="store_true",
                    help="skip the l-1-1-r form of the workload in the solve report")
    ap.add_argument("--proj-reps", type=int, default=10)
    ap.add_argument("--mode", default="solve", choices=["solve", "project", "peaks", "batched", "traffic"])
    ap.add_argument("--scheds", default="6,7:6,16:8,7:8,16:7,6:6,8:6,6:7,7:8,8",
                    help="--mode traffic: tile schedules 'S1,S2:S1,S2:...'")
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--anchor", default="fp64tc", choices=["fp64", "fp64tc"],
                    help="FP64-accurate projections of the mixed modes")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--sched", default="", help="--mode project: pin the tile schedules 'S1,S2'")
    ap.add_argument("--strategy", default="lr", choices=["lr", "l11r"],
                    help="--mode project: the LR form (Eq. 11) or the l-1-1-r form (Eq. 13)")
    ap.add_argument("--no-graphs", action="store_true",
                    help="--mode project: launch the projection kernels directly")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "peaks":
        return run_peaks()
    if args.mode == "project":
        return run_project(args)
    if args.mode == "batched":
        return run_batched(args)
    if args.mode == "traffic":
        return run_traffic(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")

    import __graft_entry__
    __graft_entry__.build()
    from dmrg_inputs import warmup
    from paper_1309_5571_gb300 import Plan, capi

    lib = capi.load()
    prec = args.prec
    if prec == "auto":
        # BF16x2 projections with FP64-accurate anchors: the fastest solve of the arithmetics
        # (the per-arithmetic report of this line measures all of them), golden-tested
        prec = "bf16x2" if capi.tc_available() else "fp64"
    sb = warmup.workload(args.workload)
    # the timed steps cycle through up to 8 start vectors: the iteration count of a mixed
    # solve moves with rounding-level changes, so one start vector alone is a noisy sample
    seeds = [rank * 1000 + s for s in range(max(1, min(args.steps, 8)))]
    x0 = warmup.start_vector(sb.n, seed=seeds[0])
    x0_t = torch.from_numpy(x0).cuda()
    x0s_t = [x0_t] + [torch.from_numpy(warmup.start_vector(sb.n, seed=sd)).cuda() for sd in seeds[1:]]
    stream = torch.cuda.current_stream()

    t0 = time.perf_counter()
    plan = Plan(sb, prec=prec, tol=1e-10, anchor_prec=args.anchor)
    torch.cuda.synchronize()
    plan_ms = (time.perf_counter() - t0) * 1e3
    flops = plan.stats["flops"]

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- warm-up solves
    for _ in range(args.warmup):
        x, info = plan.solve(x0_t)
    barrier()
    # ---- timed solves (whole hot path), device-resident inputs
    infos = []
    launches0 = capi.kernel_launches()
    with ClockSampler(local) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier()
        # profiler range = the timed solves only (ncu --profile-from-start off); no effect
        # without a profiler
        torch.cuda.profiler.start()
        ev0.record(stream)
        step_ms = []
        for s in range(args.steps):
            ts = time.perf_counter()
            x, info = plan.solve(x0s_t[s % len(x0s_t)])
            step_ms.append((time.perf_counter() - ts) * 1e3)
            infos.append(info)
        ev1.record(stream)
        barrier()
        torch.cuda.profiler.stop()
    launches = capi.kernel_launches() - launches0
    t_step = max_over_ranks(ev0.elapsed_time(ev1) / 1e3 / args.steps, device="cuda")
    proj_per_step = statistics.mean(i["projections"] + i["fp64_projections"] for i in infos)
    value = job_throughput(proj_per_step * flops, ws, t_step) / 1e12

    # ---- end to end through the host-buffer entry point: every step copies its start
    # vector from pinned host memory to the device and the result back inside the timing
    # (the same K steps and start vectors as above; one untimed call first)
    xh_in = [torch.empty(sb.n, dtype=torch.float64).pin_memory() for _ in x0s_t]
    for h, d in zip(xh_in, x0s_t):
        h.copy_(d.cpu())
    xh_out = torch.empty(sb.n, dtype=torch.float64).pin_memory()
    plan.solve_host(xh_in[0].numpy(), xh_out.numpy())
    barrier()
    te = time.perf_counter()
    e2e_proj = 0
    for s in range(args.steps):
        _, infoh = plan.solve_host(xh_in[s % len(xh_in)].numpy(), xh_out.numpy())
        e2e_proj += infoh["projections"] + infoh["fp64_projections"]
    barrier()
    t_e2e = max_over_ranks((time.perf_counter() - te) / args.steps, device="cuda")
    e2e_val = job_throughput(e2e_proj / args.steps * flops, ws, t_e2e) / 1e12

    # ---- the dominant kernel: the projection (all its launches), timed alone in every
    # arithmetic, L2 flushed before each
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x0_t)
    proj, proj_out = {}, {}
    variants = ["fp64", "tf32", "bf16x3", "bf16x2", "fp64tc"]
    for p in variants:
        for _ in range(2):
            plan.project(x0_t, y, prec=p)
        times = []
        for _ in range(args.proj_reps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.project(x0_t, y, prec=p)
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b) / 1e3)
        proj[p] = statistics.mean(times)
        proj_out[p] = y.cpu().numpy()

    # ---- full solves in the other arithmetics (the FP64 path is the comparison arm of the
    # metric), over the same start vectors as the first timed steps, one plan each
    nvar = min(3, len(x0s_t))
    solves = {}
    for name, opts in (("fp64", dict(prec="fp64")),
                       ("fp64tc", dict(prec="fp64tc")),
                       ("tf32", dict(prec="tf32", anchor_prec=args.anchor)),
                       ("bf16x3", dict(prec="bf16x3", anchor_prec=args.anchor)),
                       ("bf16x2", dict(prec="bf16x2", anchor_prec=args.anchor))):
        if name == prec:
            solves[name] = {"ms": [i_ms for i_ms in step_ms[:nvar]],
                            "iters": [i["iters"] for i in infos[:nvar]],
                            "energy": [i["energy"] for i in infos[:nvar]]}
        else:
            pv = Plan(sb, tol=1e-10, **opts)
            pv.solve(x0s_t[0])  # builds and tunes the plan's operand images
            ms_l, it_l, e_l = [], [], []
            for sv in range(nvar):
                torch.cuda.synchronize()
                a = time.perf_counter()
                _, iv = pv.solve(x0s_t[sv])
                torch.cuda.synchronize()
                ms_l.append((time.perf_counter() - a) * 1e3)
                it_l.append(iv["iters"])
                e_l.append(iv["energy"])
            pv.close()
            solves[name] = {"ms": ms_l, "iters": it_l, "energy": e_l}
        solves[name]["mean_ms"] = statistics.mean(solves[name]["ms"])
    fp64_solve_ms = solves["fp64"]["mean_ms"]
    e_fp64 = solves["fp64"]["energy"][0]

    # ---- the same superblock in the l-1-1-r form (Sec. 4.2): projection and solves with the
    # run's arithmetic, over the same start vectors (the same Hamiltonian, so the same energy)
    l11r = None
    if not args.no_l11r:
        sb4 = warmup.workload_l11r(args.workload)
        p4 = Plan(sb4, prec=prec, tol=1e-10, anchor_prec=args.anchor)
        for _ in range(2):
            p4.project(x0_t, y, prec=prec)
        t4 = []
        for _ in range(args.proj_reps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            p4.project(x0_t, y, prec=prec)
            b.record(stream)
            torch.cuda.synchronize()
            t4.append(a.elapsed_time(b) / 1e3)
        p4.solve(x0s_t[0])
        ms4, it4, e4 = [], [], []
        for sv in range(nvar):
            torch.cuda.synchronize()
            a = time.perf_counter()
            _, iv = p4.solve(x0s_t[sv])
            torch.cuda.synchronize()
            ms4.append((time.perf_counter() - a) * 1e3)
            it4.append(iv["iters"])
            e4.append(iv["energy"])
        l11r = {"records": p4.stats["records"], "flops_per_projection": p4.stats["flops"],
                "projection_ms": statistics.mean(t4) * 1e3,
                "projection_tflops": p4.stats["flops"] / statistics.mean(t4) / 1e12,
                "solve_ms": statistics.mean(ms4), "solve_ms_each": ms4, "iters": it4,
                "dE_vs_fp64_path": max(abs(e - e_fp64) for e in e4),
                "start_vector_seeds": seeds[:nvar], "prec": prec}
        p4.close()

    pk, pk_kind = peaks()
    if prec == "fp64":
        bound, peak, unit = "alu", FP64_DGEMM_TFLOPS, "TFLOP/s"
        peak_note = "measured cuBLAS dgemm 8192^3 on this pool's GB300 (FP64 units)"
    elif prec == "tf32":
        bound, peak, unit = "tensor", TF32_TFLOPS, "TFLOP/s"
        peak_note = "measured cuBLAS TF32 8192^3 on this pool's GB300"
    elif prec == "bf16x2":
        bound, peak, unit = "tensor", pk["bf16_tflops"] / 3.0, "TFLOP/s"
        peak_note = f"{pk_kind} bf16 burst / 3 products (algorithmic FLOPs of a BF16x2 GEMM)"
    else:
        bound, peak, unit = "tensor", pk["bf16_tflops"] / 6.0, "TFLOP/s"
        peak_note = f"{pk_kind} bf16 burst / 6 products (algorithmic FLOPs of a BF16x3 GEMM)"
    achieved = flops / proj[prec] / 1e12
    sched = tuple(plan.get_stats()["tc_schedule"])
    traffic = TC_TRAFFIC.get((prec, sched)) if args.workload == WORKLOAD else None
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": traffic, "kernel": f"projection ({prec})",
                "peak_source": peak_note, "tc_schedule": list(sched),
                "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the "
                                   f"projection launches, captured with tile schedules {list(sched)}")
                if traffic else ("no ncu capture of these kernels with the tile schedules this run "
                                 f"picked ({list(sched)})")}

    # ---- CPU oracle baseline (rank 0, N = 1 only), bounded sample; its output is the
    # reference for the projection error of every GPU arithmetic
    cpu = None
    proj_err = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        val, reps, dt, y_ref = cpu_oracle_projection_sample(sb, x0)
        cpu = {"value": val, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{reps} FP64 oracle projections (NumPy, Eq. 11) of the same "
                         f"superblock, {dt:.2f} s each"}
        one = cpu_oracle_single_thread(sb)
        cpu["single_thread"] = None if one is None else {
            "value": one[0], "unit": "TFLOP/s", "cores": 1,
            "sample": f"{one[1]} projections with the host BLAS held to one thread, "
                      f"{one[2]:.2f} s each"}
        ymax = float(np.max(np.abs(y_ref)))
        proj_err = {p: float(np.max(np.abs(proj_out[p] - y_ref)) / ymax) for p in variants}

    e_ref = infos[0]["energy"]  # start vector seeds[0], as the FP64-path solve
    if rank == 0:
        line = {
            "metric": METRIC if args.workload == WORKLOAD else
                      f"H*psi TFLOP/s over a full Davidson solve (tol 1e-10), {args.workload}",
            "value": value, "unit": "TFLOP/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else f"{prec}+f64",
            "data": "synthetic (seeded warm-up generator; operators shaped like the paper's runs)",
            "config": workload_config(args.workload, sb.n, flops, ws),
            "run": {"prec": prec, "anchor_prec": args.anchor, "records": plan.stats["records"],
                    "tc_schedule": plan.get_stats()["tc_schedule"],
                    "device_gb": (plan.get_stats()["device_bytes"] + 8 * 44 * sb.n) / 1e9},
            "solve": {"ms": t_step * 1e3, "start_vector_seeds": seeds,
                      "iters": statistics.mean(i["iters"] for i in infos),
                      "iters_per_step": [i["iters"] for i in infos],
                      "projections": statistics.mean(i["projections"] for i in infos),
                      "fp64_projections": statistics.mean(i["fp64_projections"] for i in infos),
                      "anchor_updates": statistics.mean(i["anchor_updates"] for i in infos),
                      "restarts": statistics.mean(i["restarts"] for i in infos), "energy": e_ref,
                      "resnorm": max(i["resnorm"] for i in infos), "plan_ms": plan_ms,
                      "fp64_path_solve_ms": fp64_solve_ms, "fp64_path_energy": e_fp64,
                      "fp64_path_iters": solves["fp64"]["iters"],
                      "dE_vs_fp64_path": abs(e_ref - e_fp64),
                      "dE_between_steps": max(abs(i["energy"] - e_ref) for i in infos),
                      "speedup_vs_fp64_path": fp64_solve_ms / statistics.mean(solves[prec]["ms"]),
                      "speedup_note": f"FP64-path solve vs this arithmetic's solve, both over start "
                                      f"vectors {seeds[:nvar]} (host wall clock per solve)"},
            "variants": {p: {"projection_ms": proj[p] * 1e3,
                             "projection_tflops": flops / proj[p] / 1e12,
                             "projection_err_vs_oracle": proj_err[p] if proj_err else None,
                             "solve_ms": solves[p]["mean_ms"], "solve_ms_each": solves[p]["ms"],
                             "iters": solves[p]["iters"],
                             "dE_vs_fp64_path": max(abs(e - e_fp64) for e in solves[p]["energy"])}
                         for p in variants},
            "projection_ms": {p: v * 1e3 for p, v in proj.items()},
            "l11r": l11r,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "TFLOP/s", "h2d_bytes_per_step": 8 * sb.n,
                    "d2h_bytes_per_step": 8 * sb.n, "ms": t_e2e * 1e3,
                    "host_buffers": "pinned", "steps": args.steps},
            "clocks": clk.summary(),
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
