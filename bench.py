"""Benchmark: warm-started HJI reachability solves on the GB300.

One bench step is one whole solve through the C ABI (set-up reductions for
alpha and dt, init V0 = min(k, l), the fused ENO/WENO + Hamiltonian + LF +
RK-stage + min(l) march, and the max|dV| convergence test until it stops) of
the 1001 x 1001 double integrator with disturbance |d| <= 0.2, WENO5 / RK3,
CFL 0.5, tol 1e-6, warm-started from the d = 0 solution (computed once,
outside the timed region).  The metric is cell-updates/s: nodes x steps
advanced per second.  Inputs are synthetic and seeded (workloads/).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision f32|f64]
    python bench.py --impl reference   # the FP64 CPU oracle on a bounded sample

Under torchrun (N > 1) every rank solves its own instance (independent
problems: weak scaling, no collective on the data path); the job's value is
the cell-updates of all ranks over the slowest rank's time.
"""
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

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

N_SIDE, DMAX = 1001, 0.2
SOLVE = dict(scheme="weno5", rk=3, cfl=0.5, tol=1e-6, max_steps=200000, check_every=32)
WORKLOAD = ("double integrator x1'=x2, x2'=u+d, |u|<=1, |d|<=0.2, 1001x1001 on [-2,2]^2, "
            "l=1-|x1|, WENO5/RK3, cfl 0.5, tol 1e-6, warm start from the d=0 solution")
# Algorithmic work of one node through one RK stage of WENO5 in 2-D, counted
# from the textbook formulas (FP operations: +, -, *, /, max, abs):
#   per axis: 6 differences, 2 x 78 for the two WENO5 reconstructions
#   (15 candidates, 33 smoothness, 11 epsilon, 9 raw weights, 10 normalise
#   and combine), 2 scalings by 1/dx -> 164;  two axes -> 328;
#   Hamiltonian (averaged gradient 4, drift 8, <p,f0> 3, control 6,
#   disturbance 6) -> 27;  Lax-Friedrichs 6;  Euler stage 2;  RK combine 3;
#   min(., l), |dV| and max 4.
FLOPS_PER_NODE_STAGE = 328 + 27 + 6 + 2 + 3 + 4
# Algorithmic memory words per node per RK3 step with per-stage kernels.
# FP64 (stage states): stage 1 reads V, writes W1; stage 2 reads W1, V,
# writes W2; stage 3 reads W2, V, l, writes V' -> 9 words (72 B).
# FP32 (compensated hi/lo value, stage increments): stage 1 reads hi, lo,
# writes D1; stage 2 reads hi, lo, D1, writes D2; stage 3 reads hi, lo, D2,
# l, writes hi', lo' -> 13 words (52 B).
WORDS_PER_NODE_STEP = {"f64": 9, "f32": 13}


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                self.rows.append([c.strip() for c in line.split(",")])

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def reduce_over_ranks(dist, torch, ms, updates, device):
    """Job-level timing for independent per-rank instances: the slowest
    rank's time and the sum of every rank's cell-updates."""
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(updates)], device=device, dtype=torch.float64)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def _flush_l2(torch, buf):
    buf.add_(1)  # 512 MB written: larger than the 129 MB L2


def cpu_baseline(n_steps=None, budget_s=15.0):
    """The FP64 oracle as it stands, on a bounded sample of the same workload:
    `n_steps` RK3 steps of the 1001^2 WENO5 march (from V0 = l: a step costs
    the same whatever the start)."""
    import oracle
    gd, dyn, l = W.di_config(N_SIDE, dmax=DMAX)
    P = oracle.problem(gd, dyn)
    alpha, dt = oracle.alpha_dt(P, SOLVE["cfl"])
    V = oracle.init(P, l)
    cells = W.num_cells(gd)
    t0 = time.perf_counter()
    steps = 0
    while True:
        V, _ = oracle.step(P, "weno5", 3, dt, alpha, l, V)
        steps += 1
        el = time.perf_counter() - t0
        if (n_steps is not None and steps >= n_steps) or (n_steps is None and el >= budget_s):
            break
    return {"value": cells * steps / el, "unit": "cell-updates/s", "cores": oracle.max_threads(),
            "kind": "oracle",
            "sample": "%d WENO5/RK3 FP64 steps of the 1001^2 double-integrator march "
                      "(%.1f s on the host cores)" % (steps, el)}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    samples = []
    for _ in range(args.warmup):
        cpu_baseline(n_steps=1)
    t_all = 0.0
    cells = 0
    for _ in range(args.steps):
        r = cpu_baseline(n_steps=4)
        samples.append(r)
        steps = int(r["sample"].split()[0])
        t_all += W.num_cells(W.di_config(N_SIDE, dmax=DMAX)[0]) * steps / r["value"]
        cells += W.num_cells(W.di_config(N_SIDE, dmax=DMAX)[0]) * steps
    value = cells / t_all
    line = {"impl": "reference", "metric": "cell-updates/s", "value": value,
            "unit": "cell-updates/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "nodes": W.num_cells(W.di_config(N_SIDE, dmax=DMAX)[0]),
                       "sample": "each step: 4 RK3 steps of the march by the FP64 oracle on the "
                                 "host cores"},
            "cpu_baseline": {"value": value, "unit": "cell-updates/s",
                             "cores": samples[-1]["cores"], "kind": "oracle",
                             "sample": samples[-1]["sample"]},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="profiling aid: run only this many steps of the workload's march "
                         "with each RK stage kernel launched on its own (hji_stage_times), "
                         "from V0 = l, and print their mean durations; no bench line")
    ap.add_argument("--workload", default="di1001",
                    choices=["di1001", "quad61", "batch256", "di8192"],
                    help="di1001: whole warm-started solves of the 1001^2 double integrator "
                         "(default); quad61 / batch256 / di8192: 50-step FP32 marches of the "
                         "HBM-bound 61^4 quadrotor subsystem / 256 uneven double integrators / "
                         "8192^2 double integrator")
    args = ap.parse_args()

    rank, world = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import paper_1903_07715_gb300 as hji

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    hji.load()
    if args.profile_steps > 0:
        return profile_stages(args, hji, torch)
    if args.workload != "di1001":
        return run_hbm_workload(args, hji, torch, dist, rank, world, local_rank)

    prec = args.precision
    npdt = np.float32 if prec == "f32" else np.float64
    tdt = torch.float32 if prec == "f32" else torch.float64
    gd, dyn, l = W.di_config(N_SIDE, dmax=DMAX)
    _, dyn0, _ = W.di_config(N_SIDE, dmax=0.0)
    cells = W.num_cells(gd)
    esize = np.dtype(npdt).itemsize

    # Warm start k: the converged d = 0 solution (an input, computed untimed).
    g = hji.Grid(gd, prec)
    g.set_dynamics(dyn0)
    l_dev = torch.from_numpy(l.astype(npdt)).cuda()
    g.solve(l_dev, **SOLVE)
    k_dev = torch.empty_like(l_dev)
    g.value(k_dev)
    g.set_dynamics(dyn)
    # Tile shape for this problem class, picked once by the autotuner (untimed).
    tuned, tune_ms = g.autotune(l_dev, steps=30, **{k: v for k, v in SOLVE.items()
                                                   if k not in ("max_steps", "check_every")})

    stream = torch.cuda.current_stream()
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def timed_solves(n, host=False):
        total_ms, updates, launches, stats = 0.0, 0, 0, []
        if host:
            l_h = torch.empty(l_dev.shape, dtype=tdt, pin_memory=True)
            l_h.copy_(l_dev)
            k_h = torch.empty(l_dev.shape, dtype=tdt, pin_memory=True)
            k_h.copy_(k_dev)
            out_h = torch.empty(l_dev.shape, dtype=tdt, pin_memory=True)
            l_np, k_np, out_np = l_h.numpy(), k_h.numpy(), out_h.numpy()
        for _ in range(n):
            _flush_l2(torch, flush)
            torch.cuda.synchronize()
            if dist is not None:
                dist.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if host:
                st = g.solve(l_np, k_np, **SOLVE)
                g.value(out_np)
            else:
                st = g.solve(l_dev, k_dev, **SOLVE)
            e1.record(stream)
            torch.cuda.synchronize()
            total_ms += e0.elapsed_time(e1)
            updates += cells * st["steps"]
            launches += st["kernel_launches"]
            stats.append(st)
        return total_ms, updates, launches, stats

    timed_solves(args.warmup)
    clocks = ClockSampler(local_rank)
    clocks.start()
    ms, updates, launches, stats = timed_solves(args.steps)
    clk = clocks.stop()
    if dist is not None:
        ms, updates = reduce_over_ranks(dist, torch, ms, updates, "cuda")
    value = updates / (ms / 1000.0)

    e2e_ms, e2e_updates, _, _ = timed_solves(max(1, args.steps), host=True)
    e2e = {"value": e2e_updates / (e2e_ms / 1000.0), "unit": "cell-updates/s",
           "h2d_bytes_per_step": 2 * cells * esize, "d2h_bytes_per_step": cells * esize}

    steps_per_solve = statistics.mean(s["steps"] for s in stats)
    stage_launches_with_work = steps_per_solve * SOLVE["rk"]
    avg_stage_ms = (ms / args.steps) / stage_launches_with_work
    flops = FLOPS_PER_NODE_STAGE * cells
    achieved_tflops = flops / (avg_stage_ms * 1e-3) / 1e12
    # The arithmetic roofline's denominator: this GPU's FMA rate in the
    # kernel's precision, measured here (after the timed region) by the
    # library's FMA microbenchmark, CUDA-event timed, fastest of five.
    peak, peak_ms = hji.peak_fma(prec, target_ms=20.0)
    peak_other, _ = hji.peak_fma("f64" if prec == "f32" else "f32", target_ms=20.0)
    # DRAM bytes per stage launch (dram__bytes_read.sum + dram__bytes_write.sum)
    # from an ncu capture of the current stage kernels; none is recorded for
    # them at present (the last capture, of the kernels before the change to
    # the last stage's step bookkeeping, gave 8.1, 12.2 and 16.2 MB for the
    # three RK3 stages: the first touch of each field, everything else served
    # by L2), so `traffic` is null.
    traffic = None
    roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved_tflops / peak, "traffic": traffic,
                "kernel": "stage_kernel<%s,2,WENO5> (per-stage, 3 per RK3 step)" % prec,
                "flops_per_node_stage": FLOPS_PER_NODE_STAGE,
                "mem_words_per_node_step": WORDS_PER_NODE_STEP[prec],
                "peak_source": "measured: hji_peak_fma (%s FMA chains on every SM, "
                               "CUDA events, fastest of 5 launches of %.1f ms)" % (prec, peak_ms),
                "measured_fma_tflops": {prec: peak,
                                        ("f64" if prec == "f32" else "f32"): peak_other},
                "unit_count_fp32_tflops": 152 * 128 * 2 * 2070e6 / 1e12}

    # Each stage kernel alone between two CUDA events on this stream
    # (hji_stage_times: 300 steps from V0 = l, after the timed region): the
    # kernel durations without the gaps between graph launches and the
    # host's convergence checks that the timed-region average includes.
    st_ms = g.stage_times(l_dev, steps=300, **{k: v for k, v in SOLVE.items()
                                                if k in ("scheme", "rk", "cfl")})
    ev_ms = statistics.mean(st_ms)
    ev_tflops = flops / (ev_ms * 1e-3) / 1e12
    roofline["event_timed"] = {"stage_ms": st_ms, "achieved": ev_tflops, "frac": ev_tflops / peak,
                               "note": "mean of the three stage kernels, each timed alone "
                                       "between two CUDA events (300 steps)"}

    line = {"metric": "cell-updates/s", "value": value, "unit": "cell-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "nodes": cells, "steps_per_solve": steps_per_solve,
                       "precision": prec + " storage and stencil, FP64 dt/alpha and max|dV|",
                       "l2": "flushed (512 MB write) before every timed solve; the 1001^2 "
                             "fields stay L2-resident within a solve",
                       "parallelism": "independent instance per GPU" if world > 1 else "1 GPU",
                       "tile_shape": ["31x32", "15x64", "63x16"][tuned],
                       "autotune_ms_per_step": tune_ms},
            "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "clocks": clk}

    if rank == 0 and not args.no_variants:
        line["time_to_converge"] = time_to_converge(hji, torch, gd, dyn, l, l_dev, k_dev)
        line["hbm_workloads"] = hbm_workloads(hji, torch)
        line["serving"] = serving_both(hji, torch)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(budget_s=12.0)
    g.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def profile_stages(args, hji, torch):
    """A short march of one workload with each stage kernel launched alone
    (few launches, for a profiler): FP32, the workload's scheme and RK order."""
    if args.workload == "di1001":
        gd, dyn, l = W.di_config(N_SIDE, dmax=DMAX)
        opts = dict(scheme="weno5", rk=3, cfl=0.5)
    elif args.workload == "di8192":
        gd, dyn, l = W.di_config(8192)
        opts = dict(scheme="eno2", rk=2, cfl=0.5)
    elif args.workload == "quad61":
        gd, dyn, l = W.quad4d_config(61, dmax=0.3)
        opts = dict(scheme="eno2", rk=2, cfl=0.5)
    else:
        raise SystemExit("--profile-steps supports di1001, di8192 and quad61")
    g = hji.Grid(gd, args.precision)
    g.set_dynamics(dyn)
    npdt = np.float32 if args.precision == "f32" else np.float64
    l_dev = torch.from_numpy(l.astype(npdt)).cuda()
    ms = g.stage_times(l_dev, steps=args.profile_steps, **opts)
    g.close()
    print(json.dumps({"profile": args.workload, "precision": args.precision,
                      "steps": args.profile_steps, "stage_ms": ms}), flush=True)
    return 0


def _timed(torch, fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fn()
    torch.cuda.synchronize()
    return r, 1000.0 * (time.perf_counter() - t0)


def time_to_converge(hji, torch, gd, dyn, l, l_dev, k_dev):
    """Warm vs standard time-to-converge on the bench workload (each one
    solve, device-resident inputs): FP64 standard and warm, FP32 warm, and
    the precision pattern (FP32 warm march, then an FP64 re-validation sweep
    warm-started from it), with max-abs and BRT errors against the FP64
    standard solve."""
    out = {}
    l64, k64 = l_dev.double(), k_dev.double()
    l32, k32 = l_dev.float(), k_dev.float()
    g64 = hji.Grid(gd, "f64")
    g64.set_dynamics(dyn)
    st, ms = _timed(torch, lambda: g64.solve(l64, **SOLVE))
    ref = torch.empty_like(l64)
    g64.value(ref)
    out["f64_standard"] = {"ms": ms, "steps": st["steps"], "converged": st["converged"],
                           "intervals_0.01": st["tau"] / 0.01}
    st, ms = _timed(torch, lambda: g64.solve(l64, k64, **SOLVE))
    out["f64_warm"] = {"ms": ms, "steps": st["steps"], "converged": st["converged"],
                       "intervals_0.01": st["tau"] / 0.01}
    g32 = hji.Grid(gd, "f32")
    g32.set_dynamics(dyn)

    def pattern():
        s32 = g32.solve(l32, k32, **SOLVE)
        g64.take_value(g32)
        s64 = g64.solve(l64, init=hji.HJI_INIT_RESIDENT, **SOLVE)
        return s32, s64

    (s32, s64), ms = _timed(torch, pattern)
    v32 = torch.empty_like(l32)
    g32.value(v32)
    v64 = torch.empty_like(l64)
    g64.value(v64)
    scale = float(l64.abs().max())

    def errs(v):
        d = (v.double() - ref).abs().max().item()
        brt_diff = int(((v.double() <= 0) != (ref <= 0)).sum().item())
        return {"max_abs": d, "max_abs_over_max_l": d / scale, "brt_nodes_differing": brt_diff}

    out["f32_warm"] = dict({"steps": s32["steps"], "converged": s32["converged"]}, **errs(v32))
    _, ms32 = _timed(torch, lambda: g32.solve(l32, k32, **SOLVE))
    out["f32_warm"]["ms"] = ms32
    out["f32_warm_then_f64_revalidation"] = dict(
        {"ms": ms, "f32_steps": s32["steps"], "f64_steps": s64["steps"],
         "converged": s64["converged"]}, **errs(v64))
    out["speedup_pattern_vs_f64_standard"] = out["f64_standard"]["ms"] / ms
    g32.close()
    g64.close()
    return out


def run_hbm_workload(args, hji, torch, dist, rank, world, local_rank):
    """Main line for the HBM-bound workloads: each bench step is one 50-step
    FP32 ENO2/RK2 march (set-up, init from V0 = l, 100 stage launches)."""
    name = {"quad61": "quad4d_61^4", "batch256": "batch256_di_101..501",
            "di8192": "di_8192^2"}[args.workload]
    clocks = ClockSampler(local_rank)
    res = hbm_workloads(hji, torch, steps=50, only=name, repeats=args.steps, warmup=args.warmup,
                        clocks=clocks)[name]
    ms, upd = res["ms_total"], res["updates_total"]
    if dist is not None:
        ms, upd = reduce_over_ranks(dist, torch, ms, upd, "cuda")
    line = {"metric": "cell-updates/s", "value": upd / (ms * 1e-3), "unit": "cell-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": name + ", FP32 ENO2/RK2, cfl 0.5, 50 steps from V0 = l per "
                                          "bench step", "nodes": res["nodes"],
                       "l2": "inputs larger than L2"},
            "e2e": None, "gpu_launches": res["launches"], "roofline": res["roofline"],
            "clocks": res["clocks"]}
    if res.get("stage_kernels"):
        line["stage_kernels"] = res["stage_kernels"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def serving_both(hji, torch):
    """The specified stream (50 requests/s, far above one GPU's capacity for
    these grid sizes) and a stream below capacity (1.5 requests/s)."""
    return {"rate_50_per_s": serving(hji, torch, duration=6.0, rate=50.0, time_cap=60.0),
            "rate_1.5_per_s": serving(hji, torch, duration=20.0, rate=1.5, time_cap=60.0)}


def serving(hji, torch, duration=6.0, rate=50.0, time_cap=90.0):
    """Config-5 serving: a Poisson stream (rate 50/s, seed 7715) of mass /
    disturbance updates for quadrotor 4-D subsystems (sides 31, 41, 51, 61)
    and 2-D double integrators (sides 201..1001 in steps of 200), each
    warm-started from its system's resident previous value.  Every system is
    solved once before the clock starts (untimed), so each timed request is
    an update of a resident solution.  FP32 storage, FP64 convergence test,
    ENO2/RK2, stopping by Sec. IV's rule (max|dV| below 0.001 per 0.01 of
    time: tol_rate = 0.1)."""
    from paper_1903_07715_gb300.serve import ReachabilityServer, summarize
    quad_sides, di_sides = [31, 41, 51, 61], [201, 401, 601, 801, 1001]
    rng = np.random.Generator(np.random.PCG64(7715))
    reqs = W.poisson_requests(rate=rate, duration=duration, seed=7715)
    for r in reqs:  # the stream's sizes, quantised to the resident systems
        r["side"] = int(rng.choice(quad_sides if r["kind"] == "quad4d" else di_sides))
    opts = dict(scheme="eno2", rk=2, cfl=0.5, tol=0.0, tol_rate=0.1, max_steps=20000,
                check_every=16)
    srv = ReachabilityServer(W.serving_system, precision="f32", max_slots=64, opts=opts)
    warm = [{"t": 0.0, "kind": k, "side": s, "change": "disturbance", "value": 0.0}
            for k, sides in (("quad4d", quad_sides), ("di", di_sides)) for s in sides]
    srv.run(warm, time_cap=time_cap)
    records, wall = srv.run(reqs, time_cap=time_cap)
    srv.close()
    out = summarize(records, wall)
    out.update({"rate_per_s": rate, "stream_s": duration, "systems": len(warm),
                "mix": "50% quad4d (31..61^4), 50% double integrator (201..1001^2); mass x "
                       "U[1,1.5] or |d| ~ U[0,0.3]"})
    return out


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# each ENO2 stage kernel from an ncu capture of the current kernels, keyed by
# (workload, stage); none is recorded for them at present, so `traffic` is
# null.
DRAM_BYTES_PER_LAUNCH = {}


def _measured_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def hbm_workloads(hji, torch, steps=50, only=None, repeats=1, warmup=1, clocks=None):
    """HBM-bound marches (working sets well above the 129 MB L2), FP32
    compensated storage, ENO2/RK2: 50 steps each from V0 = l, CUDA-event
    timed after a warm-up.  Algorithmic bytes per node per RK2 step: stage 1
    reads hi, lo and writes D1 (12 B); stage 2 reads hi, lo, D1, l and writes
    hi', lo' (24 B): 36 B."""
    peak, src = _measured_hbm()
    out = {}
    bytes_per_update = 36
    cases = []
    if only in (None, "quad4d_61^4"):
        gd, dyn, l = W.quad4d_config(61, dmax=0.3)
        cases.append(("quad4d_61^4", [gd], [dyn], [l]))
    if only in (None, "batch256_di_101..501"):
        insts = W.batch_instances(count=256, seed=1903)
        cases.append(("batch256_di_101..501", [i["grid"] for i in insts],
                      [i["dyn"] for i in insts], [W.instance_target(i) for i in insts]))
    if only in (None, "di_8192^2"):
        # 2-D stress grid with the 101^2 workload's dynamics (|u| <= 1, no
        # disturbance, l = 1 - |x1|): 67 M nodes, 268 MB per FP32 field.
        gd, dyn, l = W.di_config(8192)
        cases.append(("di_8192^2", [gd], [dyn], [l]))
    opts = dict(scheme="eno2", rk=2, cfl=0.5, tol=0.0, max_steps=steps, check_every=steps)
    stream = torch.cuda.current_stream()
    for name, gds, dyns, ls in cases:
        grids = []
        for gd, dyn in zip(gds, dyns):
            g = hji.Grid(gd, "f32")
            g.set_dynamics(dyn)
            grids.append(g)
        ldev = [torch.from_numpy(l.astype(np.float32)).cuda() for l in ls]
        cells = sum(int(np.prod(gd["n"])) for gd in gds)
        med = sorted(range(len(grids)), key=lambda i: int(np.prod(gds[i]["n"])))[len(grids) // 2]
        tuned, _ = grids[med].autotune(ldev[med], steps=20, scheme="eno2", rk=2, cfl=0.5)

        def run():
            if len(grids) == 1:
                return [grids[0].solve(ldev[0], **opts)]
            return hji.batch_solve(grids, ldev, **opts)[0]

        for _ in range(max(1, warmup)):
            run()
        if clocks is not None:
            clocks.start()
        ms, upd, launches = 0.0, 0, 0
        for _ in range(repeats):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sts = run()
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            upd += sum(int(np.prod(gd["n"])) * s["steps"] for gd, s in zip(gds, sts))
            launches += max(s["kernel_launches"] for s in sts)
        clk = clocks.stop() if clocks is not None else None
        stage = None
        if len(grids) == 1:
            # Each of the two stage kernels alone between two CUDA events
            # (20 steps from V0 = l): stage 1 moves 12 B per node, the fused
            # last stage (min(l), max|dV|) 24 B.
            sms = grids[0].stage_times(ldev[0], steps=20, scheme="eno2", rk=2, cfl=0.5)
            # Two byte counts per node: what the compensated FP32 layout moves
            # (high and low words of V^n, stage increments) and the method's
            # own per-stage count with one FP32 word per field (stage 1 reads
            # V and writes W1: 8 B; the last stage reads W1, V^n, l and writes
            # V^{n+1}: 16 B).
            stage = {}
            for key, t, b, bm in (("first_stage", sms[0], 12, 8),
                                  ("fused_last_stage", sms[1], 24, 16)):
                a = b * cells / (t * 1e-3) / 1e9
                am = bm * cells / (t * 1e-3) / 1e9
                stage[key] = {"ms": t, "bytes_per_node": b, "achieved": a, "frac": a / peak,
                              "method_bytes_per_node": bm, "method_achieved": am,
                              "method_frac": am / peak,
                              "traffic": DRAM_BYTES_PER_LAUNCH.get((name, key))}
        gbs = upd * bytes_per_update / (ms * 1e-3) / 1e9
        # The method's counts per node-step: per-stage kernels of RK2 move 6
        # words (24 B in FP32); a march fused in time needs 3 (read V^n and l,
        # write V^{n+1}: 12 B).
        gbs_stage = upd * 24 / (ms * 1e-3) / 1e9
        gbs_strict = upd * 12 / (ms * 1e-3) / 1e9
        out[name] = {"nodes": cells, "steps": steps, "ms": ms / repeats, "tile_shape": ["31x32", "15x64", "63x16"][tuned],
                     "cell_updates_per_s": upd / (ms * 1e-3), "ms_total": ms,
                     "updates_total": upd, "launches": launches, "clocks": clk,
                     "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                  "frac": gbs / peak, "peak_source": src,
                                  "bytes_per_node_step": bytes_per_update, "traffic": None,
                                  "method_per_stage": {"bytes_per_node_step": 24,
                                                       "achieved": gbs_stage,
                                                       "frac": gbs_stage / peak},
                                  "method_strict": {"bytes_per_node_step": 12,
                                                    "achieved": gbs_strict,
                                                    "frac": gbs_strict / peak},
                                  "note": "whole-march time (set-up, init and 50 steps of "
                                          "2 stage launches) in the denominator"},
                     "stage_kernels": stage}
        for g in grids:
            g.close()
    return out


if __name__ == "__main__":
    sys.exit(main())
