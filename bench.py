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


def alu_roofline(cells, steps, stages, ms, peak_tflops, flops_per_node_stage=FLOPS_PER_NODE_STAGE):
    """Algorithmic TFLOP/s of a whole solve (cells x steps x stages x the
    per-node-stage count, over its wall time in ms) and its fraction of a
    measured FMA rate."""
    tflops = flops_per_node_stage * cells * stages * steps / (ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": tflops, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": tflops / peak_tflops, "flops_per_node_stage": flops_per_node_stage,
            "basis": "whole solve, host wall time with synchronisation"}


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
        self.rows = []
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


THROTTLE_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def clocks_rejected(clk, low_frac=0.9):
    """Why a timed region's clock record disqualifies its number, or None: a
    hardware or thermal slowdown was active, or the median SM clock sat well
    below the maximum with no reason active (a clock lock left by another
    user).  A power cap alone is kept (normal on this part under load)."""
    reasons = set(clk.get("reasons") or [])
    bad = sorted(reasons.intersection(THROTTLE_REASONS))
    if bad:
        return "throttled: " + ",".join(bad)
    sm, smax = clk.get("sm_mhz"), clk.get("sm_max_mhz")
    if sm and smax and not reasons and sm < low_frac * smax:
        return "SM clock %.0f MHz of %.0f with no reason active" % (sm, smax)
    return None


def measure_with_clock_check(timed, make_sampler, dist=None, torch=None, device="cuda"):
    """Runs the timed region `timed()` under a clock sampler; if the clocks
    disqualify it (on any rank), runs it once more.  Returns (result of the
    kept run, its clock record, the rejected attempts' records).  Every rank
    takes the same decision (one max-reduction of a flag), so the ranks'
    barriers inside `timed` stay matched."""
    rejected = []
    for attempt in range(2):
        sampler = make_sampler()
        sampler.start()
        res = timed()
        clk = sampler.stop()
        why = clocks_rejected(clk)
        again = why is not None
        if dist is not None:
            flag = torch.tensor([1.0 if again else 0.0], device=device, dtype=torch.float64)
            dist.all_reduce(flag, op=dist.ReduceOp.MAX)
            again = float(flag.item()) > 0.0
        if not again:
            return res, clk, rejected
        clk = dict(clk, rejected=why or "another rank's clocks")
        if attempt == 1:
            return res, clk, rejected
        rejected.append(clk)
    return res, clk, rejected


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
    ap.add_argument("--march", default="auto", choices=["auto", "per_stage", "multi_step"],
                    help="launch form of the timed solves (hji_solve_opts.march)")
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
    SOLVE["march"] = args.march
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
    (ms, updates, launches, stats), clk, clk_rejected = measure_with_clock_check(
        lambda: timed_solves(args.steps), lambda: ClockSampler(local_rank), dist, torch)
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
    # DRAM bytes per stage launch from the ncu capture of these kernels (mean
    # over the three RK3 stages; cold caches under ncu, so an upper bound).
    traffic = statistics.mean(DRAM_BYTES_DI1001)
    roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved_tflops / peak, "traffic": traffic,
                "kernel": "stage_kernel<%s,2,WENO5> (per-stage, 3 per RK3 step)" % prec,
                "flops_per_node_stage": FLOPS_PER_NODE_STAGE,
                "traffic_per_stage": DRAM_BYTES_DI1001,
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
                       "autotune_ms_per_step": tune_ms, "march": args.march},
            "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "clocks": clk}
    if clk_rejected:
        line["clocks_rejected_attempts"] = clk_rejected

    if rank == 0 and not args.no_variants:
        ttc = time_to_converge(hji, torch, gd, dyn, l, l_dev, k_dev)
        # the FP64 solves run at the FP64 FMA rate: their fraction of the rate measured above
        for key in ("f64_standard", "f64_warm"):
            ttc[key]["alu_roofline"] = alu_roofline(cells, ttc[key]["steps"], SOLVE["rk"],
                                                    ttc[key]["ms"],
                                                    roofline["measured_fma_tflops"]["f64"])
        line["time_to_converge"] = ttc
        line["hbm_workloads"] = hbm_workloads(hji, torch)
        line["config_rows"] = config_rows(hji, torch)
        line["batch_vs_f64_standard"] = {
            "paper_interval_test_0.001": batch_vs_f64_standard(hji, torch, 1e-3),
            "tight_interval_test_1e-4": batch_vs_f64_standard(hji, torch, 1e-4, max_steps=20000)}
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
                        clocks=clocks, march=args.march)[name]
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


def _brt_cells(torch, a, b):
    """Hausdorff distance in grid cells between the sub-zero node sets of two
    device arrays (Euclidean, by brute force over boundary-free sets: the
    symmetric difference's nodes against the other set), for the bench's
    accuracy rows.  Returns 0 when the sets agree."""
    ma, mb = (a <= 0), (b <= 0)
    if bool(torch.equal(ma, mb)):
        return 0.0
    import numpy as _np
    from scipy.ndimage import distance_transform_edt
    A, B = ma.cpu().numpy(), mb.cpu().numpy()
    if not A.any() or not B.any():
        return float("inf")
    da, db = distance_transform_edt(~A), distance_transform_edt(~B)
    return float(max(da[B].max(), db[A].max()))


def _errs(torch, v, ref, scale):
    d = float((v.double() - ref.double()).abs().max().item())
    return {"max_abs": d, "max_abs_over_max_l": d / scale,
            "brt_hausdorff_cells": _brt_cells(torch, v, ref)}


def _solve_timed(torch, g, l, k=None, init=None, **opts):
    st, ms = _timed(torch, lambda: g.solve(l, k, init=init, **opts))
    return {"ms": ms, "steps": st["steps"], "converged": st["converged"],
            "intervals_0.01": st["tau"] / 0.01, "dt": st["dt"]}


def config_rows(hji, torch):
    """Warm vs standard time-to-converge on the paper's other scenarios, one
    solve each on device-resident inputs (wall time of the C-ABI call):
      c1: 101^2 double integrator, FP64 ENO2/RK2, tol 1e-6, warm start from
          the umax = 1.2 solution (control authority shrinks: Sec. V-B,
          Table 1's control-authority rows), and discounted reachability
          from the same start (Sec. II-C; 0.999 per step, then 1 once
          converged, as Sec. V describes its comparison);
      c2: the benchmark's 1001^2 problem (FP32 WENO5/RK3, d 0 -> 0.2), under
          the per-step rule (max|dV| < 1e-6) and Sec. IV's rate rule
          (max|dV| < 0.001 per 0.01 of time), with where the last step's
          largest change sits and after how many steps the sub-zero set
          reaches its final shape;
      c3: quadrotor subsystems of Sec. VI, FP32 ENO2/RK2: 4-D at 41^4 and
          61^4 (|d| 0 -> 0.3 on v) under Sec. V's interval test (largest
          change over 0.01 of time below 0.001: ENO2 settles into a small
          limit cycle there, so no per-step tolerance near 1e-6, nor the
          per-step rate bound, is ever met), and the 2-D vertical subsystem at
          501^2 (m 1.0 -> 1.3, |d| 0 -> 0.3) under max|dV| < 1e-6 max|l|."""
    out = {}
    # ---- c1
    gd, dyn, l = W.di_config(101)
    _, dyn12, _ = W.di_config(101, umax=1.2)
    o1 = dict(scheme="eno2", rk=2, cfl=0.5, tol=1e-6, max_steps=100000)
    l64 = torch.from_numpy(l).cuda()
    g = hji.Grid(gd, "f64")
    g.set_dynamics(dyn12)
    g.solve(l64, **o1)
    k = torch.empty_like(l64)
    g.value(k)
    g.set_dynamics(dyn)
    std = _solve_timed(torch, g, l64, **o1)
    vs = torch.empty_like(l64)
    g.value(vs)
    warm = _solve_timed(torch, g, l64, k, **o1)
    vw = torch.empty_like(l64)
    g.value(vw)
    # Sec. V's third column: discounted reachability from the same start,
    # 0.999 per step until converged, then 1 from the converged value
    disc = _solve_timed(torch, g, l64, k, discount=0.999, **o1)
    vd = torch.empty_like(l64)
    g.value(vd)
    ann = _solve_timed(torch, g, l64, init=hji.HJI_INIT_RESIDENT, **o1)
    va = torch.empty_like(l64)
    g.value(va)
    g.close()
    out["c1_di101_f64_umax_1.2_to_1.0"] = {
        "standard": std, "warm": warm, "step_ratio": std["steps"] / max(1, warm["steps"]),
        "time_ratio": std["ms"] / warm["ms"], "warm_vs_standard": _errs(torch, vw, vs, 1.0),
        "discounted_0.999": disc, "then_annealed_to_1": ann,
        "discounted_total_steps": disc["steps"] + ann["steps"],
        "discounted_vs_warm_steps": (disc["steps"] + ann["steps"]) / max(1, warm["steps"]),
        "discounted_vs_standard": _errs(torch, vd, vs, 1.0),
        "annealed_vs_standard": _errs(torch, va, vs, 1.0)}
    # ---- c2
    out["c2_di1001_f32_weno5"] = c2_analysis(hji, torch)
    # ---- c3
    rate = dict(scheme="eno2", rk=2, cfl=0.5, tol=0.0, interval=0.01, interval_tol=1e-3,
                max_steps=40000, check_every=64)
    for n in (41, 61):
        gd, dyn0, l = W.quad4d_config(n, dmax=0.0)
        _, dyn3, _ = W.quad4d_config(n, dmax=0.3)
        l32 = torch.from_numpy(l.astype(np.float32)).cuda()
        g = hji.Grid(gd, "f32")
        g.set_dynamics(dyn0)
        prior = _solve_timed(torch, g, l32, **rate)
        k = torch.empty_like(l32)
        g.value(k)
        g.set_dynamics(dyn3)
        std = _solve_timed(torch, g, l32, **rate)
        vs = torch.empty_like(l32)
        g.value(vs)
        warm = _solve_timed(torch, g, l32, k, **rate)
        vw = torch.empty_like(l32)
        g.value(vw)
        g.close()
        cells = W.num_cells(gd)
        out["c3_quad4d_%d^4_f32_d_0_to_0.3" % n] = {
            "prior_d0": prior, "standard": std, "warm": warm,
            "step_ratio": std["steps"] / max(1, warm["steps"]),
            "time_ratio": std["ms"] / warm["ms"],
            "cell_updates_per_s_standard": cells * std["steps"] / (std["ms"] * 1e-3),
            "warm_vs_standard": _errs(torch, vw, vs, 4.0),
            "rule": "Sec. V: largest change of V over 0.01 of time below 0.001"}
    gd, dyn_a, l = W.quadz_config(501, mass=1.0, dmax=0.0)
    _, dyn_b, _ = W.quadz_config(501, mass=1.3, dmax=0.3)
    oz = dict(scheme="eno2", rk=2, cfl=0.5, tol=4e-6, max_steps=200000)
    l32 = torch.from_numpy(l.astype(np.float32)).cuda()
    g = hji.Grid(gd, "f32")
    g.set_dynamics(dyn_a)
    prior = _solve_timed(torch, g, l32, **oz)
    k = torch.empty_like(l32)
    g.value(k)
    g.set_dynamics(dyn_b)
    std = _solve_timed(torch, g, l32, **oz)
    vs = torch.empty_like(l32)
    g.value(vs)
    warm = _solve_timed(torch, g, l32, k, **oz)
    vw = torch.empty_like(l32)
    g.value(vw)
    g.close()
    out["c3_quadz_501^2_f32_m_1.0_to_1.3_d_0_to_0.3"] = {
        "prior": prior, "standard": std, "warm": warm,
        "step_ratio": std["steps"] / max(1, warm["steps"]), "time_ratio": std["ms"] / warm["ms"],
        "warm_vs_standard": _errs(torch, vw, vs, 4.0), "rule": "max|dV| < 1e-6 max|l| = 4e-6"}
    return out


def c2_analysis(hji, torch):
    """Why the warm start saves few steps on the benchmark problem: the
    per-step test's last steps are set by the slow drift of V far from the
    zero level set, at the grid's edges."""
    gd, dyn0, l = W.di_config(N_SIDE, dmax=0.0)
    _, dyn, _ = W.di_config(N_SIDE, dmax=DMAX)
    l32 = torch.from_numpy(l.astype(np.float32)).cuda()
    g = hji.Grid(gd, "f32")
    out = {}
    for rule_name, rule in (("per_step_1e-6", dict(tol=1e-6)),
                            ("rate_0.001_per_0.01_per_step", dict(tol=0.0, tol_rate=0.1)),
                            ("sec5_interval_change_below_0.001_over_0.01",
                             dict(tol=0.0, interval=0.01, interval_tol=1e-3))):
        o = dict(scheme="weno5", rk=3, cfl=0.5, max_steps=200000, **rule)
        g.set_dynamics(dyn0)
        g.solve(l32, **o)
        k = torch.empty_like(l32)
        g.value(k)
        g.set_dynamics(dyn)
        row = {}
        finals = {}
        for name, kk in (("standard", None), ("warm", k)):
            row[name] = _solve_timed(torch, g, l32, kk, **o)
            v = torch.empty_like(l32)
            g.value(v)
            finals[name] = v
        row["step_ratio"] = row["standard"]["steps"] / max(1, row["warm"]["steps"])
        row["warm_vs_standard"] = _errs(torch, finals["warm"], finals["standard"], 1.0)
        out[rule_name] = row
    # Where the standard solve's last changes sit: one more step from its
    # converged value (the resident value continues the march exactly).
    o = dict(scheme="weno5", rk=3, cfl=0.5, tol=1e-6, max_steps=200000)
    g.set_dynamics(dyn)
    g.solve(l32, **o)
    v0 = torch.empty_like(l32)
    g.value(v0)
    g.solve(l32, init=hji.HJI_INIT_RESIDENT, scheme="weno5", rk=3, cfl=0.5, tol=0.0, max_steps=1)
    v1 = torch.empty_like(l32)
    g.value(v1)
    dv = (v1.double() - v0.double()).abs()
    i = int(dv.argmax().item())
    r, c = divmod(i, N_SIDE)
    xs = W.node_coords(gd)
    band = v0.abs() < 0.05
    out["last_step_change"] = {
        "max_dV": float(dv.max().item()), "at_x1": float(xs[0][r]), "at_x2": float(xs[1][c]),
        "V_there": float(v0[r, c].item()),
        "cells_from_grid_edge": int(min(r, c, N_SIDE - 1 - r, N_SIDE - 1 - c)),
        "max_dV_where_|V|<0.05": float(dv[band].max().item()) if bool(band.any()) else None,
        "max_dV_beyond_10_cells_of_the_edge": float(dv[10:-10, 10:-10].max().item())}
    # After how many steps the sub-zero set takes its final shape: march in
    # chunks of 50 steps (resident continuation) and compare with the final
    # converged set.
    chunk = 50
    for name, kk in (("standard", None), ("warm", k)):
        g.set_dynamics(dyn)
        st = g.solve(l32, kk, **o)
        final = torch.empty_like(l32)
        g.value(final)
        fin = final <= 0
        total = st["steps"]
        steps = 0
        last_diff = 0
        g.solve(l32, kk, scheme="weno5", rk=3, cfl=0.5, tol=0.0, max_steps=chunk)
        while steps < total:
            steps += chunk
            v = torch.empty_like(l32)
            g.value(v)
            if not bool(torch.equal(v <= 0, fin)):
                last_diff = steps
            if steps < total:
                g.solve(l32, init=hji.HJI_INIT_RESIDENT, scheme="weno5", rk=3, cfl=0.5, tol=0.0,
                        max_steps=chunk)
        out["steps_until_final_sub_zero_set_" + name] = {
            "steps": last_diff + chunk if last_diff else chunk, "of_total": total,
            "resolution_steps": chunk}
    g.close()
    return out


def batch_vs_f64_standard(hji, torch, interval_tol, budget_s=40.0, max_steps=100000):
    """The 256-instance batch (config 4) solved as the batched FP32 warm
    form (one hji_batch_solve, each instance warm-started from its d = 0
    solution) against the plain per-instance FP64 standard solve (V0 = l,
    one hji_solve per instance, one after another) on the same GPU: time to
    converge and the FP32 results' distance to the FP64 ones.  ENO2/RK2,
    cfl 0.5, Sec. V's interval test (largest change over 0.01 of time below
    interval_tol: the paper's 0.001, or a tighter one for the accuracy bar;
    the per-step test max|dV| < 1e-6 is never met by some of these instances,
    whose ENO2 marches settle into small limit cycles).  The FP64
    solves run in instance order until
    budget_s of wall time is spent; the comparison covers those instances
    (their count is reported) and the batched time is scaled by their share
    of the batch's cell-updates."""
    insts = W.batch_instances(count=256, seed=1903)
    o = dict(scheme="eno2", rk=2, cfl=0.5, tol=0.0, interval=0.01, interval_tol=interval_tol,
             max_steps=max_steps, check_every=32)
    ls = [W.instance_target(i) for i in insts]
    l32 = [torch.from_numpy(x.astype(np.float32)).cuda() for x in ls]
    grids = []
    for inst in insts:
        grids.append(hji.Grid(inst["grid"], "f32"))
    # priors (untimed): d = 0
    for g, inst in zip(grids, insts):
        g.set_dynamics(W.double_integrator(umax=inst["umax"], dmax=0.0))
    hji.batch_solve(grids, l32, **o)
    ks = []
    for g, x in zip(grids, l32):
        k = torch.empty_like(x)
        g.value(k)
        ks.append(k)
    for g, inst in zip(grids, insts):
        g.set_dynamics(inst["dyn"])
    (sts, rc), ms_batch = _timed(torch, lambda: hji.batch_solve(grids, l32, ks, **o))
    v32 = []
    for g, x in zip(grids, l32):
        v = torch.empty_like(x)
        g.value(v)
        v32.append(v)
        g.close()
    upd_batch = [W.num_cells(i["grid"]) * s["steps"] for i, s in zip(insts, sts)]
    # per-instance FP64 standard solves
    t0 = time.perf_counter()
    done, ms64, worst_abs, worst_h, upd64, conv64, both = 0, 0.0, 0.0, 0.0, 0, 0, 0
    # the same over the instances that converged in both forms
    ms64_both, upd_b_both, worst_abs_both, worst_h_both = 0.0, 0, 0.0, 0.0
    for i, inst in enumerate(insts):
        if time.perf_counter() - t0 > budget_s:
            break
        g = hji.Grid(inst["grid"], "f64")
        g.set_dynamics(inst["dyn"])
        l64 = torch.from_numpy(ls[i]).cuda()
        st, ms = _timed(torch, lambda: g.solve(l64, **o))
        v = torch.empty_like(l64)
        g.value(v)
        g.close()
        conv64 += int(st["converged"])
        ms64 += ms
        upd64 += W.num_cells(inst["grid"]) * st["steps"]
        scale = float(l64.abs().max().item())
        e = _errs(torch, v32[i], v, scale)
        worst_abs = max(worst_abs, e["max_abs_over_max_l"])
        worst_h = max(worst_h, e["brt_hausdorff_cells"])
        if st["converged"] and sts[i]["converged"]:
            both += 1
            ms64_both += ms
            upd_b_both += upd_batch[i]
            worst_abs_both = max(worst_abs_both, e["max_abs_over_max_l"])
            worst_h_both = max(worst_h_both, e["brt_hausdorff_cells"])
        done += 1
    share = sum(upd_batch[:done]) / max(1, sum(upd_batch))
    return {"instances": len(insts), "batched_f32_warm": {
                "ms": ms_batch, "all_converged": rc == 0,
                "converged": sum(int(s["converged"]) for s in sts),
                "cell_updates": sum(upd_batch)},
            "per_instance_f64_standard": {"instances_solved": done, "converged": conv64,
                                          "ms": ms64, "cell_updates": upd64},
            "compared_instances_converged_in_both": both,
            "converged_in_both": {
                "instances": both, "f64_ms": ms64_both,
                "batched_ms_share": ms_batch * upd_b_both / max(1, sum(upd_batch)),
                "speedup": ms64_both / max(1e-9, ms_batch * upd_b_both / max(1, sum(upd_batch))),
                "worst_max_abs_over_max_l": worst_abs_both,
                "worst_brt_hausdorff_cells": worst_h_both},
            "batched_ms_for_those_instances": ms_batch * share,
            "speedup": ms64 / max(1e-9, ms_batch * share),
            "worst_max_abs_over_max_l": worst_abs, "worst_brt_hausdorff_cells": worst_h,
            "rule": "ENO2/RK2, cfl 0.5, Sec. V's interval test (change below %g over 0.01 "
                    "of time)" % interval_tol}


def serving_both(hji, torch):
    """The specified stream (50 requests/s for 60 s: far above one GPU's
    capacity for these grid sizes, so requests still queued or marching at
    the 60 s cap are counted as censored) and a stream below capacity (1.5
    requests/s for 20 s), whose requests are then compared with plain
    per-request FP64 standard solves."""
    return {"rate_50_per_s": serving(hji, torch, duration=60.0, rate=50.0, time_cap=60.0),
            "rate_1.5_per_s": serving(hji, torch, duration=20.0, rate=1.5, time_cap=60.0,
                                      compare_f64_s=30.0)}


def serving(hji, torch, duration=6.0, rate=50.0, time_cap=90.0, compare_f64_s=0.0):
    """Config-5 serving: a Poisson stream (seed 7715) of mass / disturbance
    updates for quadrotors (4-D horizontal subsystems, sides 31, 41, 51, 61)
    and 2-D double integrators (sides 201..1001 in steps of 200), each
    warm-started from its system's resident previous value.  A quadrotor
    mass update is a solve of its 2-D vertical subsystem (mass enters Eq.
    (22) only there; side 8 (s - 1) + 1 for a quadrotor of side s), a
    disturbance update a solve of a 4-D horizontal subsystem.  Every system
    is solved once before the clock starts (untimed), so each timed request
    is an update of a resident solution.  FP32 storage, FP64 convergence
    test, ENO2/RK2, stopping by Sec. V's test (largest change of V over 0.01
    of time below 0.001).  With compare_f64_s > 0, the completed
    requests are then solved one by one as plain FP64 standard solves
    (V0 = l) on the same GPU, in arrival order until that much wall time is
    spent, and each system's last served result is compared with its FP64
    counterpart."""
    from paper_1903_07715_gb300.serve import ReachabilityServer, summarize
    quad_sides, di_sides = [31, 41, 51, 61], [201, 401, 601, 801, 1001]
    rng = np.random.Generator(np.random.PCG64(7715))
    reqs = W.poisson_requests(rate=rate, duration=duration, seed=7715)
    for r in reqs:  # the stream's sizes, quantised to the resident systems
        r["side"] = int(rng.choice(quad_sides if r["kind"] == "quad4d" else di_sides))
    reqs = [W.route_request(r) for r in reqs]
    opts = dict(scheme="eno2", rk=2, cfl=0.5, tol=0.0, interval=0.01, interval_tol=1e-3,
                max_steps=20000, check_every=16)
    srv = ReachabilityServer(W.serving_system, precision="f32", max_slots=64, opts=opts)
    systems = sorted({(r["kind"], r["side"]) for r in reqs})
    warm = [{"t": 0.0, "kind": k, "side": s, "change": "disturbance", "value": 0.0}
            for k, s in systems]
    srv.run(warm, time_cap=300.0)
    records, wall = srv.run(reqs, time_cap=time_cap)
    out = summarize(records, wall)
    out.update({"rate_per_s": rate, "stream_s": duration, "time_cap_s": time_cap,
                "systems": len(systems),
                "by_kind": {k: sum(1 for r in reqs if r["kind"] == k)
                            for k in ("quad4d", "quadz", "di")},
                "mix": "50% quadrotor (disturbance: 4-D 31..61^4; mass: vertical 2-D "
                       "241..481^2), 50% double integrator (201..1001^2); mass x U[1,1.5] "
                       "or |d| ~ U[0,0.3]"})
    if compare_f64_s > 0.0:
        out["vs_f64_standard"] = _served_vs_f64(hji, torch, srv, reqs, records, opts,
                                                compare_f64_s)
    srv.close()
    return out


def _served_vs_f64(hji, torch, srv, reqs, records, opts, budget_s):
    """Completed requests of the stream re-solved as plain FP64 standard
    solves (V0 = l, same dynamics, same stopping rule) on the same GPU, in
    arrival order until budget_s of wall time is spent: the FP64 solve time
    against the served latency, and, for the last served request of each
    system (the value still resident in the server), the distance of the
    served FP32 value to the FP64 one."""
    order = sorted(records, key=lambda i: reqs[i]["t"])
    last_of = {}
    for rid in order:
        if "latency" in records[rid]:
            last_of[(reqs[rid]["kind"], reqs[rid]["side"])] = rid
    t0 = time.perf_counter()
    rows = []
    for rid in order:
        rec = records[rid]
        if "latency" not in rec:
            continue
        if time.perf_counter() - t0 > budget_s:
            break
        r = reqs[rid]
        gd, dyn_fn, l = W.serving_system(r["kind"], r["side"])
        g = hji.Grid(gd, "f64")
        g.set_dynamics(dyn_fn(r["change"], r["value"]))
        l64 = torch.from_numpy(l).cuda()
        st, ms = _timed(torch, lambda: g.solve(l64, **opts))
        row = {"kind": r["kind"], "side": r["side"], "change": r["change"],
               "f64_standard_ms": ms, "f64_steps": st["steps"],
               "served_latency_ms": rec["latency"] * 1e3, "served_steps": rec["steps"]}
        if last_of.get((r["kind"], r["side"])) == rid:
            v = torch.empty_like(l64)
            g.value(v)
            vs = torch.empty(v.shape, dtype=torch.float32, device="cuda")
            srv.sys[(r["kind"], r["side"])]["grid"].value(vs)
            row.update(_errs(torch, vs, v, float(l64.abs().max().item())))
        g.close()
        rows.append(row)
    tot64 = sum(x["f64_standard_ms"] for x in rows)
    totlat = sum(x["served_latency_ms"] for x in rows)
    checked = [x for x in rows if "max_abs" in x]
    return {"requests_compared": len(rows), "f64_standard_total_ms": tot64,
            "served_latency_total_ms": totlat,
            "f64_standard_over_served_latency": tot64 / max(1e-9, totlat),
            "value_checks": len(checked),
            "worst_max_abs_over_max_l": max((x["max_abs_over_max_l"] for x in checked),
                                            default=None),
            "worst_brt_hausdorff_cells": max((x["brt_hausdorff_cells"] for x in checked),
                                             default=None),
            "rows": rows}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# each ENO2 stage kernel, keyed by (workload, stage), from the ncu capture
# `ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,
# dram__bytes_write.sum --clock-control none python bench.py
# --profile-steps 2 --workload W` of the current stage kernels (mean of the
# two launches of each stage; summaries under profiles/).
DRAM_BYTES_PER_LAUNCH = {
    ("di_8192^2", "first_stage"): (542247168 + 237938688 + 543044864 + 238681344) / 2,
    ("di_8192^2", "fused_last_stage"): (1205116160 + 506549760 + 1207448320 + 505432320) / 2,
    ("quad4d_61^4", "first_stage"): (120999168 + 36645888 + 121103360 + 37157120) / 2,
    ("quad4d_61^4", "fused_last_stage"): (252988160 + 93743360 + 252901888 + 93992704) / 2,
}
# The multi-step march kernel on 8192^2 (one launch of 20 steps, read +
# written, from `ncu ... -k regex:march_kernel -s 2 -c 2 python bench.py
# --workload di8192 --steps 1 --warmup 1 --march multi_step`), per RK2 step.
DRAM_BYTES_MARCH_8192_PER_STEP = (34917801216 + 16077754880) / 20
# The same for the 256-grid batch (`ncu ... -k regex:march_kernel python
# bench.py --workload batch256 --steps 1 --warmup 1 --march multi_step
# --no-cpu-baseline`: two launches of 50 steps, tile shape 63x16), per RK2 step.
DRAM_BYTES_MARCH_BATCH_PER_STEP = (33359375616 + 15277051136 + 33355850752 + 15273392640) / 100
# The 1001^2 WENO5 stage kernels, one launch of each stage from the
# `ncu --set full ... -k regex:stage_kernel -c 3 python bench.py
# --profile-steps 4 --workload di1001` capture (first touch of each field per
# launch: ncu flushes the caches between launches, so these are upper bounds
# of what a launch inside a solve moves; no DRAM writes were counted).
DRAM_BYTES_DI1001 = [8110080, 12146176, 16188160]


def march_traffic(name, multi_step):
    """Captured DRAM bytes per RK2 step of a workload's march in the launch
    form it ran (None where no capture of that form exists)."""
    if multi_step:
        return {"di_8192^2": DRAM_BYTES_MARCH_8192_PER_STEP,
                "batch256_di_101..501": DRAM_BYTES_MARCH_BATCH_PER_STEP}.get(name)
    b = (DRAM_BYTES_PER_LAUNCH.get((name, "first_stage"), 0) +
         DRAM_BYTES_PER_LAUNCH.get((name, "fused_last_stage"), 0))
    return b or None


def _measured_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def hbm_workloads(hji, torch, steps=50, only=None, repeats=1, warmup=1, clocks=None,
                  march="auto"):
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
    opts = dict(scheme="eno2", rk=2, cfl=0.5, tol=0.0, max_steps=steps, check_every=steps,
                march=march)
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
        # clocks sampled during this case's timed marches (a sampler of its own
        # unless the caller passed one)
        def timed_marches():
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
            return ms, upd, launches

        make_sampler = ((lambda: clocks) if clocks is not None
                        else (lambda: ClockSampler(_env_int("LOCAL_RANK", 0))))
        (ms, upd, launches), clk, clk_rejected = measure_with_clock_check(timed_marches,
                                                                          make_sampler)
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
        # The launch form that ran: the solve's launch count less the set-up
        # launches (two per grid, three with a term table) is below the step
        # count only for the multi-step launch.
        setup = sum(2 + (1 if d.get("terms") else 0) for d in dyns)
        multi_step = launches / max(1, repeats) - setup < steps
        # The method's counts per node-step: per-stage kernels of RK2 move 6
        # words (24 B in FP32); a march fused in time needs 3 (read V^n and l,
        # write V^{n+1}: 12 B).
        gbs_stage = upd * 24 / (ms * 1e-3) / 1e9
        gbs_strict = upd * 12 / (ms * 1e-3) / 1e9
        out[name] = {"nodes": cells, "steps": steps, "ms": ms / repeats, "tile_shape": ["31x32", "15x64", "63x16"][tuned],
                     "cell_updates_per_s": upd / (ms * 1e-3), "ms_total": ms,
                     "updates_total": upd, "launches": launches, "clocks": clk,
                     "clocks_rejected_attempts": clk_rejected,
                     "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                  "frac": gbs / peak, "peak_source": src,
                                  "bytes_per_node_step": bytes_per_update,
                                  "traffic": march_traffic(name, multi_step),
                                  "traffic_unit": "DRAM bytes per RK2 step of the launch form that "
                                                  "ran (ncu)",
                                  "launch_form": "multi_step" if multi_step else "per_stage",
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
