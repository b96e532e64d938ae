"""bench.py's host helpers on CPU: which clock records disqualify a timed
region, the single retake (all ranks together under a multi-rank launch), and
the arithmetic of the whole-solve FMA-rate fraction."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _clk(sm, smax, reasons):
    return {"sm_mhz": sm, "sm_max_mhz": smax, "reasons": list(reasons), "samples": 10}


def test_clock_records_that_disqualify():
    assert bench.clocks_rejected(_clk(2070, 2070, [])) is None
    assert bench.clocks_rejected(_clk(1900, 2070, ["sw_power_cap"])) is None
    assert bench.clocks_rejected(_clk(1500, 2070, ["sw_power_cap"])) is None
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        why = bench.clocks_rejected(_clk(2070, 2070, [r, "sw_power_cap"]))
        assert why is not None and r in why
    # stuck well below the maximum with nothing active: a leftover clock lock
    assert "no reason" in bench.clocks_rejected(_clk(1200, 2070, []))
    assert bench.clocks_rejected(_clk(1950, 2070, [])) is None
    # no nvidia-smi: nothing to judge
    assert bench.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None,
                                  "reasons": ["nvidia-smi unavailable"]}) is None


class _FakeSampler:
    def __init__(self, records):
        self.records = records

    def start(self):
        pass

    def stop(self):
        return self.records.pop(0)


def _measure(records, dist=None, torch=None):
    calls = []
    samplers = []

    def make():
        samplers.append(_FakeSampler(records))
        return samplers[-1]

    def timed():
        calls.append(len(calls))
        return "run%d" % len(calls)

    res, clk, rejected = bench.measure_with_clock_check(timed, make, dist, torch, "cpu")
    return res, clk, rejected, len(calls)


def test_clean_run_is_kept():
    res, clk, rejected, n = _measure([_clk(2070, 2070, [])])
    assert (res, n, rejected) == ("run1", 1, []) and "rejected" not in clk


def test_throttled_run_is_retaken_once():
    res, clk, rejected, n = _measure([_clk(2070, 2070, ["hw_slowdown"]), _clk(2070, 2070, [])])
    assert (res, n) == ("run2", 2)
    assert len(rejected) == 1 and "hw_slowdown" in rejected[0]["rejected"]
    assert "rejected" not in clk


def test_second_bad_run_is_kept_and_marked():
    res, clk, rejected, n = _measure([_clk(1000, 2070, []), _clk(1000, 2070, [])])
    assert (res, n) == ("run2", 2)
    assert len(rejected) == 1 and "no reason" in clk["rejected"]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench as b
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    # only rank 1 sees a throttled first run: both ranks must retake together
    recs = [_clk(2070, 2070, ["sw_thermal_slowdown"] if rank == 1 else []), _clk(2070, 2070, [])]
    runs = []

    def timed():
        dist.barrier()   # the real timed region has a barrier per solve
        runs.append(1)
        return len(runs)

    res, clk, rejected = b.measure_with_clock_check(timed, lambda: _FakeSampler(recs), dist,
                                                    torch, "cpu")
    out[rank] = (res, len(rejected), rejected[0]["rejected"] if rejected else "")
    dist.destroy_process_group()


def test_ranks_retake_together_over_gloo():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0][:2] == (2, 1) and out[1][:2] == (2, 1)
    assert "another rank" in out[0][2] and "sw_thermal_slowdown" in out[1][2]


def test_alu_roofline_arithmetic():
    """370 flops per node-stage, 1001^2 nodes, RK3, 4006 steps in 5.4 s: the
    product over the time, and its fraction of a 1.056 TFLOP/s rate."""
    r = bench.alu_roofline(1002001, 4006, 3, 5400.0, 1.056)
    want = 370 * 1002001 * 3 * 4006 / 5.4 / 1e12
    assert r["achieved"] == want or abs(r["achieved"] - want) < 1e-12 * want
    assert abs(r["frac"] - want / 1.056) < 1e-12 and r["unit"] == "TFLOP/s"
    assert bench.FLOPS_PER_NODE_STAGE == 370
