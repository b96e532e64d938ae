"""Serving loop for reachability updates (continuous batching).

Each request names a system (quadrotor 4-D subsystem or 2-D double
integrator, with its grid side) and a change (mass or disturbance bound).
The server keeps one grid per system resident on the device with its last
converged value, sets the changed dynamics and submits the update to a
continuous-batching engine warm-started from that value (Sec. III: a warm
start from the previous solution is conservative, and exact when the change
only shrinks the control set or grows the disturbance, Props. 1-2 and
Sec. V-C).  Requests for a system that is still marching wait for it.  One
engine per state dimension, each on its own CUDA stream, so the 4-D and 2-D
batches overlap on the GPU.  All arithmetic runs in the CUDA library; this
module only routes requests and records latencies.
"""
import collections
import time

import numpy as np

from . import HJI_INIT_RESIDENT, HJI_INIT_STANDARD, HJI_OK, Engine, Grid


class ReachabilityServer:
    def __init__(self, systems, precision="f32", max_slots=64, budget_bytes=0, opts=None):
        """systems: callable (kind, side) -> (grid dict, base dynamics dict
        factory taking (change, value), target l numpy array)."""
        import torch
        self.torch = torch
        self.systems_fn = systems
        self.precision = precision
        self.opts = dict(scheme="eno2", rk=2, cfl=0.5, tol=1e-6, max_steps=20000, check_every=16)
        if opts:
            self.opts.update(opts)
        self.streams = {}
        self.engines = {}
        self.max_slots = max_slots
        self.budget = budget_bytes
        self.sys = {}
        self.pending = collections.defaultdict(collections.deque)
        self.busy = set()
        self.inflight = {}

    def _engine(self, ndim):
        if ndim not in self.engines:
            s = self.torch.cuda.Stream()
            self.streams[ndim] = s
            self.engines[ndim] = Engine(ndim, self.precision, max_slots=self.max_slots,
                                        budget_bytes=self.budget, stream=s.cuda_stream,
                                        **self.opts)
        return self.engines[ndim]

    def _system(self, key):
        if key not in self.sys:
            gd, dyn_fn, l = self.systems_fn(*key)
            g = Grid(gd, self.precision)
            tdt = self.torch.float32 if self.precision == "f32" else self.torch.float64
            ldev = self.torch.as_tensor(l, dtype=tdt, device="cuda").contiguous()
            self.sys[key] = {"grid": g, "l": ldev, "dyn_fn": dyn_fn, "warm": False,
                             "ndim": len(gd["n"])}
        return self.sys[key]

    def _submit(self, rid, req):
        key = (req["kind"], req["side"])
        s = self._system(key)
        s["grid"].set_dynamics(s["dyn_fn"](req["change"], req["value"]))
        init = HJI_INIT_RESIDENT if s["warm"] else HJI_INIT_STANDARD
        self.torch.cuda.current_stream().synchronize()
        self._engine(s["ndim"]).submit(s["grid"], s["l"], init=init, tag=rid)
        self.busy.add(key)
        self.inflight[rid] = key

    def run(self, requests, time_cap=None):
        """Replay `requests` (dicts with arrival time 't' in seconds) in real
        time.  Returns per-request records and the wall time."""
        t0 = time.perf_counter()
        order = sorted(range(len(requests)), key=lambda i: requests[i]["t"])
        nxt = 0
        records = {}
        done = 0
        while done < len(requests):
            now = time.perf_counter() - t0
            if time_cap is not None and now > time_cap:
                break
            while nxt < len(order) and requests[order[nxt]]["t"] <= now:
                rid = order[nxt]
                req = requests[rid]
                key = (req["kind"], req["side"])
                records[rid] = {"arrival": req["t"], "kind": req["kind"], "side": req["side"]}
                if key in self.busy:
                    self.pending[key].append(rid)
                else:
                    self._submit(rid, req)
                nxt += 1
            idle = True
            for ndim, eng in list(self.engines.items()):
                a, q = eng.step()
                idle = idle and a == 0 and q == 0
                for tag, st, rc in eng.poll():
                    t_done = time.perf_counter() - t0
                    key = self.inflight.pop(tag)
                    self.busy.discard(key)
                    s = self.sys[key]
                    s["warm"] = s["warm"] or st["steps"] > 0
                    records[tag].update({"done": t_done, "latency": t_done - records[tag]["arrival"],
                                         "steps": st["steps"], "status": rc,
                                         "converged": st["converged"],
                                         "cells": int(np.prod(s["grid"].shape))})
                    done += 1
                    if self.pending[key]:
                        nrid = self.pending[key].popleft()
                        self._submit(nrid, requests[nrid])
            if idle and nxt < len(order):
                wait = requests[order[nxt]]["t"] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.002))
        wall = time.perf_counter() - t0
        return records, wall

    def close(self):
        for e in self.engines.values():
            e.close()
        for s in self.sys.values():
            s["grid"].close()


def summarize(records, wall):
    """Latency percentiles over every arrival.  A request still queued or
    marching when the loop stopped is censored: its latency is at least
    (wall - arrival), and that lower bound enters the percentiles; a
    percentile is flagged as a lower bound when a censored request could
    move it."""
    lat_done = [r["latency"] for r in records.values() if "latency" in r]
    cens = [max(0.0, wall - r["arrival"]) for r in records.values() if "latency" not in r]
    ok = sum(1 for r in records.values() if r.get("status") == HJI_OK)
    upd = sum(r["cells"] * r["steps"] for r in records.values() if "steps" in r)
    allv = np.array(lat_done + cens)
    done = np.array(lat_done)

    srt = np.sort(allv)

    def pct(q):
        # numpy's linear interpolation between the order statistics at
        # floor(h) and ceil(h), h = (N - 1) q / 100: a censored request at or
        # below the upper one of them could still move the result.
        if not allv.size:
            return None, False
        v = float(np.percentile(allv, q))
        upper = float(srt[int(np.ceil((allv.size - 1) * q / 100.0))])
        return v * 1e3, bool(cens) and min(cens) <= upper

    p50, p50_lb = pct(50)
    p99, p99_lb = pct(99)
    return {"requests": len(records), "completed": int(done.size), "converged": ok,
            "unfinished": len(cens),
            "p50_ms": p50, "p50_is_lower_bound": p50_lb,
            "p99_ms": p99, "p99_is_lower_bound": p99_lb,
            "completed_p50_ms": float(np.percentile(done, 50) * 1e3) if done.size else None,
            "completed_p99_ms": float(np.percentile(done, 99) * 1e3) if done.size else None,
            "mean_completed_ms": float(done.mean() * 1e3) if done.size else None,
            "throughput_req_per_s": done.size / wall if wall > 0 else None,
            "cell_updates_per_s": upd / wall if wall > 0 else None, "wall_s": wall}
