"""Host logic of the serving loop (paper_1903_07715_gb300/serve.py) on the CPU:
the request routing is driven against a fake engine and fake grids, so no
device work happens.  Checked: every request completes; a system's requests
never overlap (a request for a busy system waits for it); the first request
of a system starts from V0 = l and later ones from its resident value
(Sec. III); 2-D and 4-D systems go to separate engines; the summary's
percentiles; the time cap."""
import collections
import types

import numpy as np

import paper_1903_07715_gb300 as hji
from paper_1903_07715_gb300 import serve


class FakeGrid:
    def __init__(self, gd, precision="f32"):
        self.shape = tuple(int(v) for v in gd["n"])
        self.dyn = None

    def set_dynamics(self, dyn):
        self.dyn = dyn

    def close(self):
        pass


class FakeEngine:
    """Admits up to max_slots requests; a cold request needs 3 engine steps,
    a resident warm start 1."""
    made = []

    def __init__(self, ndim, precision, max_slots=64, budget_bytes=0, stream=None, **opts):
        self.ndim = ndim
        self.max_slots = max_slots
        self.queue = collections.deque()
        self.active = {}
        self.finished = []
        self.log = []  # (tag, init, id of the grid)
        FakeEngine.made.append(self)

    def submit(self, grid, l, init=hji.HJI_INIT_STANDARD, tag=0):
        for g, _, _ in self.active.values():
            assert g is not grid, "a system was submitted while it was still marching"
        for _, g, _ in self.queue:
            assert g is not grid, "a system was queued twice"
        self.log.append((tag, init, id(grid)))
        self.queue.append((tag, grid, init))

    def step(self):
        while self.queue and len(self.active) < self.max_slots:
            tag, grid, init = self.queue.popleft()
            self.active[tag] = (grid, init, [0])
        done = []
        for tag, (grid, init, n) in self.active.items():
            n[0] += 1
            if n[0] >= (1 if init == hji.HJI_INIT_RESIDENT else 3):
                done.append(tag)
        for tag in done:
            _, _, n = self.active.pop(tag)
            self.finished.append((tag, {"steps": n[0], "converged": True}, hji.HJI_OK))
        return len(self.active), len(self.queue)

    def poll(self):
        out, self.finished = self.finished, []
        return out

    def close(self):
        pass


def _fake_torch():
    class Stream:
        cuda_stream = None

    cuda = types.SimpleNamespace(Stream=Stream,
                                 current_stream=lambda: types.SimpleNamespace(synchronize=lambda: None))
    return types.SimpleNamespace(float32="f32", float64="f64", cuda=cuda,
                                 as_tensor=lambda a, dtype=None, device=None:
                                 types.SimpleNamespace(contiguous=lambda: a))


def _systems(kind, side):
    nd = 4 if kind == "quad4d" else 2
    gd = {"n": [side] * nd, "lo": [-1.0] * nd, "hi": [1.0] * nd}
    return gd, (lambda change, value: {"change": change, "value": value}), np.zeros([side] * nd)


def _server(monkeypatch, max_slots=2):
    monkeypatch.setattr(serve, "Engine", FakeEngine)
    monkeypatch.setattr(serve, "Grid", FakeGrid)
    FakeEngine.made = []
    srv = serve.ReachabilityServer(_systems, precision="f32", max_slots=max_slots)
    srv.torch = _fake_torch()
    return srv


def _requests():
    spec = [(0.000, "di", 41), (0.001, "di", 41), (0.002, "quad4d", 11), (0.003, "di", 41),
            (0.004, "di", 51), (0.005, "quad4d", 11), (0.006, "di", 61), (0.007, "di", 71)]
    return [{"t": t, "kind": k, "side": s, "change": "disturbance", "value": 0.1 * i}
            for i, (t, k, s) in enumerate(spec)]


def test_every_request_completes_and_systems_never_overlap(monkeypatch):
    srv = _server(monkeypatch)
    reqs = _requests()
    records, wall = srv.run(reqs, time_cap=30.0)
    srv.close()
    assert sorted(records) == list(range(len(reqs)))
    assert all("latency" in r and r["latency"] >= 0.0 for r in records.values())
    # One engine per state dimension.
    assert sorted(e.ndim for e in FakeEngine.made) == [2, 4]
    # Each system: first submission from V0 = l, later ones from the resident
    # value, in arrival order.
    by_sys = collections.defaultdict(list)
    for e in FakeEngine.made:
        for tag, init, _ in e.log:
            by_sys[(reqs[tag]["kind"], reqs[tag]["side"])].append((tag, init))
    for key, subs in by_sys.items():
        tags = [t for t, _ in subs]
        assert tags == sorted(tags), key
        assert [i for _, i in subs] == [hji.HJI_INIT_STANDARD] + [hji.HJI_INIT_RESIDENT] * (len(subs) - 1)
    assert len(by_sys[("di", 41)]) == 3 and len(by_sys[("quad4d", 11)]) == 2
    # Cold starts take the fake engine's three steps, resident warm starts one.
    assert records[7]["steps"] == 3 and records[3]["steps"] == 1
    # Each system's grid carries the dynamics of its last request.
    last = {}
    for r in reqs:
        last[(r["kind"], r["side"])] = r["value"]
    for key, s in srv.sys.items():
        assert s["grid"].dyn == {"change": "disturbance", "value": last[key]}
    s = serve.summarize(records, wall)
    assert s["requests"] == s["completed"] == s["converged"] == len(reqs)
    assert s["p99_ms"] >= s["p50_ms"] >= 0.0
    assert s["cell_updates_per_s"] > 0


def test_time_cap_stops_the_loop(monkeypatch):
    srv = _server(monkeypatch)
    reqs = [dict(r, t=r["t"] + 5.0) for r in _requests()]  # nothing arrives before the cap
    records, wall = srv.run(reqs, time_cap=0.05)
    srv.close()
    assert records == {} and wall < 5.0
    s = serve.summarize(records, wall)
    assert s["completed"] == 0 and s["p50_ms"] is None


def test_summary_counts_unfinished_requests_as_censored():
    """Percentiles are taken over every arrival: a request still running at
    the cap enters with the lower bound (wall - arrival) and flags the
    percentiles it can move."""
    recs = {0: {"arrival": 0.0, "latency": 0.1, "steps": 1, "status": hji.HJI_OK, "cells": 10},
            1: {"arrival": 0.0, "latency": 0.2, "steps": 1, "status": hji.HJI_OK, "cells": 10},
            2: {"arrival": 1.0},   # unfinished at wall = 5 s: latency >= 4 s
            3: {"arrival": 4.5}}   # unfinished: latency >= 0.5 s
    s = serve.summarize(recs, 5.0)
    assert s["requests"] == 4 and s["completed"] == 2 and s["unfinished"] == 2
    assert s["p99_ms"] >= 3800.0 and s["p99_is_lower_bound"]
    assert abs(s["p50_ms"] - 350.0) < 1e-6 and s["p50_is_lower_bound"]
    assert abs(s["completed_p50_ms"] - 150.0) < 1e-6
    done_only = serve.summarize({k: recs[k] for k in (0, 1)}, 5.0)
    assert not done_only["p99_is_lower_bound"] and done_only["unfinished"] == 0


def test_quadrotor_mass_updates_go_to_the_vertical_subsystem():
    import workloads as W
    r = W.route_request({"t": 0.1, "kind": "quad4d", "side": 41, "change": "mass", "value": 1.2})
    assert r["kind"] == "quadz" and r["side"] == 321 and r["value"] == 1.2
    d = {"t": 0.1, "kind": "quad4d", "side": 41, "change": "disturbance", "value": 0.2}
    assert W.route_request(d) == d
    gd, dyn_fn, l = W.serving_system("quadz", 321)
    assert gd["n"] == [321, 321]
    assert abs(dyn_fn("mass", 1.25)["G"][1][0] - W.QUAD_KT / 1.25) < 1e-15
    assert dyn_fn("disturbance", 0.2)["dhi"] == [0.2]
