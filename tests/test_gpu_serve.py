"""Continuous batching (hji_engine_*): requests admitted while others march,
slots refilled as requests finish, HBM-budget admission, resident warm
starts.  Each request's result must equal a solo hji_solve of the same
request bit for bit, whatever else shares its launches."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

# Engines launch one kernel per RK stage; the solo reference solves use the
# same launch form, so the arithmetic (and with it every bit) is the same.
OPTS = dict(scheme="weno5", rk=3, cfl=0.5, tol=1e-6, max_steps=6000, check_every=8)


def _grids(hji, insts, prec="f32"):
    out = []
    for inst in insts:
        g = hji.Grid(inst["grid"], prec)
        g.set_dynamics(inst["dyn"])
        out.append(g)
    return out


def test_alone_equals_in_mix(hji_lib):
    import torch
    assert torch.cuda.is_available()
    hji = hji_lib
    insts = W.batch_instances(count=7, seed=21, side=(31, 121))
    ls = [W.instance_target(i).astype(np.float32) for i in insts]
    solo = []
    for inst, l in zip(insts, ls):
        g = hji.Grid(inst["grid"], "f32")
        g.set_dynamics(inst["dyn"])
        st = g.solve(l, march="per_stage", **OPTS)
        solo.append((g.value(), st))
        g.close()
    grids = _grids(hji, insts)
    eng = hji.Engine(2, "f32", max_slots=3, **OPTS)
    done = {}
    for i in range(3):
        eng.submit(grids[i], ls[i], tag=i)
    for _ in range(4):  # the first three march for a while
        eng.step()
        done.update({t: (st, rc) for t, st, rc in eng.poll()})
    for i in range(3, 7):  # the rest arrive mid-march and wait for slots
        eng.submit(grids[i], ls[i], tag=i)
    max_active = 0
    while True:
        a, q = eng.step()
        max_active = max(max_active, a)
        done.update({t: (st, rc) for t, st, rc in eng.poll()})
        if a == 0 and q == 0:
            break
    assert max_active <= 3
    assert sorted(done) == list(range(7))
    for i, g in enumerate(grids):
        st, rc = done[i]
        assert rc == (hji.HJI_OK if solo[i][1]["converged"] else hji.HJI_E_NOT_CONVERGED)
        assert st["steps"] == solo[i][1]["steps"]
        assert np.array_equal(g.value(), solo[i][0])
        g.close()
    eng.close()


def test_budget_admission_and_resident_warm_start(hji_lib):
    import torch
    assert torch.cuda.is_available()
    hji = hji_lib
    insts = W.batch_instances(count=4, seed=5, side=(41, 41))
    grids = _grids(hji, insts, "f64")
    ls = [W.instance_target(i) for i in insts]
    # V x2, l, W1, W2 (rows padded to a multiple of 8 nodes: 41 -> 48) + term table
    per_grid = 41 * 48 * 8 * 5 + 8 * 41 * 8
    eng = hji.Engine(2, "f64", max_slots=8, budget_bytes=2 * per_grid + 100, **OPTS)
    for i, (g, l) in enumerate(zip(grids, ls)):
        eng.submit(g, l, tag=i)
    max_active = 0
    done = []
    while True:
        a, q = eng.step()
        max_active = max(max_active, a)
        done += eng.poll()
        if a == 0 and q == 0:
            break
    assert max_active == 2 and len(done) == 4
    # Resident warm start through the engine equals the solo resident flow.
    new_dyn = W.double_integrator(umax=insts[0]["umax"] * 0.8, dmax=insts[0]["dmax"])
    ref = hji.Grid(insts[0]["grid"], "f64")
    ref.set_dynamics(insts[0]["dyn"])
    ref.solve(ls[0], march="per_stage", **OPTS)
    ref.set_dynamics(new_dyn)
    st_ref = ref.solve(ls[0], init=hji.HJI_INIT_RESIDENT, march="per_stage", **OPTS)
    grids[0].set_dynamics(new_dyn)
    eng.submit(grids[0], ls[0], init=hji.HJI_INIT_RESIDENT, tag=99)
    out = eng.drain()
    assert out[0][0] == 99 and out[0][1]["steps"] == st_ref["steps"]
    assert np.array_equal(grids[0].value(), ref.value())
    ref.close()
    for g in grids:
        g.close()
    eng.close()


def test_engine_reports_bad_input_and_goes_on(hji_lib):
    import torch
    assert torch.cuda.is_available()
    hji = hji_lib
    insts = W.batch_instances(count=2, seed=9, side=(31, 41))
    grids = _grids(hji, insts)
    bad = W.instance_target(insts[0]).astype(np.float32)
    bad[2, 3] = np.nan
    eng = hji.Engine(2, "f32", max_slots=4, **OPTS)
    eng.submit(grids[0], bad, tag=1)
    eng.submit(grids[1], W.instance_target(insts[1]).astype(np.float32), tag=2)
    res = {t: rc for t, st, rc in eng.drain()}
    assert res[1] == hji.HJI_E_INVALID and res[2] == hji.HJI_OK
    g64 = hji.Grid(insts[1]["grid"], "f64")
    g64.set_dynamics(insts[1]["dyn"])
    with pytest.raises(hji.HJIError) as e:
        eng.submit(g64, W.instance_target(insts[1]), tag=3)
    assert e.value.status == hji.HJI_E_INVALID
    g64.close()
    for g in grids:
        g.close()
    eng.close()


def test_server_replays_a_poisson_stream(hji_lib):
    """The request loop: small Poisson stream over a few resident systems of
    both dimensionalities; every request completes, later requests of a
    system warm-start from its previous value, and latencies are recorded."""
    import torch
    assert torch.cuda.is_available()
    from paper_1903_07715_gb300.serve import ReachabilityServer, summarize
    reqs = W.poisson_requests(rate=40.0, duration=0.5, seed=3, quad_side=(11, 13),
                              di_side=(41, 45))
    assert len(reqs) >= 8
    srv = ReachabilityServer(W.serving_system, precision="f32", max_slots=8,
                             opts=dict(tol=1e-5, max_steps=4000))
    records, wall = srv.run(reqs, time_cap=120.0)
    srv.close()
    s = summarize(records, wall)
    assert s["completed"] == len(reqs)
    assert all(r["status"] in (hji_lib.HJI_OK, hji_lib.HJI_E_NOT_CONVERGED) for r in records.values())
    assert s["p99_ms"] >= s["p50_ms"] > 0
