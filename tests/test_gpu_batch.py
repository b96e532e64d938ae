"""Batched marches: many uneven grids in one persistent launch per RK stage.

Each node's update does not depend on which tile list it came from, and the
max reductions are order independent, so every grid of a batch must reach
exactly (bit for bit) the value and step count it reaches alone; the FP64
batch also matches the oracle.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _instances(count, seed, side=(31, 97)):
    return W.batch_instances(count=count, seed=seed, side=side)


@pytest.mark.parametrize("prec,scheme,rk", [("f64", "eno2", 2), ("f32", "weno5", 3),
                                            ("f32", "eno2", 2)])
def test_batch_equals_alone(hji_lib, prec, scheme, rk):
    import torch
    assert torch.cuda.is_available()
    insts = _instances(9, seed=3)
    npdt = np.float64 if prec == "f64" else np.float32
    opts = dict(scheme=scheme, rk=rk, cfl=0.5, tol=1e-6, max_steps=40000, check_every=16)
    ls = [W.instance_target(i).astype(npdt) for i in insts]
    grids = []
    for inst in insts:
        g = hji_lib.Grid(inst["grid"], prec)
        g.set_dynamics(inst["dyn"])
        grids.append(g)
    stats, rc = hji_lib.batch_solve(grids, ls, **opts)
    batched = [g.value() for g in grids]
    for g, l, st, Vb in zip(grids, ls, stats, batched):
        alone = g.solve(l, **opts)
        Va = g.value()
        assert alone["steps"] == st["steps"]
        assert np.array_equal(Va, Vb)
    for g in grids:
        g.close()


def test_batch_warm_start_and_oracle(orc, hji_lib):
    import torch
    assert torch.cuda.is_available()
    insts = _instances(5, seed=11, side=(41, 71))
    opts = dict(scheme="eno2", rk=2, cfl=0.5, tol=1e-6, max_steps=40000)
    grids, ls, ks = [], [], []
    for inst in insts:
        g = hji_lib.Grid(inst["grid"], "f64")
        g.set_dynamics(inst["dyn"])
        grids.append(g)
        l = W.instance_target(inst)
        ls.append(l)
        ks.append(np.minimum(l, W.warm_circles(inst["grid"], 5)))
    stats, rc = hji_lib.batch_solve(grids, ls, ks, **opts)
    for inst, g, l, k, st in zip(insts, grids, ls, ks, stats):
        Vo, so = orc.solve(orc.problem(inst["grid"], inst["dyn"]), l, k, **opts)
        assert st["steps"] == so["steps"]
        assert np.abs(g.value() - Vo).max() <= 1e-9
        g.close()


def test_batch_rejects_mixed_precision(hji_lib):
    insts = _instances(2, seed=5)
    g1 = hji_lib.Grid(insts[0]["grid"], "f64")
    g2 = hji_lib.Grid(insts[1]["grid"], "f32")
    for g, inst in ((g1, insts[0]), (g2, insts[1])):
        g.set_dynamics(inst["dyn"])
    with pytest.raises(hji_lib.HJIError) as e:
        hji_lib.batch_solve([g1, g2], [W.instance_target(insts[0]),
                                       W.instance_target(insts[1]).astype(np.float32)])
    assert e.value.status == hji_lib.HJI_E_INVALID
    g1.close()
    g2.close()


@pytest.mark.parametrize("prec,scheme,rk", [("f32", "weno5", 3), ("f64", "eno2", 2)])
def test_tile_shapes_give_identical_results_and_autotune(hji_lib, prec, scheme, rk):
    """Every tile shape computes the same per-node arithmetic, so forcing each
    shape gives bit-identical marches; the autotuner times them and its
    choice is then used by default."""
    import torch
    assert torch.cuda.is_available()
    gd, dyn, l = W.di_config(203, dmax=0.1)
    l = l.astype(np.float32 if prec == "f32" else np.float64)
    opts = dict(scheme=scheme, rk=rk, cfl=0.5, tol=1e-6, max_steps=3000)
    g = hji_lib.Grid(gd, prec)
    g.set_dynamics(dyn)
    vals, steps = [], []
    for v in range(1, hji_lib.HJI_TILE_VARIANTS + 1):
        st = g.solve(l, tile_variant=v, **opts)
        vals.append(g.value())
        steps.append(st["steps"])
    assert len(set(steps)) == 1
    for V in vals[1:]:
        assert np.array_equal(V, vals[0])
    chosen, ms = g.autotune(l, steps=10, **opts)
    assert 0 <= chosen < hji_lib.HJI_TILE_VARIANTS and all(m > 0 for m in ms)
    st = g.solve(l, **opts)
    assert st["steps"] == steps[0] and np.array_equal(g.value(), vals[0])
    g.close()


def test_f32_last_stage_has_no_read_write_overlap(hji_lib):
    """On a grid with several waves of tiles per stage (1001^2: about 1000
    tiles for about 600 resident CTAs), a tile's last stage must not see the low
    words its neighbours already wrote for V^{n+1}: the march is then
    independent of the order in which tiles run, so every tile shape gives
    the same bits."""
    import torch
    assert torch.cuda.is_available()
    gd, dyn, l = W.di_config(1001, dmax=0.2)
    l = l.astype(np.float32)
    g = hji_lib.Grid(gd, "f32")
    g.set_dynamics(dyn)
    vals = []
    for v in range(1, hji_lib.HJI_TILE_VARIANTS + 1):
        st = g.solve(l, scheme="weno5", rk=3, cfl=0.5, tol=0.0, max_steps=60, tile_variant=v)
        assert st["steps"] == 60
        vals.append(g.value())
    for V in vals[1:]:
        assert np.array_equal(V, vals[0])
    g.close()
