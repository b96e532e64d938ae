"""Discounted reachability (Sec. II-C) through the C ABI against the oracle:
each step ends with V <- min(l, gamma V~), gamma = exp(-lambda dt) the
discount of one CFL step.

* FP64 one step from the oracle's own trajectory within 1e-10, 1-D to 4-D,
  every scheme;
* whole discounted marches to convergence (FP64: the oracle's step count,
  values within 1e-9; FP32 compensated: steps within 2 %, values within
  1e-4 max|l|), with one launch per stage and with the multi-step launch;
* Sec. V's schedule (0.999, then 1 once converged) as a discounted solve
  followed by an undiscounted one from the resident value;
* a batch of instances and the allocation-free entry point against solo
  hji_solve calls;
* option checks (outside [0, 1], with brs)."""
import numpy as np
import pytest

import workloads as W
from test_gpu_options import _case

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


@pytest.mark.parametrize("ndim", [1, 2, 3, 4])
@pytest.mark.parametrize("scheme,rk", [("eno1", 1), ("eno2", 2), ("weno5", 3)])
def test_discounted_one_step(orc, hji_lib, torch_cuda, ndim, scheme, rk):
    gamma = 0.97
    gd, dyn, l = _case(ndim)
    P = orc.problem(gd, dyn)
    alpha, dt = orc.alpha_dt(P, 0.5)
    V = orc.init(P, l)
    traj = [V]
    for _ in range(8):
        V, _ = orc.step(P, scheme, rk, dt, alpha, l, V, discount=gamma)
        traj.append(V)
    for n in (0, 4, 8):
        want, _ = orc.step(P, scheme, rk, dt, alpha, l, traj[n], discount=gamma)
        g = hji_lib.Grid(gd, "f64")
        g.set_dynamics(dyn)
        st = g.solve(l, traj[n], scheme=scheme, rk=rk, tol=0.0, max_steps=1, discount=gamma)
        got = g.value()
        g.close()
        assert st["steps"] == 1
        assert np.abs(got - want).max() <= TOL, (n, np.abs(got - want).max())
    # the discount acted: the undiscounted step differs
    plain, _ = orc.step(P, scheme, rk, dt, alpha, l, traj[4])
    disc, _ = orc.step(P, scheme, rk, dt, alpha, l, traj[4], discount=gamma)
    assert np.abs(plain - disc).max() > 1e-3


def _gpu_solve(hji, gd, dyn, l, prec, k=None, init=None, grid=None, **opts):
    dt = np.float64 if prec == "f64" else np.float32
    g = grid if grid is not None else hji.Grid(gd, prec)
    if grid is None:
        g.set_dynamics(dyn)
    st = g.solve(l.astype(dt), None if k is None else k.astype(dt), init=init, **opts)
    return g, st, g.value().astype(np.float64)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("march", ["per_stage", "multi_step"])
def test_discounted_march_to_convergence(orc, hji_lib, torch_cuda, prec, march):
    gd, dyn, l = W.di_config(61)
    opts = dict(scheme="eno2", rk=2, cfl=0.5, tol=1e-6, max_steps=20000, discount=0.999)
    Vo, so = orc.solve(orc.problem(gd, dyn), l, **opts)
    g, st, V = _gpu_solve(hji_lib, gd, dyn, l, prec, march=march, check_every=32, **opts)
    g.close()
    assert so["converged"] and st["converged"]
    if prec == "f64":
        assert st["steps"] == so["steps"]
        assert np.abs(V - Vo).max() <= 1e-9
    else:
        assert abs(st["steps"] - so["steps"]) <= max(3, 0.02 * so["steps"])
        assert np.abs(V - Vo).max() <= 1e-4 * np.abs(l).max()
    # far slower than the undiscounted march from the same start (Sec. V)
    _, plain = orc.solve(orc.problem(gd, dyn), l, scheme="eno2", rk=2, cfl=0.5, tol=1e-6)
    assert st["steps"] > 5 * plain["steps"]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_discount_then_anneal_schedule(orc, hji_lib, torch_cuda, prec):
    """Sec. V's comparison: march with 0.999 to convergence, then with 1 from
    the converged value (the resident value on the GPU, a warm start k in
    the oracle, where min(k, l) = k since the discounted value is <= l)."""
    gd, dyn, l = W.di_config(61)
    base = dict(scheme="eno2", rk=2, cfl=0.5, tol=1e-6, max_steps=20000)
    P = orc.problem(gd, dyn)
    Vd, sd = orc.solve(P, l, discount=0.999, **base)
    Va, sa = orc.solve(P, l, k=Vd, **base)
    g, st1, _ = _gpu_solve(hji_lib, gd, dyn, l, prec, discount=0.999, **base)
    g, st2, V = _gpu_solve(hji_lib, gd, dyn, l, prec, init=hji_lib.HJI_INIT_RESIDENT, grid=g,
                           **base)
    g.close()
    assert st1["converged"] and st2["converged"] and sa["converged"]
    if prec == "f64":
        assert (st1["steps"], st2["steps"]) == (sd["steps"], sa["steps"])
        assert np.abs(V - Va).max() <= 1e-9
    else:
        assert abs(st1["steps"] - sd["steps"]) <= max(3, 0.02 * sd["steps"])
        assert abs(st2["steps"] - sa["steps"]) <= max(3, 0.05 * sa["steps"])
        assert np.abs(V - Va).max() <= 1e-4 * np.abs(l).max()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_discounted_batch_equals_solo(hji_lib, torch_cuda, prec):
    insts = W.batch_instances(count=5, seed=9, side=(41, 90))
    dt = np.float64 if prec == "f64" else np.float32
    opts = dict(scheme="eno2", rk=2, tol=1e-6, max_steps=3000, check_every=16, discount=0.995,
                march="per_stage")
    grids, solo = [], []
    for inst in insts:
        l = W.instance_target(inst)
        g, st, V = _gpu_solve(hji_lib, inst["grid"], inst["dyn"], l, prec, **opts)
        g.close()
        solo.append((st, V))
        g = hji_lib.Grid(inst["grid"], prec)
        g.set_dynamics(inst["dyn"])
        grids.append(g)
    sts, _ = hji_lib.batch_solve(grids, [W.instance_target(i).astype(dt) for i in insts], **opts)
    for (s0, v0), s1, g in zip(solo, sts, grids):
        assert s0["steps"] == s1["steps"]
        assert np.array_equal(v0, g.value().astype(np.float64))
        g.close()


def test_discounted_noalloc_equals_solve(hji_lib, torch_cuda):
    from test_zz_no_alloc import _noalloc
    import torch
    gd, dyn, l = W.di_config(45, dmax=0.1)
    opts = dict(scheme="weno5", rk=3, tol=0.0, max_steps=40, discount=0.98, tile_variant=1,
                march="per_stage")
    for prec in ("f64", "f32"):
        dt = np.float64 if prec == "f64" else np.float32
        g, st, V = _gpu_solve(hji_lib, gd, dyn, l, prec, **opts)
        g.close()
        no = dict(opts)
        no.pop("march")
        no.pop("tile_variant")
        rc, out, nst = _noalloc(hji_lib, torch, gd, dyn, l.astype(dt), None, prec, **no)
        assert rc in (hji_lib.HJI_OK, hji_lib.HJI_E_NOT_CONVERGED)
        assert nst.steps == st["steps"]
        assert np.abs(out.astype(np.float64) - V).max() <= TOL


def test_discount_values_are_checked(hji_lib, torch_cuda):
    gd, dyn, l = W.di_config(21)
    g = hji_lib.Grid(gd, "f64")
    g.set_dynamics(dyn)
    for bad in (dict(discount=-0.1), dict(discount=1.5), dict(discount=float("nan")),
                dict(discount=0.9, brs=True)):
        with pytest.raises(hji_lib.HJIError) as e:
            g.solve(l, max_steps=3, **bad)
        assert e.value.status == hji_lib.HJI_E_INVALID
    for off in (0.0, 1.0):
        g.solve(l, max_steps=3, discount=off)
    g.close()
