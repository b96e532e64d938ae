"""The multi-step march launch (one cooperative kernel runs every RK stage of
check_every steps, with grid-wide barriers) against one launch per stage.
Both run the same per-node arithmetic from the same source, but the two
kernels are compiled in different inlining contexts, where the compiler may
contract a different set of multiply-adds into FMAs: results agree to
rounding (FP64 1e-10, the per-step parity bar; FP32 1e-5 max|l|) rather than
bit for bit, with the same step counts.  Covers both precisions, every scheme, RK
orders, ragged and minimal grids, periodic axes (ghost nodes read from
global memory), 3-D and 4-D grids (a multi-step launch asked for there falls
back to one launch per stage), a batch of uneven grids, and convergence
inside a launch (steps after the stop point never run)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def _both(hji, gd, dyn, l, prec, k=None, **opts):
    out = []
    for march in ("per_stage", "multi_step"):
        g = hji.Grid(gd, prec)
        g.set_dynamics(dyn)
        dt = np.float64 if prec == "f64" else np.float32
        st = g.solve(l.astype(dt), None if k is None else k.astype(dt), march=march, **opts)
        out.append((st, g.value()))
        g.close()
    (s0, v0), (s1, v1) = out
    assert s0["steps"] == s1["steps"] and s0["converged"] == s1["converged"], (s0, s1)
    assert abs(s0["tau"] - s1["tau"]) <= 1e-12 * max(1.0, s0["tau"])
    tol = 1e-10 if prec == "f64" else 1e-5 * float(np.abs(l).max())
    err = float(np.abs(v0.astype(np.float64) - v1.astype(np.float64)).max())
    assert err <= tol, err
    return s0, s1


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("scheme,rk", [("eno1", 1), ("eno2", 2), ("weno5", 3), ("eno2", 3)])
def test_2d_to_convergence(hji_lib, torch_cuda, prec, scheme, rk):
    gd, dyn, l = W.di_config(101, dmax=0.2)
    s0, s1 = _both(hji_lib, gd, dyn, l, prec, scheme=scheme, rk=rk, tol=1e-6 if scheme != "eno1"
                   else 0.0, max_steps=3000 if scheme != "eno1" else 700, check_every=32)
    # one launch per graph: far fewer kernel launches than one per stage
    assert s1["kernel_launches"] < s0["kernel_launches"]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_ragged_minimal_periodic_and_1d(hji_lib, torch_cuda, prec):
    gd, dyn, l = W.di_config(37, dmax=0.2)
    _both(hji_lib, gd, dyn, l, prec, scheme="weno5", rk=3, tol=0.0, max_steps=45, check_every=16)
    # periodic, minimal n = 2g + 1 along axis 0
    gd = W.grid([7, 48], [-np.pi, -np.pi], [np.pi, np.pi], periodic=[1, 1])
    dyn = {"terms": [(0, 1, "sin", 1.0)], "G": [[0.0], [1.0]], "ulo": [-1.0], "uhi": [1.0]}
    X1, X2 = W.mesh(gd)
    _both(hji_lib, gd, dyn, np.cos(X2) + 0.3 * X1, prec, k=np.sin(X1 + X2), scheme="weno5", rk=3,
          tol=0.0, max_steps=40, check_every=8)
    gd = W.grid([263], [-2.0], [2.0])
    dyn = {"c": [0.3], "G": [[1.0]], "ulo": [-0.5], "uhi": [1.0], "E": [[1.0]],
           "dlo": [-0.2], "dhi": [0.1], "terms": [(0, 0, "sin", 0.4)]}
    _both(hji_lib, gd, dyn, W.target_strip(gd, 0, 1.0), prec, scheme="eno2", rk=2, tol=1e-7,
          max_steps=5000)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_3d_and_4d_forced_multi_step(hji_lib, torch_cuda, prec):
    rng = np.random.Generator(np.random.PCG64(3))
    gd = W.grid([13, 19, 35], [-1.0, -2.0, -1.5], [1.0, 2.0, 1.5], periodic=[1, 0, 0])
    dyn = {"A": rng.normal(size=(3, 3)) * 0.5, "c": [0.1, -0.2, 0.3],
           "G": [[1.0, 0.0], [0.0, 1.0], [0.5, -0.5]], "ulo": [-1, -0.5], "uhi": [1, 0.7],
           "E": [[0.2], [0.0], [0.3]], "dlo": [-0.3], "dhi": [0.3],
           "terms": [(2, 0, "cos", 0.7), (0, 1, "tan", 0.2)]}
    X = W.mesh(gd)
    l = np.sqrt(X[0] ** 2 + X[1] ** 2 + X[2] ** 2) - 0.8
    _both(hji_lib, gd, dyn, l, prec, scheme="weno5", rk=3, tol=0.0, max_steps=20, check_every=8)
    gd, dyn, l = W.quad4d_config(17, dmax=0.3)
    _both(hji_lib, gd, dyn, l, prec, scheme="eno2", rk=2, tol=0.0, max_steps=25, check_every=8)


def test_forced_modes_agree_on_4d_auto(hji_lib, torch_cuda):
    """AUTO keeps one launch per stage for 4-D grids."""
    gd, dyn, l = W.quad4d_config(13)
    g = hji_lib.Grid(gd, "f32")
    g.set_dynamics(dyn)
    st = g.solve(l.astype(np.float32), scheme="eno2", rk=2, tol=0.0, max_steps=16, check_every=8)
    g.close()
    assert st["kernel_launches"] >= 16 * 2


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batch_of_uneven_grids(hji_lib, torch_cuda, prec):
    insts = W.batch_instances(count=9, seed=5, side=(41, 140))
    dt = np.float64 if prec == "f64" else np.float32
    res = []
    for march in ("per_stage", "multi_step"):
        grids = []
        for inst in insts:
            g = hji_lib.Grid(inst["grid"], prec)
            g.set_dynamics(inst["dyn"])
            grids.append(g)
        ls = [W.instance_target(i).astype(dt) for i in insts]
        sts, rc = hji_lib.batch_solve(grids, ls, scheme="eno2", rk=2, tol=1e-6, max_steps=4000,
                                      check_every=16, march=march)
        res.append((sts, [g.value() for g in grids]))
        for g in grids:
            g.close()
    (a, va), (b, vb) = res
    tol = 1e-10 if prec == "f64" else 1e-5 * 3.0
    for sa, sb, x, y in zip(a, b, va, vb):
        assert sa["steps"] == sb["steps"] and sa["converged"] == sb["converged"]
        assert np.abs(x.astype(np.float64) - y.astype(np.float64)).max() <= tol
    # instances stop on their own tests at different steps
    assert len({s["steps"] for s in a}) > 1


def test_invalid_march_mode_is_rejected(hji_lib, torch_cuda):
    gd, dyn, l = W.di_config(21)
    g = hji_lib.Grid(gd, "f64")
    g.set_dynamics(dyn)
    with pytest.raises(hji_lib.HJIError) as e:
        g.solve(l, march=5, max_steps=3)
    assert e.value.status == hji_lib.HJI_E_INVALID
    g.close()
