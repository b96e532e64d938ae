"""The march's options against the oracle through the C ABI:

* brs: the HJI PDE of Eq. (5) alone (no projection onto V <= l): the value
  of the backward reachable set at time tau;
* local_lf: Lax-Friedrichs dissipation with each node's own coefficients
  alpha_a(x) = max_{u,d} |f_a(x,u,d)|.

FP64 one step from the oracle's own trajectory within 1e-10, whole marches
with the oracle's step count, FP32 within 1e-4 max|l|."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def _case(ndim):
    rng = np.random.Generator(np.random.PCG64(40 + ndim))
    if ndim == 1:
        gd = W.grid([263], [-2.0], [2.0])
        dyn = {"c": [0.3], "A": [[0.4]], "G": [[1.0]], "ulo": [-0.5], "uhi": [1.0], "E": [[1.0]],
               "dlo": [-0.2], "dhi": [0.1], "terms": [(0, 0, "sin", 0.4)]}
        l = W.target_strip(gd, 0, 1.0)
    elif ndim == 2:
        gd, dyn, l = W.di_config(61, dmax=0.2)
        gd = W.grid([61, 70], [-2.0, -2.0], [2.0, 2.0])
        l = W.target_strip(gd, 0, 1.0)
    elif ndim == 3:
        gd = W.grid([13, 19, 35], [-1.0, -2.0, -1.5], [1.0, 2.0, 1.5])
        dyn = {"A": rng.normal(size=(3, 3)) * 0.5, "c": [0.1, -0.2, 0.3],
               "G": [[1.0, 0.0], [0.0, 1.0], [0.5, -0.5]], "ulo": [-1, -0.5], "uhi": [1, 0.7],
               "E": [[0.2], [0.0], [0.3]], "dlo": [-0.3], "dhi": [0.3],
               "terms": [(2, 0, "cos", 0.7), (0, 1, "tan", 0.2)]}
        X = W.mesh(gd)
        l = np.sqrt(X[0] ** 2 + X[1] ** 2 + X[2] ** 2) - 0.8
    else:
        gd, dyn, l = W.quad4d_config(15, dmax=0.3)
    return gd, dyn, l


def _one_step(orc, hji, gd, dyn, l, scheme, rk, steps, **flags):
    P = orc.problem(gd, dyn)
    alpha, dt = orc.alpha_dt(P, 0.5)
    V = orc.init(P, l)
    traj = [V]
    for _ in range(steps):
        V, _ = orc.step(P, scheme, rk, dt, alpha, l, V, **flags)
        traj.append(V)
    for n in (0, steps // 2, steps):
        want, _ = orc.step(P, scheme, rk, dt, alpha, l, traj[n], **flags)
        g = hji.Grid(gd, "f64")
        g.set_dynamics(dyn)
        st = g.solve(l, traj[n], scheme=scheme, rk=rk, tol=0.0, max_steps=1, **flags)
        got = g.value()
        g.close()
        assert st["steps"] == 1
        assert np.abs(got - want).max() <= TOL, (n, np.abs(got - want).max())
    return traj


@pytest.mark.parametrize("ndim", [1, 2, 3, 4])
@pytest.mark.parametrize("scheme,rk", [("eno2", 2), ("weno5", 3), ("eno1", 1)])
def test_local_lf_one_step(orc, hji_lib, torch_cuda, ndim, scheme, rk):
    gd, dyn, l = _case(ndim)
    _one_step(orc, hji_lib, gd, dyn, l, scheme, rk, 8, local_lf=True)


@pytest.mark.parametrize("ndim", [1, 2, 3])
@pytest.mark.parametrize("scheme,rk", [("eno2", 2), ("weno5", 3)])
def test_brs_one_step(orc, hji_lib, torch_cuda, ndim, scheme, rk):
    gd, dyn, l = _case(ndim)
    traj = _one_step(orc, hji_lib, gd, dyn, l, scheme, rk, 10, brs=True)
    assert (traj[-1] > l + 1e-6).any()  # the unprojected march rises above l somewhere


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_brs_march_to_a_horizon(orc, hji_lib, torch_cuda, prec):
    gd, dyn, l = W.di_config(101, dmax=0.1)
    opts = dict(scheme="eno2", rk=2, cfl=0.5, tol=0.0, horizon=0.8, brs=True)
    Vo, so = orc.solve(orc.problem(gd, dyn), l, **opts)
    g = hji_lib.Grid(gd, prec)
    g.set_dynamics(dyn)
    st = g.solve(l.astype(np.float64 if prec == "f64" else np.float32), **opts)
    V = g.value().astype(np.float64)
    g.close()
    assert st["steps"] == so["steps"]
    assert np.abs(V - Vo).max() <= (1e-9 if prec == "f64" else 1e-4 * np.abs(l).max())


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_local_lf_march_to_convergence(orc, hji_lib, torch_cuda, prec):
    """Per-step and interval tests together (the local-dissipation last
    stage carries the interval test)."""
    gd, dyn, l = W.di_config(101, dmax=0.1)
    opts = dict(scheme="eno2", rk=2, cfl=0.5, tol=1e-6, interval=0.05, interval_tol=1e-4,
                max_steps=20000, local_lf=True)
    Vo, so = orc.solve(orc.problem(gd, dyn), l, **opts)
    g = hji_lib.Grid(gd, prec)
    g.set_dynamics(dyn)
    st = g.solve(l.astype(np.float64 if prec == "f64" else np.float32), **opts)
    V = g.value().astype(np.float64)
    g.close()
    assert so["converged"] and st["converged"]
    if prec == "f64":
        assert st["steps"] == so["steps"] and np.abs(V - Vo).max() <= 1e-9
    else:
        assert abs(st["steps"] - so["steps"]) <= max(3, 0.02 * so["steps"])
        assert np.abs(V - Vo).max() <= 1e-4 * np.abs(l).max()


def test_option_values_are_checked(hji_lib, torch_cuda):
    gd, dyn, l = W.di_config(21)
    g = hji_lib.Grid(gd, "f64")
    g.set_dynamics(dyn)
    for bad in (dict(brs=2), dict(local_lf=3)):
        with pytest.raises(hji_lib.HJIError) as e:
            g.solve(l, max_steps=3, **bad)
        assert e.value.status == hji_lib.HJI_E_INVALID
    g.close()
