"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

* One step from an identical V^n (taken from the oracle's own trajectory):
  FP64 must agree to 1e-10 max-abs per step, for every scheme, RK order and
  dimensionality, ragged tile tails, periodic axes and minimal grids.
* Whole marches (standard and warm): same step count, same value to 1e-9.
* FP32 storage with FP64 reductions: within 1e-4 max|l| of the FP64 oracle
  at convergence and the same BRT to one cell.
* Full-size workloads (1001^2 WENO5/RK3, 61^4 ENO2/RK2) in the launch
  configuration the benchmark times: one step compared at every node.
"""
import numpy as np
import pytest

import workloads as W
from conftest import brt_hausdorff

pytestmark = pytest.mark.gpu

TOL_STEP_F64 = 1e-10


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def _grid(hji, gd, dyn, prec="f64"):
    g = hji.Grid(gd, prec)
    g.set_dynamics(dyn)
    return g


def gpu_one_step(hji, gd, dyn, l, Vn, scheme, rk, prec="f64", cfl=0.5):
    g = _grid(hji, gd, dyn, prec)
    st = g.solve(l, Vn, scheme=scheme, rk=rk, cfl=cfl, tol=0.0, max_steps=1)
    out = g.value()
    g.close()
    assert st["steps"] == 1
    return out, st


def oracle_traj(orc, gd, dyn, l, scheme, rk, steps, cfl=0.5, k=None):
    P = orc.problem(gd, dyn)
    alpha, dt = orc.alpha_dt(P, cfl)
    V = orc.init(P, l, k)
    out = [V]
    for _ in range(steps):
        V, _ = orc.step(P, scheme, rk, dt, alpha, l, V)
        out.append(V)
    return P, alpha, dt, out


def _di_rect(ny, nx, dmax=0.1):
    gd = W.grid([ny, nx], [-2.0, -2.0], [2.0, 2.0])
    return gd, W.double_integrator(dmax=dmax), W.target_strip(gd, 0, 1.0)


CASES = [
    # (name, grid dict, dyn, l)
    ("di101", *W.di_config(101)),
    ("di_dist_ragged", *W.di_config(37, dmax=0.2)),
    # 2 x 2 whole 31 x 32 tiles, rows exactly 8-aligned (no padding)
    ("exact_tiles_62x64", *_di_rect(62, 64)),
    # one node row / column into a second tile, rows padded 33 -> 40
    ("one_past_32x33", *_di_rect(32, 33)),
]


@pytest.mark.parametrize("scheme,rk", [("eno1", 1), ("eno2", 2), ("weno5", 3), ("eno2", 3),
                                       ("weno5", 2), ("eno1", 3)])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_one_step_fp64_2d(orc, hji_lib, torch_cuda, case, scheme, rk):
    name, gd, dyn, l = case
    P, alpha, dt, traj = oracle_traj(orc, gd, dyn, l, scheme, rk, 40)
    for n in (0, 1, 5, 20, 40):
        want, _ = orc.step(P, scheme, rk, dt, alpha, l, traj[n])
        got, st = gpu_one_step(hji_lib, gd, dyn, l, traj[n], scheme, rk)
        assert abs(st["dt"] - dt) <= 1e-15 * dt
        err = np.abs(got - want).max()
        assert err <= TOL_STEP_F64, (n, err)


def _quad_case(n):
    gd, dyn, l = W.quad4d_config(n, dmax=0.3)
    return gd, dyn, l


def _nd_case(ndim):
    rng = np.random.Generator(np.random.PCG64(ndim))
    if ndim == 1:
        gd = W.grid([263], [-2.0], [2.0])
        dyn = {"c": [0.3], "G": [[1.0]], "ulo": [-0.5], "uhi": [1.0], "E": [[1.0]],
               "dlo": [-0.2], "dhi": [0.1], "terms": [(0, 0, "sin", 0.4)]}
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
        gd, dyn, l = _quad_case(15)
    return gd, dyn, l


@pytest.mark.parametrize("ndim", [1, 3, 4])
@pytest.mark.parametrize("scheme,rk", [("eno2", 2), ("weno5", 3), ("eno1", 1)])
def test_one_step_fp64_nd(orc, hji_lib, torch_cuda, ndim, scheme, rk):
    gd, dyn, l = _nd_case(ndim)
    P, alpha, dt, traj = oracle_traj(orc, gd, dyn, l, scheme, rk, 12)
    for n in (0, 3, 12):
        want, _ = orc.step(P, scheme, rk, dt, alpha, l, traj[n])
        got, _ = gpu_one_step(hji_lib, gd, dyn, l, traj[n], scheme, rk)
        err = np.abs(got - want).max()
        assert err <= TOL_STEP_F64, (n, err)


@pytest.mark.parametrize("ndim", [1, 3, 4])
@pytest.mark.parametrize("scheme,rk", [("eno2", 2), ("weno5", 3), ("eno1", 1)])
def test_fp32_steps_nd(orc, hji_lib, torch_cuda, ndim, scheme, rk):
    """FP32 compensated storage in 1-D, 3-D and 4-D (the FP32 kernels evaluate
    the slow axes' derivatives two nodes per packed instruction): twelve
    steps from V0 = l against twelve FP64 oracle steps, within the FP32
    rounding of the values."""
    gd, dyn, l = _nd_case(ndim)
    _, _, _, traj = oracle_traj(orc, gd, dyn, l, scheme, rk, 12)
    g = _grid(hji_lib, gd, dyn, "f32")
    st = g.solve(l.astype(np.float32), scheme=scheme, rk=rk, cfl=0.5, tol=0.0, max_steps=12)
    got = g.value().astype(np.float64)
    g.close()
    assert st["steps"] == 12
    assert np.abs(got - traj[12]).max() <= 1e-5 * np.abs(l).max()


@pytest.mark.parametrize("scheme,rk", [("eno2", 2), ("weno5", 3), ("eno1", 1)])
def test_one_step_periodic_and_minimal(orc, hji_lib, torch_cuda, scheme, rk):
    g = orc.ghost_width(scheme)
    nmin = 2 * g + 1
    gd = W.grid([nmin, 48], [-np.pi, -np.pi], [np.pi, np.pi], periodic=[0, 1])
    dyn = {"terms": [(0, 1, "sin", 1.0)], "G": [[0.0], [1.0]], "ulo": [-1.0], "uhi": [1.0]}
    X1, X2 = W.mesh(gd)
    l = np.cos(X2) + 0.3 * X1
    P, alpha, dt, traj = oracle_traj(orc, gd, dyn, l, scheme, rk, 10, k=np.sin(X1 + X2))
    for n in (0, 10):
        want, _ = orc.step(P, scheme, rk, dt, alpha, l, traj[n])
        got, _ = gpu_one_step(hji_lib, gd, dyn, l, traj[n], scheme, rk)
        assert np.abs(got - want).max() <= TOL_STEP_F64


@pytest.mark.parametrize("warm", [False, True])
def test_whole_march_config1(orc, hji_lib, torch_cuda, warm):
    """101^2 double integrator, ENO2/RK2, cfl 0.5, tol 1e-6; warm start from
    the umax = 1.2 solution (Prop. 2)."""
    gd, dyn, l = W.di_config(101)
    opts = dict(scheme="eno2", rk=2, cfl=0.5, tol=1e-6, max_steps=20000)
    P = orc.problem(gd, dyn)
    k = None
    if warm:
        k, _ = orc.solve(orc.problem(gd, W.double_integrator(umax=1.2)), l, **opts)
    Vo, so = orc.solve(P, l, k, **opts)
    g = _grid(hji_lib, gd, dyn)
    st = g.solve(l, k, **opts)
    V = g.value()
    g.close()
    assert st["converged"] and so["converged"]
    assert st["steps"] == so["steps"]
    assert abs(st["tau"] - so["tau"]) <= 1e-12
    assert np.abs(V - Vo).max() <= 1e-9


def test_resident_warm_start_matches_user_k(orc, hji_lib, torch_cuda):
    gd, dyn_old, l = W.di_config(51, umax=1.2)
    dyn = W.double_integrator(umax=1.0)
    opts = dict(scheme="eno2", rk=2, cfl=0.5, tol=1e-6, max_steps=20000)
    g = _grid(hji_lib, gd, dyn_old)
    g.solve(l, **opts)
    k = g.value()
    g.set_dynamics(dyn)
    s1 = g.solve(l, init=hji_lib.HJI_INIT_RESIDENT, **opts)
    V1 = g.value()
    s2 = g.solve(l, k, **opts)
    V2 = g.value()
    g.close()
    assert s1["steps"] == s2["steps"] and np.array_equal(V1, V2)


@pytest.mark.parametrize("n,scheme,rk,dmax", [(101, "eno2", 2, 0.0), (101, "weno5", 3, 0.2),
                                              (201, "weno5", 3, 0.2), (101, "eno2", 3, 0.1)])
def test_fp32_matches_fp64_oracle_at_convergence(orc, hji_lib, torch_cuda, n, scheme, rk, dmax):
    """FP32 storage (increments + compensated value) with FP64 dt/alpha and
    max|dV|: max-abs <= 1e-4 max|l| and the same BRT to one cell."""
    gd, dyn, l = W.di_config(n, dmax=dmax)
    Vo, so = orc.solve(orc.problem(gd, dyn), l, scheme=scheme, rk=rk, cfl=0.5, tol=1e-6)
    g = _grid(hji_lib, gd, dyn, "f32")
    st = g.solve(l.astype(np.float32), scheme=scheme, rk=rk, cfl=0.5, tol=1e-6, max_steps=200000,
                 horizon=so["tau"] * 1.5)
    assert st["converged"], st
    V = g.value().astype(np.float64)
    g.close()
    assert np.abs(V - Vo).max() <= 1e-4 * np.abs(l).max()
    assert brt_hausdorff(V, Vo) <= 1.0


@pytest.mark.parametrize("scheme,rk", [("eno1", 1), ("eno2", 2), ("weno5", 3)])
def test_fp32_matches_fp64_oracle_fixed_horizon(orc, hji_lib, torch_cuda, scheme, rk):
    """FP32 vs the FP64 oracle after the same number of steps (tau = 2).  ENO1's
    max|dV| decays so slowly near 1e-6 that its stopping step is ill-posed, so
    a fixed horizon is the comparison for every scheme here."""
    gd, dyn, l = W.di_config(101, dmax=0.1)
    Vo, so = orc.solve(orc.problem(gd, dyn), l, scheme=scheme, rk=rk, cfl=0.5, tol=0.0,
                       horizon=2.0)
    g = _grid(hji_lib, gd, dyn, "f32")
    st = g.solve(l.astype(np.float32), scheme=scheme, rk=rk, cfl=0.5, tol=0.0, horizon=2.0)
    V = g.value().astype(np.float64)
    g.close()
    assert st["steps"] == so["steps"]
    assert np.abs(V - Vo).max() <= 1e-4 * np.abs(l).max()
    assert brt_hausdorff(V, Vo) <= 1.0


def test_full_size_config2_one_step(orc, hji_lib, torch_cuda):
    """1001^2, |d| <= 0.2, WENO5/RK3: every node of one step from the oracle's
    V^n (n = 0 and n = 3), FP64."""
    gd, dyn, l = W.di_config(1001, dmax=0.2)
    P, alpha, dt, traj = oracle_traj(orc, gd, dyn, l, "weno5", 3, 3)
    for n in (0, 3):
        want, _ = orc.step(P, "weno5", 3, dt, alpha, l, traj[n])
        got, _ = gpu_one_step(hji_lib, gd, dyn, l, traj[n], "weno5", 3)
        assert np.abs(got - want).max() <= TOL_STEP_F64


def test_full_size_quad61_one_step_fp32(orc, hji_lib, torch_cuda):
    """61^4 quadrotor subsystem, ENO2/RK2, FP32 storage: one step from V^0 = l
    against the FP64 oracle, within the FP32 rounding of the values."""
    gd, dyn, l = W.quad4d_config(61, dmax=0.3)
    P = orc.problem(gd, dyn)
    alpha, dt = orc.alpha_dt(P, 0.5)
    l32 = l.astype(np.float32)
    want, _ = orc.step(P, "eno2", 2, dt, alpha, l32.astype(np.float64), l32.astype(np.float64))
    got, _ = gpu_one_step(hji_lib, gd, dyn, l32, l32, "eno2", 2, prec="f32")
    assert np.abs(got.astype(np.float64) - want).max() <= 1e-5 * np.abs(l).max()


def test_invalid_inputs_rejected(hji_lib, torch_cuda):
    gd, dyn, l = W.di_config(21)
    g = _grid(hji_lib, gd, dyn)
    bad = l.copy()
    bad[3, 4] = np.nan
    with pytest.raises(hji_lib.HJIError) as e:
        g.solve(bad, max_steps=5)
    assert e.value.status == hji_lib.HJI_E_INVALID
    with pytest.raises(hji_lib.HJIError) as e:
        g.solve(l, cfl=1.5, max_steps=5)
    assert e.value.status == hji_lib.HJI_E_INVALID
    st = g.solve(l, tol=0.0, max_steps=7)
    assert st["steps"] == 7 and not st["converged"]
    g.close()
    g2 = hji_lib.Grid(gd, "f64")
    with pytest.raises(hji_lib.HJIError) as e:
        g2.solve(l, max_steps=5)
    assert e.value.status == hji_lib.HJI_E_STATE
    g2.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_rate_rule_stops_like_the_oracle(orc, hji_lib, torch_cuda, prec):
    """Sec. IV's convergence rule as a rate (tol_rate = 0.1: change < 0.001
    per 0.01 of time): same stopping step as the oracle."""
    gd, dyn, l = W.di_config(101, dmax=0.1)
    opts = dict(scheme="eno2", rk=2, cfl=0.5, tol=0.0, tol_rate=0.1, max_steps=20000)
    Vo, so = orc.solve(orc.problem(gd, dyn), l, **opts)
    g = _grid(hji_lib, gd, dyn, prec)
    st = g.solve(l.astype(np.float64 if prec == "f64" else np.float32), **opts)
    V = g.value().astype(np.float64)
    g.close()
    assert so["converged"] and st["converged"]
    assert st["steps"] == so["steps"]
    assert np.abs(V - Vo).max() <= (1e-9 if prec == "f64" else 1e-4 * np.abs(l).max())
