"""GPU parity at the configurations the benchmark measures, against the FP64
oracle (FP32 storage with FP64 reductions on the GPU, as benchmarked):

* the benchmark's own solve: 1001^2 double integrator with |d| <= 0.2,
  WENO5/RK3, warm-started from the d = 0 solution and marched to
  convergence (max|dV| < 1e-6), against the oracle's converged FP64 solution
  of the same problem.  Growing the disturbance is one of the exact cases of
  Sec. V-C / Thm. 2, so the warm and the standard march share their limit;
  the oracle marches from V0 = l.
* the 61^4 quadrotor subsystem of Sec. VI (Eq. (22), |d| <= 0.3, ENO2/RK2)
  for 20 steps from V0 = l, every node against the oracle's 20th step.
* the 501^2 vertical subsystem of Sec. VI (the only one with the mass in
  its dynamics): converged for m = 1.0, |d| = 0, then the update m = 1.3,
  |d| <= 0.3 warm-started from that solution (resident on the device), both
  marched to convergence (max|dV| < 1e-6 max|l|), against the oracle's warm
  march from its own converged m = 1.0 solution.

Bars (the FP32 tolerances of this build): max-abs <= 1e-4 max|l| and
zero-level-set Hausdorff distance <= 1 cell; the GPU's stopping step within
2 % of the oracle's (FP32 rounding can move the step where max|dV| first
drops below the tolerance by a few steps).
"""
import numpy as np
import pytest

import workloads as W
from conftest import brt_hausdorff

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def _gpu_grid(hji, gd, dyn, prec="f32"):
    g = hji.Grid(gd, prec)
    g.set_dynamics(dyn)
    return g


def _steps_close(a, b, rel=0.02, slack=3):
    return abs(a - b) <= max(slack, rel * max(a, b))


def test_bench_solve_1001_weno5_fp32_warm_to_convergence(orc, hji_lib, torch_cuda):
    """The benchmark configuration itself, solved to convergence."""
    gd, dyn, l = W.di_config(1001, dmax=0.2)
    _, dyn0, _ = W.di_config(1001, dmax=0.0)
    opts = dict(scheme="weno5", rk=3, cfl=0.5, tol=1e-6, max_steps=200000)
    l32 = l.astype(np.float32)
    g = _gpu_grid(hji_lib, gd, dyn0)
    s0 = g.solve(l32, **opts)
    assert s0["converged"], s0
    g.set_dynamics(dyn)
    st = g.solve(l32, init=hji_lib.HJI_INIT_RESIDENT, **opts)
    V = g.value().astype(np.float64)
    g.close()
    assert st["converged"], st
    Vo, so = orc.solve(orc.problem(gd, dyn), l, **opts)
    assert so["converged"], so
    err = float(np.abs(V - Vo).max())
    scale = float(np.abs(l).max())
    print("1001^2 WENO5 FP32 warm: steps %d (oracle standard %d), max-abs %.3e (%.3e of max|l|)"
          % (st["steps"], so["steps"], err, err / scale))
    assert err <= 1e-4 * scale
    assert brt_hausdorff(V, Vo) <= 1.0
    # the warm march takes no more steps than the standard one (Sec. V-C)
    assert st["steps"] <= so["steps"] + 3


def test_quad4d_61_fp32_twenty_steps(orc, hji_lib, torch_cuda):
    """61^4 quadrotor subsystem (13.8 M nodes), 20 ENO2/RK2 steps from V0 = l,
    every node against the oracle after the same 20 steps."""
    gd, dyn, l = W.quad4d_config(61, dmax=0.3)
    l32 = l.astype(np.float32)
    g = _gpu_grid(hji_lib, gd, dyn)
    st = g.solve(l32, scheme="eno2", rk=2, cfl=0.5, tol=0.0, max_steps=20)
    V = g.value().astype(np.float64)
    g.close()
    assert st["steps"] == 20
    l64 = l32.astype(np.float64)  # the oracle starts from the same rounded l
    Vo, so = orc.solve(orc.problem(gd, dyn), l64, scheme="eno2", rk=2, cfl=0.5, tol=0.0,
                       max_steps=20)
    assert so["steps"] == 20
    assert abs(st["dt"] - so["dt"]) <= 1e-15 * so["dt"]
    err = float(np.abs(V - Vo).max())
    scale = float(np.abs(l).max())
    print("61^4 FP32 20 steps: max-abs %.3e (%.3e of max|l|)" % (err, err / scale))
    assert err <= 1e-4 * scale
    assert brt_hausdorff(V, Vo) <= 1.0


def test_quad_z_501_mass_update_warm_start(orc, hji_lib, torch_cuda):
    """501^2 vertical subsystem: m 1.0 -> 1.3 with |d| 0 -> 0.3, warm-started
    from the resident m = 1.0 solution, to convergence."""
    gd, dyn_a, l = W.quadz_config(501, mass=1.0, dmax=0.0)
    _, dyn_b, _ = W.quadz_config(501, mass=1.3, dmax=0.3)
    scale = float(np.abs(l).max())
    opts = dict(scheme="eno2", rk=2, cfl=0.5, tol=1e-6 * scale, max_steps=200000)
    l32 = l.astype(np.float32)
    g = _gpu_grid(hji_lib, gd, dyn_a)
    sa = g.solve(l32, **opts)
    assert sa["converged"], sa
    g.set_dynamics(dyn_b)
    sb = g.solve(l32, init=hji_lib.HJI_INIT_RESIDENT, **opts)
    V = g.value().astype(np.float64)
    g.close()
    assert sb["converged"], sb
    Ka, soa = orc.solve(orc.problem(gd, dyn_a), l, **opts)
    Vo, sob = orc.solve(orc.problem(gd, dyn_b), l, Ka, **opts)
    assert soa["converged"] and sob["converged"]
    err = float(np.abs(V - Vo).max())
    print("501^2 z subsystem warm update: steps %d (oracle %d), prior %d (oracle %d), "
          "max-abs %.3e (%.3e of max|l|)" % (sb["steps"], sob["steps"], sa["steps"],
                                            soa["steps"], err, err / scale))
    assert _steps_close(sa["steps"], soa["steps"])
    assert _steps_close(sb["steps"], sob["steps"])
    assert err <= 1e-4 * scale
    assert brt_hausdorff(V, Vo) <= 1.0
