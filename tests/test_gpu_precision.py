"""Precision pattern: an FP32 march (FP32 stencil and Hamiltonian, FP64 dt
and max|dV|) followed by an FP64 re-validation sweep warm-started from its
result.  By Thm. 1 / Thm. 2 the sweep is conservative, and exact when the
FP32 value lies above the FP64 solution; here it must land on the FP64
oracle's solution within 1e-4 max|l| with the same BRT, in far fewer FP64
steps than a standard FP64 solve."""
import numpy as np
import pytest

import workloads as W
from conftest import brt_hausdorff

pytestmark = pytest.mark.gpu


def test_value_transfer_round_trip(hji_lib):
    import torch
    assert torch.cuda.is_available()
    gd, dyn, l = W.di_config(61, dmax=0.1)
    g64 = hji_lib.Grid(gd, "f64")
    g64.set_dynamics(dyn)
    g64.solve(l, scheme="eno2", rk=2, tol=1e-6, max_steps=5000)
    V = g64.value()
    g32 = hji_lib.Grid(gd, "f32")
    g32.set_dynamics(dyn)
    g32.take_value(g64)           # exact hi/lo split of the FP64 value
    back = hji_lib.Grid(gd, "f64")
    back.set_dynamics(dyn)
    back.take_value(g32)          # hi + lo back in FP64
    assert np.abs(back.value() - V).max() <= 1e-13 * np.abs(V).max()
    assert np.array_equal(g32.value(), V.astype(np.float32))
    for g in (g64, g32, back):
        g.close()


def test_fp32_then_fp64_revalidation(orc, hji_lib):
    import torch
    assert torch.cuda.is_available()
    gd, dyn, l = W.di_config(201, dmax=0.2)
    opts = dict(scheme="weno5", rk=3, cfl=0.5, tol=1e-6, max_steps=100000)
    Vo, so = orc.solve(orc.problem(gd, dyn), l, **opts)
    g32 = hji_lib.Grid(gd, "f32")
    g32.set_dynamics(dyn)
    s32 = g32.solve(l.astype(np.float32), **opts)
    g64 = hji_lib.Grid(gd, "f64")
    g64.set_dynamics(dyn)
    g64.take_value(g32)
    s64 = g64.solve(l, init=hji_lib.HJI_INIT_RESIDENT, **opts)
    V = g64.value()
    assert s32["converged"] and s64["converged"]
    assert np.abs(V - Vo).max() <= 1e-4 * np.abs(l).max()
    assert brt_hausdorff(V, Vo) == 0.0
    assert s64["steps"] < 0.25 * so["steps"]
    g32.close()
    g64.close()
