"""hji_stage_times: the march with every RK stage kernel launched on its own
between two CUDA events.  It runs the kernels of hji_solve in the same order,
so its value must equal the oracle's (FP64) and hji_solve's (bit for bit),
and it reports one positive duration per stage."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scheme,rk", [("eno2", 2), ("weno5", 3), ("eno1", 1)])
def test_stage_times_march_matches_oracle(orc, hji_lib, scheme, rk):
    import torch
    assert torch.cuda.is_available()
    gd, dyn, l = W.di_config(45, dmax=0.2)
    g = hji_lib.Grid(gd, "f64")
    g.set_dynamics(dyn)
    ms = g.stage_times(l, steps=12, scheme=scheme, rk=rk, cfl=0.5)
    assert len(ms) == rk and all(m > 0.0 for m in ms)
    Vo, so = orc.solve(orc.problem(gd, dyn), l, scheme=scheme, rk=rk, cfl=0.5, tol=0.0, max_steps=12)
    assert so["steps"] == 12
    assert np.abs(g.value() - Vo).max() <= 1e-10
    g.close()


def test_stage_times_equals_solve_f32(hji_lib):
    import torch
    assert torch.cuda.is_available()
    gd, dyn, l = W.di_config(131, dmax=0.2)
    l32 = l.astype(np.float32)
    a = hji_lib.Grid(gd, "f32")
    a.set_dynamics(dyn)
    ms = a.stage_times(l32, steps=9, scheme="weno5", rk=3, cfl=0.5)
    assert len(ms) == 3 and all(m > 0.0 for m in ms)
    b = hji_lib.Grid(gd, "f32")
    b.set_dynamics(dyn)
    st = b.solve(l32, scheme="weno5", rk=3, cfl=0.5, tol=0.0, max_steps=9, check_every=9)
    assert st["steps"] == 9
    assert np.array_equal(a.value(), b.value())
    # The grid keeps working after the timed march (the solve path's graph
    # is captured afresh or reused).
    st2 = a.solve(l32, scheme="weno5", rk=3, cfl=0.5, tol=0.0, max_steps=9, check_every=9)
    assert st2["steps"] == 9 and np.array_equal(a.value(), b.value())
    a.close()
    b.close()


def test_stage_times_rejects_bad_steps(hji_lib):
    import torch
    assert torch.cuda.is_available()
    gd, dyn, l = W.di_config(41)
    g = hji_lib.Grid(gd, "f64")
    g.set_dynamics(dyn)
    for steps in (0, 5000):
        with pytest.raises(hji_lib.HJIError) as e:
            g.stage_times(l, steps=steps)
        assert e.value.status == hji_lib.HJI_E_INVALID
    g.close()


def test_peak_fma_rates_are_plausible(hji_lib):
    """The measured FMA rates used as the arithmetic roofline: FP32 between a
    tenth and 1.2 times the unit-count rate of 152 SMs x 128 lanes x 2 flops x
    2.07 GHz (80.5 TFLOP/s), FP64 far below FP32 on this GPU."""
    import torch
    assert torch.cuda.is_available()
    f32, ms32 = hji_lib.peak_fma("f32", target_ms=10.0)
    f64, ms64 = hji_lib.peak_fma("f64", target_ms=10.0)
    assert 8.0 <= f32 <= 1.2 * 80.5, f32
    assert 0.0 < f64 < f32 / 4, (f64, f32)
    assert ms32 > 1.0 and ms64 > 1.0
