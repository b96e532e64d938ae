"""Failure detection without a GPU fault: the waits inside the stage kernels
are bounded.  hji_selftest_bounded_wait runs the stage kernels' wait routine
on an mbarrier armed for bytes that no copy delivers (a flag nothing sets);
the wait must give up after its limit, report it, and leave the device
usable."""
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_reports(orc, hji_lib):
    import torch
    assert torch.cuda.is_available()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc = hji_lib.hji_selftest_bounded_wait(50_000_000, None)  # 50 ms
    wall = time.perf_counter() - t0
    assert rc == hji_lib.HJI_E_TIMEOUT
    assert 0.05 <= wall < 2.0
    # The context is intact: a small march still matches the oracle.
    gd, dyn, l = W.di_config(41)
    g = hji_lib.Grid(gd, "f64")
    g.set_dynamics(dyn)
    st = g.solve(l, scheme="eno2", rk=2, cfl=0.5, tol=0.0, max_steps=20)
    Vo, so = orc.solve(orc.problem(gd, dyn), l, scheme="eno2", rk=2, cfl=0.5, tol=0.0, max_steps=20)
    assert st["steps"] == so["steps"] == 20
    assert np.abs(g.value() - Vo).max() <= 1e-10
    g.close()
