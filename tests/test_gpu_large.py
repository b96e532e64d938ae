"""Largest grids: a 46000 x 46000 FP32 march (2.1e9 nodes, close to the
2^31 - 1 node limit of a grid) for one ENO2/RK2 step, checked node by node
at sampled nodes against the oracle.  After one RK2 step with ENO2 a node
depends only on nodes within 4 of it, so the oracle steps a 17 x 17 window
around each sample with the full grid's alpha and dt and must reproduce the
GPU's value there (FP32 storage: within FP32 rounding of the values)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_near_maximum_grid_sampled_against_oracle(orc, hji_lib):
    import torch
    assert torch.cuda.is_available()
    n = 46000
    free, total = torch.cuda.mem_get_info()
    need = n * n * 4 * 8
    if free < need:
        pytest.skip("needs %.0f GB of free device memory" % (need / 1e9))
    gd, dyn, _ = W.di_config(n, dmax=0.1)
    x = W.node_coords(gd)[0]
    l_dev = (1.0 - torch.from_numpy(np.abs(x)).cuda().float()).reshape(n, 1).expand(n, n)
    l_dev = l_dev.contiguous()
    g = hji_lib.Grid(gd, "f32")
    g.set_dynamics(dyn)
    st = g.solve(l_dev, scheme="eno2", rk=2, cfl=0.5, tol=0.0, max_steps=1)
    assert st["steps"] == 1
    V = torch.empty_like(l_dev)
    g.value(V)
    g.close()
    del l_dev
    alpha, dt = np.array(st["alpha"][:2]), st["dt"]
    rng = np.random.Generator(np.random.PCG64(46))
    samples = [(int(i), int(j)) for i, j in rng.integers(8, n - 8, size=(12, 2))]
    samples += [(n // 2, n // 2), (8, n - 9), (n - 9, 8)]
    h = 8
    dx = 4.0 / (n - 1)
    for i, j in samples:
        wgd = W.grid([2 * h + 1, 2 * h + 1], [-2.0 + (i - h) * dx, -2.0 + (j - h) * dx],
                     [-2.0 + (i + h) * dx, -2.0 + (j + h) * dx])
        P = orc.problem(wgd, dyn)
        X1 = W.mesh(wgd)[0]
        lw = (1.0 - np.abs(X1)).astype(np.float32).astype(np.float64)
        want, _ = orc.step(P, "eno2", 2, dt, alpha, lw, lw)
        got = float(V[i, j].item())
        assert abs(got - want[h, h]) <= 2e-6, (i, j, got, want[h, h])
