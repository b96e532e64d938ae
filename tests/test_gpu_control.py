"""GPU optimal control (Eq. (9)) against the oracle's, through the C ABI.

Both sides take the control decision from the sign of (G^T grad V)_j, with
grad V the average of the scheme's one-sided derivatives of the same value
array.  The decision is unique wherever that component is clearly away from
zero; there the GPU's choice must equal the oracle's exactly.  Where it is
zero or within rounding of zero every choice is optimal, and both are
checked to be vertices of the box.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def _decisive(orc, P, scheme, V, mat, rel):
    """Components of mat^T grad V (shape (k,) + V.shape) and a mask of the
    nodes where each is decided by a margin."""
    g = orc.gradient(P, scheme, V)
    s = np.tensordot(mat.T, g, axes=1)
    scale = np.abs(s).max(axis=tuple(range(1, s.ndim)), keepdims=True)
    return s, np.abs(s) > rel * np.maximum(scale, 1e-300)


def _check(orc, hji, gd, dyn, V, scheme, prec, rel):
    P = orc.problem(gd, dyn)
    g = hji.Grid(gd, prec)
    g.set_dynamics(dyn)
    dt = np.float64 if prec == "f64" else np.float32
    # put V into the grid as its value: a zero-step solve from the warm start V
    g.solve(V.astype(dt), scheme=scheme, rk=1, tol=0.0, max_steps=1, horizon=1e-300)
    Vg = g.value().astype(np.float64)
    u, d = g.optimal_control(scheme)
    g.close()
    uo, do = orc.optimal_control(P, scheme, Vg)
    G = np.asarray(dyn["G"], float).reshape(len(gd["n"]), -1)
    _, mask_u = _decisive(orc, P, scheme, Vg, G, rel)
    assert u.shape == uo.shape
    for j in range(G.shape[1]):
        assert np.isin(u[j], np.array([dyn["ulo"][j], dyn["uhi"][j]]).astype(u.dtype)).all()
        m = mask_u[j]
        assert m.sum() >= min(100, m.size // 10)
        assert np.array_equal(u[j][m], uo[j][m].astype(u.dtype)), j
    if "E" in dyn:
        E = np.asarray(dyn["E"], float).reshape(len(gd["n"]), -1)
        _, mask_d = _decisive(orc, P, scheme, Vg, E, rel)
        for k in range(E.shape[1]):
            assert np.isin(d[k], np.array([dyn["dlo"][k], dyn["dhi"][k]]).astype(d.dtype)).all()
            assert np.array_equal(d[k][mask_d[k]], do[k][mask_d[k]].astype(d.dtype))


def test_double_integrator_converged_f64(orc, hji_lib, torch_cuda):
    gd, dyn, l = W.di_config(101, dmax=0.2)
    g = hji_lib.Grid(gd, "f64")
    g.set_dynamics(dyn)
    g.solve(l, scheme="eno2", rk=2, tol=1e-6, max_steps=20000)
    V = g.value()
    g.close()
    _check(orc, hji_lib, gd, dyn, V, "eno2", "f64", 1e-9)
    _check(orc, hji_lib, gd, dyn, V, "weno5", "f64", 1e-9)


def test_three_d_two_controls_f64(orc, hji_lib, torch_cuda):
    rng = np.random.Generator(np.random.PCG64(3))
    gd = W.grid([13, 19, 35], [-1.0, -2.0, -1.5], [1.0, 2.0, 1.5])
    dyn = {"A": rng.normal(size=(3, 3)) * 0.5, "c": [0.1, -0.2, 0.3],
           "G": [[1.0, 0.0], [0.0, 1.0], [0.5, -0.5]], "ulo": [-1, -0.5], "uhi": [1, 0.7],
           "E": [[0.2], [0.0], [0.3]], "dlo": [-0.3], "dhi": [0.3],
           "terms": [(2, 0, "cos", 0.7), (0, 1, "tan", 0.2)]}
    X = W.mesh(gd)
    V = np.sqrt(X[0] ** 2 + X[1] ** 2 + X[2] ** 2) - 0.8 + 0.1 * np.sin(3 * X[1])
    for scheme in ("eno1", "eno2", "weno5"):
        _check(orc, hji_lib, gd, dyn, V, scheme, "f64", 1e-9)


def test_quadrotor_4d_f32(orc, hji_lib, torch_cuda):
    gd, dyn, l = W.quad4d_config(21, dmax=0.2)
    g = hji_lib.Grid(gd, "f32")
    g.set_dynamics(dyn)
    g.solve(l.astype(np.float32), scheme="eno2", rk=2, tol=0.0, max_steps=30)
    V = g.value().astype(np.float64)
    g.close()
    _check(orc, hji_lib, gd, dyn, V, "eno2", "f32", 1e-4)


def test_device_output_and_errors(orc, hji_lib, torch_cuda):
    import ctypes
    torch = torch_cuda
    gd, dyn, l = W.di_config(41, dmax=0.1)
    g = hji_lib.Grid(gd, "f64")
    g.set_dynamics(dyn)
    u = torch.empty((1, 41, 41), dtype=torch.float64, device="cuda")
    rc = hji_lib.hji_optimal_control(g.handle, hji_lib.HJI_ENO2, u.data_ptr(), None, 1, None)
    assert rc == hji_lib.HJI_E_STATE  # no value yet
    g.solve(l, scheme="eno2", rk=2, tol=1e-6, max_steps=5000)
    d = torch.empty((1, 41, 41), dtype=torch.float64, device="cuda")
    rc = hji_lib.hji_optimal_control(g.handle, hji_lib.HJI_ENO2, u.data_ptr(), d.data_ptr(), 1,
                                     None)
    assert rc == hji_lib.HJI_OK
    uh, dh = g.optimal_control("eno2")
    assert np.array_equal(u.cpu().numpy(), uh) and np.array_equal(d.cpu().numpy(), dh)
    assert hji_lib.hji_optimal_control(g.handle, 9, u.data_ptr(), None, 1, None) == \
        hji_lib.HJI_E_INVALID
    g.close()
