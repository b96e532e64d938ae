"""Pins of the oracle's optimal control, Eq. (9): u* = argmax_u min_d
<grad V, f(x,u,d)> (and the disturbance attaining the inner minimum).

* At a single state, against a brute-force max-min over dense samples of
  the control and disturbance boxes (no vertex reasoning).
* On a converged double-integrator value, against the closed-form braking
  control: with V* = 1 - max(|x1|, |z|), z = x1 + x2|x2|/(2 umax) (the
  closed-form value pinned elsewhere), dV*/dx2 = -sign(z)|x2|/umax wherever
  the braking term dominates (|z| > |x1|), so u* = -umax sign(z) there.
"""
import numpy as np
import pytest

import workloads as W


def _brute(orc, P, x, p, k=21):
    m, q = P.m, P.q
    ulo, uhi = np.array(P.ulo[:m]), np.array(P.uhi[:m])
    dlo, dhi = np.array(P.dlo[:q]), np.array(P.dhi[:q])
    us = np.stack(np.meshgrid(*[np.linspace(a, b, k) for a, b in zip(ulo, uhi)],
                              indexing="ij"), -1).reshape(-1, m)
    ds = (np.stack(np.meshgrid(*[np.linspace(a, b, k) for a, b in zip(dlo, dhi)],
                               indexing="ij"), -1).reshape(-1, q) if q else np.zeros((1, 0)))

    def inner(u):
        return min(float(np.dot(p, orc.dynamics(P, x, u, d))) for d in ds)

    best = max(inner(u) for u in us)
    return best, inner, ds


@pytest.mark.parametrize("seed", range(8))
def test_control_at_is_the_brute_force_max_min(orc, seed):
    rng = np.random.Generator(np.random.PCG64(100 + seed))
    n = int(rng.integers(2, 4))
    m = int(rng.integers(1, 3))
    q = int(rng.integers(0, 3))
    dyn = {"c": rng.normal(size=n), "A": rng.normal(size=(n, n)),
           "G": rng.normal(size=(n, m)), "ulo": -rng.uniform(0.2, 1.0, m),
           "uhi": rng.uniform(0.2, 1.0, m)}
    if q:
        dyn.update({"E": rng.normal(size=(n, q)), "dlo": -rng.uniform(0.0, 0.5, q),
                    "dhi": rng.uniform(0.0, 0.5, q)})
    gd = W.grid([5] * n, [-1.0] * n, [1.0] * n)
    P = orc.problem(gd, dyn)
    for _ in range(4):
        x = rng.uniform(-1, 1, n)
        p = rng.normal(size=n)
        u, d = orc.control_at(P, x, p)
        # u* is a vertex of U
        assert all(ui in (P.ulo[j], P.uhi[j]) for j, ui in enumerate(u))
        best, inner, ds = _brute(orc, P, x, p)
        assert inner(u) >= best - 1e-12
        # d* attains the inner minimum for u*
        val = float(np.dot(p, orc.dynamics(P, x, u, d)))
        assert val <= inner(u) + 1e-12


def test_double_integrator_braking_control(orc):
    n, umax = 201, 1.0
    gd, dyn, l = W.di_config(n, umax=umax)
    P = orc.problem(gd, dyn)
    V, st = orc.solve(P, l, scheme="eno2", rk=2, cfl=0.5, tol=1e-6, max_steps=20000)
    assert st["converged"]
    u, d = orc.optimal_control(P, "eno2", V)
    assert u.shape == (1, n, n) and d.shape == (0, n, n)
    X1, X2 = W.mesh(gd)
    z = X1 + X2 * np.abs(X2) / (2 * umax)
    dx = 4.0 / (n - 1)
    edge = 6 * dx
    sel = ((np.abs(z) > np.abs(X1) + 0.15) & (np.abs(z) > 0.15) & (np.abs(X2) > 0.15) &
           (np.abs(z) < 1.6) & (np.abs(X1) < 2 - edge) & (np.abs(X2) < 2 - edge))
    assert sel.sum() > 2000
    want = -umax * np.sign(z)
    assert np.array_equal(u[0][sel], want[sel])
