"""Pins of the oracle's discounted reachability (Sec. II-C): every step ends
with V <- min(l, gamma * V~), V~ the Runge-Kutta step's result and gamma =
exp(-lambda dt) the discount of one CFL step.

* A closed form: x' = c on a periodic grid, ENO1 / forward Euler at Courant
  number 1 is the exact one-cell shift S (upwind differencing), so the
  discounted march unrolls to V^n = min(l, gamma S l, ..., gamma^(n-1)
  S^(n-1) l, gamma^n S^n V^0), evaluated here with array rolls alone.
* The section's claim that the discounted map is a contraction, so that any
  initialisation is forgotten: on the order-preserving scheme (ENO1 +
  forward Euler at CFL <= 1, global Lax-Friedrichs) two marches from
  different starts come together at least as fast as gamma^n.  Without the
  discount a start below the solution is not forgotten (Thm. 1).
* gamma = 0 and gamma = 1 both mean "off": the undiscounted march, bit for
  bit.
"""
import numpy as np
import pytest

import workloads as W

TORUS = W.grid([48, 40], [-np.pi, -np.pi], [np.pi, np.pi], periodic=[1, 1])


def _shift_problem(orc, n=64, c=0.7):
    gd = W.grid([n], [-np.pi], [np.pi], periodic=[1])
    P = orc.problem(gd, {"c": [c], "G": np.zeros((1, 0))})
    alpha, dt = orc.alpha_dt(P, 1.0)
    x = W.node_coords(gd)[0]
    return P, alpha, dt, x


def test_courant_one_is_the_exact_shift(orc):
    """The premise of the closed form: one undiscounted step without the
    projection moves every value one node against the flow."""
    P, alpha, dt, x = _shift_problem(orc)
    assert dt == pytest.approx(2 * np.pi / 64 / 0.7, rel=1e-15)
    v = np.cos(x) + 0.3 * np.sin(3 * x)
    out, _ = orc.step(P, "eno1", 1, dt, alpha, v, v, brs=True)
    assert np.abs(out - np.roll(v, -1)).max() <= 1e-15


@pytest.mark.parametrize("gamma", [0.97, 0.5])
def test_discounted_shift_closed_form(orc, gamma):
    P, alpha, dt, x = _shift_problem(orc)
    l = np.cos(x) - 0.2 + 0.3 * np.sin(3 * x)
    k = l - 1.5 + 0.5 * np.cos(2 * x)
    V0 = orc.init(P, l, k)
    V = V0
    for n in range(1, 61):
        V, _ = orc.step(P, "eno1", 1, dt, alpha, l, V, discount=gamma)
        want = gamma ** n * np.roll(V0, -n)
        for j in range(n):
            want = np.minimum(want, gamma ** j * np.roll(l, -j))
        assert np.abs(V - want).max() <= 1e-14, n
    # the limit is min over the whole orbit of gamma^j S^j l: negative
    # wherever l is negative, and above min(l, 0) elsewhere
    assert np.all(V[l < 0] < 0)


def test_discounted_solve_reaches_the_shift_fixed_point(orc):
    """At convergence V = min(l, gamma S V): the fixed point of the closed
    form, reached from two different starts."""
    gamma = 0.9
    P, alpha, dt, x = _shift_problem(orc)
    l = np.cos(x) - 0.2 + 0.3 * np.sin(3 * x)
    fixed = l.copy()
    for j in range(1, 2000):
        fixed = np.minimum(fixed, gamma ** j * np.roll(l, -j))
    for k in (None, np.full_like(l, -4.0)):
        V, st = orc.solve(P, l, k=k, scheme="eno1", rk=1, cfl=1.0, tol=1e-13, max_steps=5000,
                          discount=gamma)
        assert st["converged"]
        assert np.abs(V - fixed).max() <= 1e-11
        assert np.abs(V - np.minimum(l, gamma * np.roll(V, -1))).max() <= 1e-12


def _torus_problem(orc):
    dyn = {"A": np.zeros((2, 2)), "terms": [(0, 1, "sin", 1.0)], "G": [[0.0], [1.0]],
           "ulo": [-1.0], "uhi": [1.0], "E": [[1.0], [0.0]], "dlo": [-0.2], "dhi": [0.2]}
    P = orc.problem(TORUS, dyn)
    alpha, dt = orc.alpha_dt(P, 0.9)
    l = np.cos(W.mesh(TORUS)[0]) - 0.2
    return P, alpha, dt, l


def test_discounted_map_is_a_contraction(orc):
    """Sec. II-C: the discounted update forgets its initialisation; on the
    order-preserving scheme two starts approach each other like gamma^n."""
    gamma = 0.98
    P, alpha, dt, l = _torus_problem(orc)
    X1, X2 = W.mesh(TORUS)
    Va = orc.init(P, l, np.full_like(l, -2.0))
    Vb = orc.init(P, l, 0.5 * np.sin(X2) - 0.1)
    gap0 = np.abs(Va - Vb).max()
    assert gap0 > 1.0
    for n in range(1, 301):
        Va, _ = orc.step(P, "eno1", 1, dt, alpha, l, Va, discount=gamma)
        Vb, _ = orc.step(P, "eno1", 1, dt, alpha, l, Vb, discount=gamma)
        assert np.abs(Va - Vb).max() <= gamma ** n * gap0 + 1e-12, n
    assert np.abs(Va - Vb).max() < 0.01 * gap0


def test_undiscounted_march_keeps_a_low_start(orc):
    """The contrast: without the discount the march from V0 = -2 never rises
    to the standard march's values (Thm. 1), so the gap does not close."""
    P, alpha, dt, l = _torus_problem(orc)
    Va = orc.init(P, l, np.full_like(l, -2.0))
    Vb = orc.init(P, l)
    for _ in range(300):
        Va, _ = orc.step(P, "eno1", 1, dt, alpha, l, Va)
        Vb, _ = orc.step(P, "eno1", 1, dt, alpha, l, Vb)
    assert np.abs(Va - Vb).max() > 1.0


@pytest.mark.parametrize("off", [0.0, 1.0])
def test_discount_off_is_the_plain_march(orc, off):
    gd, dyn, l = W.di_config(41, dmax=0.2)
    P = orc.problem(gd, dyn)
    a, sa = orc.solve(P, l, scheme="weno5", rk=3, tol=0.0, max_steps=30)
    b, sb = orc.solve(P, l, scheme="weno5", rk=3, tol=0.0, max_steps=30, discount=off)
    assert np.array_equal(a, b) and sa["steps"] == sb["steps"]
