"""Pins of the oracle against the definitions its formulas come from, computed
here by a different route than the oracle's closed forms:

* HJ-WENO5 (Jiang and Peng): each candidate is the derivative at the node of
  the cubic interpolating the values on its four nodes; the ideal weights are
  the ones that make the candidates' combination the derivative of the quintic
  through all six nodes; each smoothness indicator is the Jiang-Shu integral,
  over the central cell, of the squared first and second derivatives of the
  quadratic whose cell averages are the candidate's three first differences.
  Interpolants, the weight system and the integrals are solved numerically
  with numpy; nothing below retypes the oracle's coefficients.
* The right-biased derivative is the mirror image of the left-biased one.
* Ghost nodes: linear extrapolation of the two edge nodes, or periodic wrap.
* ENO2: the derivative of the Newton quadratic that adds the neighbour with
  the smaller second divided difference.
* The dynamics' sin / cos / tan terms, against numpy.
* Eq. (9) at a known gradient, and its tie reading (a zero component of
  G^T grad V takes the upper control bound, a zero component of E^T grad V the
  lower disturbance bound).
* Eq. (5) alone from a given start: the start is taken as it is, not
  min(k, l).
"""
import numpy as np
import pytest
from numpy.polynomial import Polynomial as Poly

import workloads as W


# ------------------------------------------------------------ references

def _interp_deriv(xs, ys, x0):
    """Derivative at x0 of the polynomial interpolating (xs, ys)."""
    p = Poly.fit(xs, ys, len(xs) - 1, domain=[min(xs), max(xs)], window=[min(xs), max(xs)])
    return p.deriv()(x0)


def _ideal_weights():
    """Weights d with sum_k d_k phi_k = derivative of the quintic through the
    six nodes -3..2 (node 0 the centre), fixed by exactness on degree 4 and 5
    and by summing to one."""
    nodes = np.arange(-3, 3, dtype=float)
    rows, rhs = [], []
    for deg in (4, 5):
        ys = nodes ** deg
        rows.append([_interp_deriv(nodes[k:k + 4], ys[k:k + 4], 0.0) for k in range(3)])
        rhs.append(_interp_deriv(nodes, ys, 0.0))
    rows.append([1.0, 1.0, 1.0])
    rhs.append(1.0)
    return np.linalg.solve(np.array(rows), np.array(rhs))


def _smoothness(avgs, first_cell):
    """Jiang-Shu indicator: the quadratic q with the given averages over the
    unit cells [c, c+1] (c = first_cell, first_cell+1, first_cell+2), then
    the integral over [0, 1] of q'^2 + q''^2 (unit spacing)."""
    A = np.zeros((3, 3))
    for r in range(3):
        a, b = first_cell + r, first_cell + r + 1
        for j in range(3):
            A[r, j] = (b ** (j + 1) - a ** (j + 1)) / (j + 1)
    q = Poly(np.linalg.solve(A, np.asarray(avgs, float)))
    tot = 0.0
    for der in (q.deriv(1), q.deriv(2)):
        integ = (der * der).integ()
        tot += integ(1.0) - integ(0.0)
    return tot


D_IDEAL = _ideal_weights()


def _weno5_backward(line, dx):
    """Left-biased HJ-WENO5 derivative at the centre of 7 values."""
    x = (np.arange(7) - 3) * dx
    line = np.asarray(line, float)
    cand = [_interp_deriv(x[k:k + 4], line[k:k + 4], 0.0) for k in range(3)]
    v = np.diff(line) / dx        # v[0..5]; the backward stencil uses v[0..4]
    beta = [_smoothness(v[0:3], -2), _smoothness(v[1:4], -1), _smoothness(v[2:5], 0)]
    eps = 1e-6 * float(np.max(v[0:5] ** 2)) + 1e-99
    a = np.array([D_IDEAL[k] / (beta[k] + eps) ** 2 for k in range(3)])
    return float(np.dot(a / a.sum(), cand))


def _ref_one_sided(scheme, line, dx):
    line = np.asarray(line, float)
    c = len(line) // 2
    if scheme == "eno1":
        return (line[c] - line[c - 1]) / dx, (line[c + 1] - line[c]) / dx
    if scheme == "eno2":
        def side(base, cands):
            # Newton quadratic through the two base nodes and whichever
            # candidate gives the smaller |second divided difference|; its
            # derivative at the centre (ties: the lower node index).
            best = None
            for k in cands:
                idx = sorted(base + [k])
                dd = np.polyfit((np.array(idx) - c) * dx, line[idx], 2)[0]
                if best is None or abs(dd) < abs(best[0]):
                    best = (dd, idx)
            idx = best[1]
            return _interp_deriv((np.array(idx) - c) * dx, line[idx], 0.0)
        return side([c - 1, c], [c - 2, c + 1]), side([c, c + 1], [c - 1, c + 2])
    pm = _weno5_backward(line, dx)
    pp = -_weno5_backward(line[::-1], dx)
    return pm, pp


def _ghosted(V, g, periodic):
    """V extended by g ghost nodes on each side: wrap, or edge + k (edge - inner)."""
    N = len(V)
    out = np.empty(N + 2 * g)
    out[g:g + N] = V
    for k in range(1, g + 1):
        if periodic:
            out[g - k] = V[(-k) % N]
            out[g + N - 1 + k] = V[(N - 1 + k) % N]
        else:
            out[g - k] = V[0] + k * (V[0] - V[1])
            out[g + N - 1 + k] = V[N - 1] + k * (V[N - 1] - V[N - 2])
    return out


# ---------------------------------------------------------------- WENO5

def test_weno_reference_reproduces_the_published_weights():
    """The numerically solved ideal weights are Jiang and Peng's 1/10, 6/10,
    3/10, and the integral indicator of the central stencil on the differences
    (1, 0, 0) is 13/12 + 1/4 = 4/3 (a check of the reference itself)."""
    assert D_IDEAL == pytest.approx([0.1, 0.6, 0.3], abs=1e-12)
    assert _smoothness([1.0, 0.0, 0.0], -1) == pytest.approx(13.0 / 12.0 + 0.25, abs=1e-12)


def test_weno5_matches_its_definition_on_rough_data(orc):
    """Random, non-smooth stencil lines (weights far from the ideal ones):
    both one-sided derivatives equal the definition's to rounding."""
    rng = np.random.Generator(np.random.PCG64(2024))
    for t in range(300):
        dx = float(rng.uniform(0.005, 0.3))
        kind = t % 3
        if kind == 0:
            line = rng.normal(size=7)
        elif kind == 1:   # a kink at a random position
            k0 = rng.uniform(-3, 3)
            line = np.abs((np.arange(7) - 3) - k0) * dx + rng.normal(scale=1e-3, size=7)
        else:             # a jump in the slope plus a smooth part
            xs = (np.arange(7) - 3) * dx
            line = np.sin(3 * xs) + np.where(xs > rng.uniform(-2, 2) * dx, 2.0 * xs, 0.0)
        pm, pp = orc.one_sided("weno5", line, dx)
        rm, rp = _ref_one_sided("weno5", line, dx)
        scale = float(np.max(np.abs(np.diff(line)))) / dx + 1e-300
        assert abs(pm - rm) <= 1e-11 * scale, (t, pm, rm)
        assert abs(pp - rp) <= 1e-11 * scale, (t, pp, rp)


def test_eno2_matches_newton_form(orc):
    rng = np.random.Generator(np.random.PCG64(7))
    for _ in range(200):
        dx = float(rng.uniform(0.01, 0.5))
        line = rng.normal(size=5)
        pm, pp = orc.one_sided("eno2", line, dx)
        rm, rp = _ref_one_sided("eno2", line, dx)
        scale = float(np.max(np.abs(np.diff(line)))) / dx
        assert abs(pm - rm) <= 1e-12 * scale and abs(pp - rp) <= 1e-12 * scale


# ------------------------------------------------- ghost nodes, gradient

@pytest.mark.parametrize("scheme", ["eno1", "eno2", "weno5"])
@pytest.mark.parametrize("periodic", [False, True])
def test_gradient_at_every_node_with_ghosts(orc, scheme, periodic):
    """oracle.gradient = (p- + p+)/2 at every node of a rough 1-D field, the
    ghost nodes built from their definition (edge nodes included: the
    second and third ghost layers feed WENO5 there)."""
    rng = np.random.Generator(np.random.PCG64(31 + periodic))
    n = 23
    gd = W.grid([n], [-1.0], [1.3], periodic=[periodic])
    P = orc.problem(gd, {"c": [1.0], "G": np.zeros((1, 0))})
    dx = orc.spacing(P, 0)
    V = rng.normal(size=n) + np.linspace(0.0, 3.0, n)
    got = orc.gradient(P, scheme, V)[0]
    g = orc.ghost_width(scheme)
    ext = _ghosted(V, g, periodic)
    for i in range(n):
        rm, rp = _ref_one_sided(scheme, ext[i:i + 2 * g + 1], dx)
        scale = float(np.max(np.abs(np.diff(ext[i:i + 2 * g + 1])))) / dx
        assert abs(got[i] - 0.5 * (rm + rp)) <= 1e-11 * scale, (i, got[i], 0.5 * (rm + rp))


def test_gradient_2d_axes(orc):
    """In 2-D each component is the 1-D gradient along its own axis (rows for
    axis 1, columns for axis 0), with ghosts of that axis only."""
    rng = np.random.Generator(np.random.PCG64(5))
    gd = W.grid([9, 12], [-1.0, 0.0], [1.0, 2.0])
    P = orc.problem(gd, {"c": [1.0, 1.0], "G": np.zeros((2, 0))})
    V = rng.normal(size=(9, 12))
    got = orc.gradient(P, "weno5", V)
    for a in range(2):
        dx = orc.spacing(P, a)
        Vt = np.moveaxis(V, a, -1)
        want = np.empty_like(Vt)
        for r in range(Vt.shape[0]):
            ext = _ghosted(Vt[r], 3, False)
            for i in range(Vt.shape[1]):
                rm, rp = _ref_one_sided("weno5", ext[i:i + 7], dx)
                want[r, i] = 0.5 * (rm + rp)
        want = np.moveaxis(want, -1, a)
        assert np.abs(got[a] - want).max() <= 1e-11 * (np.abs(want).max() + 1.0)


# -------------------------------------------------------------- dynamics

def test_dynamics_trig_terms(orc):
    """f_i = c_i + (A x)_i + sum of w sin/cos/tan(x_axis) terms + (G u)_i + (E d)_i."""
    gd = W.grid([5, 5, 5], [-1] * 3, [1] * 3)
    A = np.array([[0.1, -0.4, 0.0], [0.3, 0.0, 0.2], [0.0, 0.5, -0.7]])
    G = np.array([[1.0, 0.0], [0.0, 0.3], [0.2, -1.1]])
    E = np.array([[0.0], [0.6], [-0.4]])
    dyn = {"c": [0.2, -0.1, 0.05], "A": A, "G": G, "E": E, "ulo": [-1, -2], "uhi": [1, 2],
           "dlo": [-0.5], "dhi": [0.5],
           "terms": [(0, 1, "sin", 0.7), (1, 2, "cos", -1.3), (2, 0, "tan", 0.4),
                     (1, 0, "cos", 0.25)]}
    P = orc.problem(gd, dyn)
    rng = np.random.Generator(np.random.PCG64(9))
    for _ in range(20):
        x = rng.uniform(-1, 1, 3)
        u = rng.uniform(-1, 1, 2)
        d = rng.uniform(-0.5, 0.5, 1)
        want = np.array(dyn["c"]) + A @ x + G @ u + E @ d
        want[0] += 0.7 * np.sin(x[1])
        want[1] += -1.3 * np.cos(x[2]) + 0.25 * np.cos(x[0])
        want[2] += 0.4 * np.tan(x[0])
        assert orc.dynamics(P, x, u, d) == pytest.approx(want, abs=1e-14)


# ------------------------------------------------------- Eq. (9) control

def test_control_ties_take_upper_control_and_lower_disturbance(orc):
    """A zero component of G^T p (every control value optimal) takes uhi, a
    zero component of E^T p takes dlo; a nonzero one its bang-bang side."""
    gd = W.grid([5, 5], [-1, -1], [1, 1])
    dyn = {"c": [0.0, 0.0], "G": [[1.0, 0.0], [0.0, 1.0]], "ulo": [-1.0, -3.0],
           "uhi": [2.0, 0.5], "E": [[1.0, 0.0], [0.0, 1.0]], "dlo": [-0.2, -0.4],
           "dhi": [0.1, 0.3]}
    P = orc.problem(gd, dyn)
    x = np.array([0.1, 0.2])
    u, d = orc.control_at(P, x, np.zeros(2))
    assert list(u) == [2.0, 0.5] and list(d) == [-0.2, -0.4]
    u, d = orc.control_at(P, x, np.array([0.0, -1.0]))
    assert list(u) == [2.0, -3.0] and list(d) == [-0.2, 0.3]
    u, d = orc.control_at(P, x, np.array([1.0, 0.0]))
    assert list(u) == [2.0, 0.5] and list(d) == [-0.2, -0.4]


def test_optimal_control_uses_the_averaged_gradient(orc):
    """For V = (x2 - s)^2 / 2 + x1 / 4 the ENO1 average (p- + p+)/2 is the
    central difference, exact on quadratics, so at interior nodes
    dV/dx2 = x2 - s and the double integrator's control is umax sign(x2 - s).
    s sits a quarter cell above a node row: there x2 - s = -dx/4, which a
    one-sided gradient (off by dx/2) would get with the wrong sign."""
    n, umax = 41, 1.5
    gd = W.grid([n, n], [-2.0, -2.0], [2.0, 2.0])
    P = orc.problem(gd, W.double_integrator(umax=umax, b=1.0, dmax=0.0))
    x1, x2 = W.node_coords(gd)
    dx = x2[1] - x2[0]
    s = x2[17] + 0.25 * dx
    X1, X2 = np.meshgrid(x1, x2, indexing="ij")
    V = 0.5 * (X2 - s) ** 2 + 0.25 * X1
    u, _ = orc.optimal_control(P, "eno1", V)
    want = np.where(X2 - s > 0, umax, -umax)
    inner = (slice(1, n - 1), slice(1, n - 1))
    assert np.array_equal(u[0][inner], want[inner])
    assert (want[inner] < 0).any() and (want[inner] > 0).any()


# ------------------------------------------------ Eq. (5) from a given k

def test_brs_solve_starts_from_k_as_given(orc):
    """x' = c on a periodic line, ENO1 and one Euler step at Courant number 1:
    L = c p+, so the step moves the start one cell upstream exactly.  Without
    the projection the start is k itself, also where k is above l."""
    n = 64
    gd = W.grid([n], [0.0], [1.0], periodic=[True])
    P = orc.problem(gd, {"c": [1.0], "G": np.zeros((1, 0))})
    x = W.node_coords(gd)[0]
    l = np.cos(2 * np.pi * x)
    k = l + 0.5 + 0.3 * np.sin(6 * np.pi * x)
    assert (k > l + 0.1).all()
    V, st = orc.solve(P, l, k=k, scheme="eno1", rk=1, cfl=1.0, tol=0.0, max_steps=1, brs=True)
    assert st["steps"] == 1
    assert np.abs(V - np.roll(k, -1)).max() < 1e-13
    # with the projection, the same step starts from min(k, l) = l and ends at or below l
    V2, _ = orc.solve(P, l, k=k, scheme="eno1", rk=1, cfl=1.0, tol=0.0, max_steps=1)
    assert np.abs(V2 - np.minimum(np.roll(l, -1), l)).max() < 1e-13
