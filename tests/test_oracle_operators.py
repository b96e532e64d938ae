"""Pins for the oracle's building blocks: one-sided derivatives, dynamics,
Hamiltonian, dissipation coefficients and the CFL step.

Each check compares against something the oracle does not compute itself:
exact polynomial derivatives, measured convergence orders, the model
equations as printed in the paper, and brute-force max/min over dense samples
of the control and disturbance boxes.
"""
import json
import math
import os

import numpy as np
import pytest

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _line(fn, x0, dx, g):
    return np.array([fn(x0 + k * dx) for k in range(-g, g + 1)])


@pytest.mark.parametrize("scheme,deg", [("eno1", 1), ("eno2", 2), ("weno5", 3)])
def test_one_sided_exact_on_polynomials(orc, scheme, deg):
    """ENO1 is exact on linear data, ENO2 on quadratics, WENO5 on cubics."""
    rng = np.random.Generator(np.random.PCG64(11))
    g = orc.ghost_width(scheme)
    for _ in range(20):
        coef = rng.normal(size=deg + 1)
        fn = np.polynomial.Polynomial(coef)
        dfn = fn.deriv()
        x0, dx = rng.uniform(-1, 1), rng.uniform(0.01, 0.2)
        pm, pp = orc.one_sided(scheme, _line(fn, x0, dx, g), dx)
        scale = 1.0 + abs(dfn(x0))
        assert abs(pm - dfn(x0)) < 1e-9 * scale
        assert abs(pp - dfn(x0)) < 1e-9 * scale


def test_eno2_not_exact_on_cubics(orc):
    """Guards the previous test's power: a third-degree term must show up."""
    fn = np.polynomial.Polynomial([0, 0, 0, 1.0])
    pm, pp = orc.one_sided("eno2", _line(fn, 0.3, 0.1, 2), 0.1)
    assert abs(pm - 3 * 0.09) > 1e-4 and abs(pp - 3 * 0.09) > 1e-4


@pytest.mark.parametrize("scheme,order", [("eno1", 1), ("eno2", 2), ("weno5", 5)])
def test_one_sided_convergence_order(orc, scheme, order):
    g = orc.ghost_width(scheme)
    x0 = 0.37
    errs = []
    for dx in [0.04, 0.02, 0.01]:
        pm, pp = orc.one_sided(scheme, _line(np.sin, x0, dx, g), dx)
        errs.append(max(abs(pm - math.cos(x0)), abs(pp - math.cos(x0))))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > order - 0.35, (errs, rates)


def test_eno_picks_smooth_side_at_a_kink(orc):
    """At a kink the ENO choice uses the smooth neighbour: for |x| sampled at
    the kink, the backward derivative is -1 and the forward +1 exactly."""
    dx = 0.1
    line = np.abs(np.arange(-2, 3) * dx)
    pm, pp = orc.one_sided("eno2", line, dx)
    assert pm == pytest.approx(-1.0, abs=1e-14) and pp == pytest.approx(1.0, abs=1e-14)
    # Kink one node to the right: the backward side is linear (slope -1); the
    # forward side mixes both pieces and is not -1.
    line = np.abs((np.arange(-2, 3) - 1) * dx)
    pm, pp = orc.one_sided("eno2", line, dx)
    assert pm == pytest.approx(-1.0, abs=1e-14)
    line7 = np.abs(np.arange(-3, 4) * dx)
    pm, pp = orc.one_sided("weno5", line7, dx)
    assert abs(pm + 1.0) < 1e-3 and abs(pp - 1.0) < 1e-3


def test_weno_flat_data_is_zero(orc):
    pm, pp = orc.one_sided("weno5", np.full(7, 3.25), 0.01)
    assert pm == 0.0 and pp == 0.0


# ------------------------------------------------------------- dynamics

def _paper_params():
    with open(os.path.join(GOLDEN, "paper_parameters.json")) as f:
        return json.load(f)


def test_double_integrator_matches_eq2(orc):
    """Eq. (2): p' = v + d (paper placement), v' = b u."""
    gp = _paper_params()["double_integrator"]
    gd = W.grid([5, 5], [-1, -1], [1, 1])
    dyn = W.double_integrator(umax=gp["umax"], b=0.8, dmax=0.3, d_on="p")
    P = orc.problem(gd, dyn)
    x, u, d = np.array([0.3, -0.7]), np.array([0.9]), np.array([-0.2])
    f = orc.dynamics(P, x, u, d)
    assert f == pytest.approx([-0.7 + -0.2, 0.8 * 0.9], abs=1e-15)


def test_quadrotor_matches_eq22(orc):
    """Eq. (22), horizontal and vertical subsystems, with the constants of Sec. VI."""
    gp = _paper_params()["quadrotor"]
    d0, d1, n0, kT, g = gp["d0"], gp["d1"], gp["n0"], gp["kT"], gp["g"]
    assert (d0, d1, n0, kT) == (W.QUAD_D0, W.QUAD_D1, W.QUAD_N0, W.QUAD_KT)
    assert W.QUAD_SMAX_RAD == pytest.approx(math.radians(gp["S_max_deg"]))
    gd = W.grid([5] * 4, [-1] * 4, [1] * 4)
    P = orc.problem(gd, W.quad4d(dmax=1.0, d_on="p"))
    p, v, th, om = 0.4, -1.1, 0.2, 0.7
    S, dist = 0.1, 0.5
    f = orc.dynamics(P, np.array([p, v, th, om]), np.array([S]), np.array([dist]))
    want = [v + dist, g * math.tan(th), -d1 * th + om, -d0 * th + n0 * S]
    assert f == pytest.approx(want, abs=1e-13)
    m = gp["mass_initial"]
    Pz = orc.problem(W.grid([5, 5], [-1, -1], [1, 1]), W.quad_z(mass=m, dmax=1.0, d_on="p"))
    Tz = 3.0
    f = orc.dynamics(Pz, np.array([0.5, -0.3]), np.array([Tz]), np.array([0.25]))
    assert f == pytest.approx([-0.3 + 0.25, kT / m * Tz - g], abs=1e-13)


def _brute_hamiltonian(orc, P, x, p, m, q, ulo, uhi, dlo, dhi, k=9):
    """max over a dense u-grid of min over a dense d-grid of <p, f>."""
    ug = np.stack(np.meshgrid(*[np.linspace(ulo[j], uhi[j], k) for j in range(m)],
                              indexing="ij"), -1).reshape(-1, m)
    dg = np.stack(np.meshgrid(*[np.linspace(dlo[j], dhi[j], k) for j in range(q)],
                              indexing="ij"), -1).reshape(-1, q) if q else np.zeros((1, 0))
    best = -np.inf
    for u in ug:
        worst = min(float(np.dot(p, orc.dynamics(P, x, u, d))) for d in dg)
        best = max(best, worst)
    return best


def test_hamiltonian_is_max_min_over_boxes(orc):
    """Eq. (6): H = max_u min_d <p, f>, against dense sampling of U and D
    (random control-affine dynamics with nonlinear terms)."""
    rng = np.random.Generator(np.random.PCG64(5))
    for trial in range(12):
        n = int(rng.integers(1, 5))
        m = int(rng.integers(1, 3))
        q = int(rng.integers(0, 3))
        ulo = rng.uniform(-2, 0, m)
        uhi = ulo + rng.uniform(0.1, 2, m)
        dlo = rng.uniform(-1, 0, q)
        dhi = dlo + rng.uniform(0.0, 1, q)
        dyn = {"c": rng.normal(size=n), "A": rng.normal(size=(n, n)),
               "G": rng.normal(size=(n, m)), "ulo": ulo, "uhi": uhi,
               "terms": [(int(rng.integers(n)), int(rng.integers(n)), "sin", 0.7)]}
        if q:
            dyn.update(E=rng.normal(size=(n, q)), dlo=dlo, dhi=dhi)
        P = orc.problem(W.grid([5] * n, [-1] * n, [1] * n), dyn)
        x, p = rng.uniform(-1, 1, n), rng.normal(size=n)
        h = orc.hamiltonian(P, x, p)
        hb = _brute_hamiltonian(orc, P, x, p, m, q, ulo, uhi, dlo, dhi)
        assert h == pytest.approx(hb, abs=1e-12), trial


def test_hamiltonian_roles_double_integrator(orc):
    """The avoid game of Sec. II: for v' = u + d, |u|<=1, |d|<=0.2 and p_v = 1
    the control pushes +1 and the disturbance -0.2, so H = p_x v + 0.8."""
    P = orc.problem(W.grid([5, 5], [-1, -1], [1, 1]), W.double_integrator(dmax=0.2))
    assert orc.hamiltonian(P, np.array([0.0, 0.5]), np.array([2.0, 1.0])) == \
        pytest.approx(2.0 * 0.5 + 0.8, abs=1e-15)
    assert orc.hamiltonian(P, np.array([0.0, 0.5]), np.array([2.0, -1.0])) == \
        pytest.approx(2.0 * 0.5 + 0.8, abs=1e-15)


# ------------------------------------------------------- alpha and dt

def test_alpha_dt_double_integrator(orc):
    gd, dyn, _ = W.di_config(101)
    alpha, dt = orc.alpha_dt(orc.problem(gd, dyn), 0.5)
    assert alpha == pytest.approx([2.0, 1.0], abs=1e-15)
    assert dt == pytest.approx(0.5 / 75.0, rel=1e-14)
    gd, dyn, _ = W.di_config(1001, dmax=0.2)
    alpha, dt = orc.alpha_dt(orc.problem(gd, dyn), 0.5)
    assert alpha == pytest.approx([2.0, 1.2], abs=1e-15)
    assert dt == pytest.approx(0.5 / 800.0, rel=1e-13)


def test_alpha_dt_quadrotor_by_hand(orc):
    gd, dyn, _ = W.quad4d_config(9, dmax=0.3)
    alpha, dt = orc.alpha_dt(orc.problem(gd, dyn), 0.8)
    g, d0, d1, n0, smax = W.G_EARTH, W.QUAD_D0, W.QUAD_D1, W.QUAD_N0, W.QUAD_SMAX_RAD
    want = [4.0, g * math.tan(0.35) + 0.3, d1 * 0.35 + 3.0, d0 * 0.35 + n0 * smax]
    assert alpha == pytest.approx(want, rel=1e-13)
    dx = [10 / 8, 8 / 8, 0.7 / 8, 6 / 8]
    # All four maxima sit at the same corner (|v|, |theta|, |omega| largest,
    # theta and omega of opposite signs), so the rate is the sum of maxima.
    assert dt == pytest.approx(0.8 / sum(a / h for a, h in zip(want, dx)), rel=1e-13)


def test_alpha_point_brute_force(orc):
    rng = np.random.Generator(np.random.PCG64(9))
    P = orc.problem(W.grid([5] * 4, [-1] * 4, [1] * 4), W.quad4d(dmax=0.4))
    for _ in range(5):
        x = rng.uniform(-1, 1, 4)
        us = np.linspace(-W.QUAD_SMAX_RAD, W.QUAD_SMAX_RAD, 7)
        ds = np.linspace(-0.4, 0.4, 7)
        fmax = np.max([np.abs(orc.dynamics(P, x, [u], [d])) for u in us for d in ds], axis=0)
        assert orc.alpha_point(P, x) == pytest.approx(fmax, abs=1e-13)


def test_zero_dynamics_rejected(orc):
    P = orc.problem(W.grid([5], [-1], [1]), {"G": [[0.0]], "ulo": [-1], "uhi": [1]})
    with pytest.raises(ValueError):
        orc.alpha_dt(P, 0.5)
