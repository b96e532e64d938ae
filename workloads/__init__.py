"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke run.

This module only *describes problems*: grids, dynamics parameters, target
functions l(x), warm starts k(x), and random instance / request mixes.  It
holds none of the solver's arithmetic (no derivatives, Hamiltonians,
Runge-Kutta stages, reductions), so the CUDA path and the CPU oracle can both
consume its output without sharing any of the method's code.

Problems come from arXiv:1903.07715:
  * the double integrator of Sec. II-A, Eq. (2): p' = v (+ d), v' = b u;
  * the near-hover quadrotor of Sec. VI, Eq. (22), split into 4-D (p, v,
    theta, omega) horizontal subsystems and the 2-D vertical (p_z, v_z) one.
Disturbance placement follows the workload definitions used throughout this
repository: on the velocity equation (v' = b u + d) unless `d_on="p"`
selects the paper's placement (p' = v + d).
All random draws use numpy's PCG64 with an explicit seed.
"""
import math

import numpy as np

G_EARTH = 9.81

# Quadrotor constants printed in Sec. VI (after Eq. (22)).
QUAD_D0, QUAD_D1, QUAD_N0, QUAD_KT = 10.0, 8.0, 10.0, 4.55
QUAD_SMAX_RAD = math.radians(10.0)


# ------------------------------------------------------------------ grids

def grid(n, lo, hi, periodic=None):
    n = [int(v) for v in n]
    lo = [float(v) for v in lo]
    hi = [float(v) for v in hi]
    per = [0] * len(n) if periodic is None else [int(bool(v)) for v in periodic]
    if not (len(n) == len(lo) == len(hi) == len(per)):
        raise ValueError("grid: inconsistent lengths")
    return {"n": n, "lo": lo, "hi": hi, "periodic": per}


def node_coords(gd):
    """1-D node coordinates per axis: lo + i*dx with dx=(hi-lo)/(N-1), or
    (hi-lo)/N on a periodic axis."""
    out = []
    for N, lo, hi, per in zip(gd["n"], gd["lo"], gd["hi"], gd["periodic"]):
        dx = (hi - lo) / (N if per else (N - 1))
        out.append(lo + np.arange(N, dtype=np.float64) * dx)
    return out


def mesh(gd):
    return np.meshgrid(*node_coords(gd), indexing="ij")


def num_cells(gd):
    return int(np.prod(gd["n"]))


# --------------------------------------------------------------- dynamics

def double_integrator(umax=1.0, b=1.0, dmax=0.0, d_on="v", umin=None):
    """Sec. II-A, Eq. (2): x1' = x2 (+ d), x2' = b u (+ d); u in [umin, umax]."""
    umin = -umax if umin is None else umin
    dyn = {"c": [0.0, 0.0], "A": [[0.0, 1.0], [0.0, 0.0]], "G": [[0.0], [b]],
           "ulo": [umin], "uhi": [umax]}
    if dmax is not None and dmax > 0.0:
        dyn["E"] = [[1.0], [0.0]] if d_on == "p" else [[0.0], [1.0]]
        dyn["dlo"], dyn["dhi"] = [-dmax], [dmax]
    return dyn


def quad4d(dmax=0.0, smax=QUAD_SMAX_RAD, d0=QUAD_D0, d1=QUAD_D1, n0=QUAD_N0, g=G_EARTH,
           d_on="v"):
    """One horizontal subsystem of Eq. (22): state (p, v, theta, omega),
    p' = v, v' = g tan(theta), theta' = -d1 theta + omega,
    omega' = -d0 theta + n0 S, |S| <= smax; disturbance on v (or p)."""
    dyn = {"c": [0.0] * 4,
           "A": [[0, 1, 0, 0], [0, 0, 0, 0], [0, 0, -d1, 1], [0, 0, -d0, 0]],
           "G": [[0.0], [0.0], [0.0], [n0]], "ulo": [-smax], "uhi": [smax],
           "terms": [(1, 2, "tan", g)]}
    if dmax > 0.0:
        e = [[1.0], [0.0], [0.0], [0.0]] if d_on == "p" else [[0.0], [1.0], [0.0], [0.0]]
        dyn["E"], dyn["dlo"], dyn["dhi"] = e, [-dmax], [dmax]
    return dyn


def quad_z(mass=1.0, dmax=0.0, kT=QUAD_KT, g=G_EARTH, d_on="v"):
    """The vertical subsystem of Eq. (22): p_z' = v_z, v_z' = (kT/m) T_z - g,
    0 <= T_z <= 2 g; disturbance on v_z (or p_z)."""
    dyn = {"c": [0.0, -g], "A": [[0.0, 1.0], [0.0, 0.0]], "G": [[0.0], [kT / mass]],
           "ulo": [0.0], "uhi": [2.0 * g]}
    if dmax > 0.0:
        dyn["E"] = [[1.0], [0.0]] if d_on == "p" else [[0.0], [1.0]]
        dyn["dlo"], dyn["dhi"] = [-dmax], [dmax]
    return dyn


QUAD4D_BOX = ([-5.0, -4.0, -0.35, -3.0], [5.0, 4.0, 0.35, 3.0])
QUADZ_BOX = ([-5.0, -5.0], [5.0, 5.0])


# ------------------------------------------------------- target functions

def target_strip(gd, axis=0, half_width=1.0):
    """l(x) = w - |x_axis|: unsafe outside the strip |x_axis| <= w."""
    X = mesh(gd)[axis]
    return half_width - np.abs(X)


def target_outside(gd, axis=0, half_width=2.0):
    """l(x) = |x_axis| - w: unsafe inside the strip |x_axis| <= w (the running
    example's target set of Sec. II-B)."""
    X = mesh(gd)[axis]
    return np.abs(X) - half_width


def box_sdf(points, center, half):
    """Signed distance to an axis-aligned box (negative inside)."""
    q = [np.abs(p - c) - h for p, c, h in zip(points, center, half)]
    outside = np.sqrt(sum(np.maximum(qi, 0.0) ** 2 for qi in q))
    inside = np.minimum(np.maximum.reduce(q), 0.0) if len(q) > 1 else np.minimum(q[0], 0.0)
    return outside + inside


def target_boxes(gd, boxes):
    """l(x) = min over boxes of the box signed distance: unsafe inside any box."""
    pts = mesh(gd)
    return np.minimum.reduce([box_sdf(pts, c, h) for c, h in boxes])


def random_boxes(rng, count, center_range=1.5, half_range=(0.1, 0.5), ndim=2):
    return [(rng.uniform(-center_range, center_range, ndim).tolist(),
             rng.uniform(half_range[0], half_range[1], ndim).tolist()) for _ in range(count)]


def warm_circles(gd, seed, count=6, radius=(0.1, 0.5), axes=(0, 1)):
    """A warm start whose sub-zero set is a union of random circles
    (Sec. IV-D): k(x) = min_i (|x - c_i| - r_i)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = mesh(gd)
    lo = [gd["lo"][a] for a in axes]
    hi = [gd["hi"][a] for a in axes]
    out = None
    for _ in range(count):
        c = [rng.uniform(l, h) for l, h in zip(lo, hi)]
        r = rng.uniform(*radius)
        d = np.sqrt(sum((pts[a] - ci) ** 2 for a, ci in zip(axes, c))) - r
        out = d if out is None else np.minimum(out, d)
    return out


# ------------------------------------------------------ named workloads

def di_config(n=101, umax=1.0, dmax=0.0, lo=-2.0, hi=2.0):
    """2-D double integrator on [lo,hi]^2 with l = 1 - |x1|."""
    gd = grid([n, n], [lo, lo], [hi, hi])
    return gd, double_integrator(umax=umax, dmax=dmax), target_strip(gd, 0, 1.0)


def quad4d_config(n=41, dmax=0.0):
    gd = grid([n] * 4, QUAD4D_BOX[0], QUAD4D_BOX[1])
    return gd, quad4d(dmax=dmax), target_strip(gd, 0, 4.0)


def quadz_config(n=501, mass=1.0, dmax=0.0):
    gd = grid([n, n], QUADZ_BOX[0], QUADZ_BOX[1])
    return gd, quad_z(mass=mass, dmax=dmax), target_strip(gd, 0, 4.0)


def batch_instances(count=256, seed=1903, side=(101, 501), umax=(0.5, 2.0), dmax=(0.0, 0.3),
                    boxes=(1, 3)):
    """Uneven double-integrator instances on [-2,2]^2: side ~ U{side}, umax,
    dmax uniform, l = min over 1-3 random box signed distances."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        s = int(rng.integers(side[0], side[1] + 1))
        um = float(rng.uniform(*umax))
        dm = float(rng.uniform(*dmax))
        nb = int(rng.integers(boxes[0], boxes[1] + 1))
        bx = random_boxes(rng, nb)
        gd = grid([s, s], [-2.0, -2.0], [2.0, 2.0])
        out.append({"grid": gd, "dyn": double_integrator(umax=um, dmax=dm), "boxes": bx,
                    "umax": um, "dmax": dm})
    return out


def instance_target(inst):
    return target_boxes(inst["grid"], inst["boxes"])


def poisson_requests(rate=50.0, duration=60.0, seed=7715, quad_side=(31, 61),
                     di_side=(201, 1001), mass_scale=(1.0, 1.5), dmax=(0.0, 0.3),
                     max_requests=None):
    """A Poisson stream of reachability-update requests: half quadrotor 4-D
    subsystems, half 2-D double integrators; each changes the mass (control
    gain scaled by 1/m for the double integrator; the horizontal quadrotor
    subsystem has no mass term in Eq. (22)) or the disturbance bound."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t, out = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t > duration or (max_requests is not None and len(out) >= max_requests):
            break
        kind = "quad4d" if rng.uniform() < 0.5 else "di"
        lo_s, hi_s = quad_side if kind == "quad4d" else di_side
        side = int(rng.integers(lo_s, hi_s + 1))
        change = "mass" if rng.uniform() < 0.5 else "disturbance"
        value = float(rng.uniform(*mass_scale)) if change == "mass" else float(rng.uniform(*dmax))
        out.append({"t": t, "kind": kind, "side": side, "change": change, "value": value})
    return out


def quadz_side(side4d):
    """Grid side of the vertical (p_z, v_z) subsystem that goes with a
    quadrotor whose horizontal subsystems use `side4d` nodes per axis: eight
    times the spacing refinement of one 4-D axis (31 -> 241, 61 -> 481)."""
    return 8 * (int(side4d) - 1) + 1


def route_request(req):
    """Where a serving request lands.  Mass enters the near-hover quadrotor
    of Eq. (22) only through the vertical thrust term, so a quadrotor `mass`
    update is a solve of its 2-D vertical subsystem (grid side quadz_side);
    a `disturbance` update re-solves a 4-D horizontal subsystem.  Double
    integrator requests stay as they are."""
    if req["kind"] == "quad4d" and req["change"] == "mass":
        out = dict(req)
        out["kind"] = "quadz"
        out["side"] = quadz_side(req["side"])
        return out
    return req


def serving_system(kind, side):
    """A resident system of the serving workload: (grid, dynamics factory
    taking (change, value), target l).  Double integrator: `mass` scales the
    control gain to 1/m, `disturbance` sets |d| on the velocity equation.
    Quadrotor 4-D subsystem: `disturbance` sets |d| on v (the horizontal
    subsystem of Eq. (22) has no mass term; mass updates go to the vertical
    subsystem, see route_request).  Quadrotor vertical subsystem (`quadz`):
    `mass` sets m = value (base mass 1.0), `disturbance` sets |d| on v_z."""
    if kind == "quadz":
        gd = grid([side, side], QUADZ_BOX[0], QUADZ_BOX[1])
        l = target_strip(gd, 0, 4.0)

        def dyn(change, value):
            if change == "mass":
                return quad_z(mass=value, dmax=0.0)
            return quad_z(mass=1.0, dmax=value)
        return gd, dyn, l
    if kind == "di":
        gd = grid([side, side], [-2.0, -2.0], [2.0, 2.0])
        l = target_strip(gd, 0, 1.0)

        def dyn(change, value):
            if change == "mass":
                return double_integrator(umax=1.0, b=1.0 / value, dmax=0.0)
            return double_integrator(umax=1.0, dmax=value)
        return gd, dyn, l
    gd = grid([side] * 4, QUAD4D_BOX[0], QUAD4D_BOX[1])
    l = target_strip(gd, 0, 4.0)

    def dyn(change, value):
        return quad4d(dmax=value if change == "disturbance" else 0.0)
    return gd, dyn, l
