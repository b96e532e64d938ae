"""Closed-form values derived from the paper's definitions, used as pins.

Each follows from the cost functional of Sec. II-B, Eq. (3)-(4): the value is
the smallest target value l along the trajectory played by an optimal control
against a worst-case disturbance.  None of these reuses the solver's
arithmetic; they are answers worked out by hand for special dynamics.
"""
import numpy as np


def di_strip_value(x1, x2, u_eff, w=1.0):
    """Double integrator x1' = x2, x2' = b u + d with |u| <= umax, |d| <= dmax,
    u_eff = b umax - dmax > 0, target l = w - |x1| (unsafe outside the strip).

    Full braking is optimal; the disturbance opposes it, so the state stops at
    x1 + x2|x2| / (2 u_eff) and can then hold still.  The largest |x1| along
    that path is max(|x1|, |x1 + x2|x2|/(2 u_eff)|), hence
        V*(x) = w - max(|x1|, |x1 + x2 |x2| / (2 u_eff)|).
    Its zero super-level set is the safe set -w <= x1 + x2|x2|/(2u) <= w,
    |x1| <= w."""
    stop = x1 + x2 * np.abs(x2) / (2.0 * u_eff)
    return w - np.maximum(np.abs(x1), np.abs(stop))


def di_stop_position(x1, x2, u_eff):
    return x1 + x2 * np.abs(x2) / (2.0 * u_eff)


def di_paper_strip_value(p, v, u_eff, w=2.0):
    """Running example of Sec. II-B: unsafe strip |p| <= w, l = |p| - w.
    Moving away keeps min|p| = |p|; moving toward the strip, full braking
    stops at p + v|v|/(2u), or the path crosses p = 0 (min|p| = 0):
        V*(p,v) = min(|p|, max(0, sgn(p) (p + v|v|/(2u)))) - w."""
    stop = p + v * np.abs(v) / (2.0 * u_eff)
    return np.minimum(np.abs(p), np.maximum(0.0, np.sign(p) * stop)) - w


def advection_value(x, tau, c, l_fn):
    """x' = c (no inputs): V(x, tau) = min over s in [0, tau] of l(x + c s),
    evaluated by dense sampling of s (the minimum of Eq. (3) over the path)."""
    s = np.linspace(0.0, tau, 4001)
    pts = x[..., None] + c * s
    return l_fn(pts).min(axis=-1)
