"""Python face of the FP64 CPU oracle (test infrastructure).

This package is the slow, obviously-correct reference the CUDA solver is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may import it; the product library never does.  It
shares no code with the CUDA path: the problem description arrives as a plain
dict (see ``workloads``) and each side builds its own native struct from it.

Functions follow arXiv:1903.07715: the dynamics of Sec. II-A Eq. (1), the
Hamiltonian of Eq. (6), the HJI variational inequality of Eq. (7) marched
backwards in time with min(., l) after every step (Eq. (8)), standard or warm
initialisation (Sec. II-B, Sec. III), and the max-change convergence test
(Sec. IV), and the discounted variant of Sec. II-C.  Parity status of each
function is listed in ``PINS`` below.
"""
import ctypes
import os

import numpy as np

from . import build as _build

MAXD, MAXU, MAXT = 4, 4, 8
SCHEMES = {"eno1": 1, "eno2": 2, "weno5": 5}
FNS = {"tan": 0, "sin": 1, "cos": 2}

# What pins each oracle function (tests/test_oracle_*.py):
PINS = {
    "one_sided": "exact on polynomials of the scheme's degree; convergence order on smooth data; "
                 "WENO5 and ENO2 rebuilt from their definitions (interpolant derivatives, "
                 "solved ideal weights, Jiang-Shu integral indicators) on rough data",
    "gradient / ghost nodes": "the averaged one-sided derivatives at every node, ghosts built "
                              "from their definition (extrapolation, wrap)",
    "dynamics": "the paper's model equations; sin / cos / tan terms against numpy",
    "hamiltonian": "brute-force max-min over dense samples of U x D",
    "alpha_dt": "hand-computed values for the double integrator and quadrotor; brute force",
    "control_at / optimal_control": "brute-force argmax-min over dense samples of U x D; "
                                    "the double integrator's closed-form braking control; "
                                    "bang-bang control at a known gradient; the tie reading",
    "step/solve": "closed-form double-integrator value (Sec. II-B cost, Eq. (3)-(4)); "
                  "1-D advection closed form; stationary case; refinement order; "
                  "Thm. 1 / Lemma 1 / Thm. 2 / Props. 1-2 / Remarks 1-2 orderings; "
                  "BRS option: advection closed form, a given start kept as it is",
    "step/solve, discounted": "closed form of the discounted one-cell shift (Courant number 1, "
                              "periodic); contraction from two starts (Sec. II-C); "
                              "gamma 0 or 1 equals the plain march",
}


class _Problem(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("n", ctypes.c_int64 * MAXD),
        ("lo", ctypes.c_double * MAXD),
        ("hi", ctypes.c_double * MAXD),
        ("periodic", ctypes.c_int * MAXD),
        ("m", ctypes.c_int),
        ("q", ctypes.c_int),
        ("nterms", ctypes.c_int),
        ("c", ctypes.c_double * MAXD),
        ("A", ctypes.c_double * (MAXD * MAXD)),
        ("G", ctypes.c_double * (MAXD * MAXU)),
        ("E", ctypes.c_double * (MAXD * MAXU)),
        ("term_row", ctypes.c_int * MAXT),
        ("term_axis", ctypes.c_int * MAXT),
        ("term_fn", ctypes.c_int * MAXT),
        ("term_w", ctypes.c_double * MAXT),
        ("ulo", ctypes.c_double * MAXU),
        ("uhi", ctypes.c_double * MAXU),
        ("dlo", ctypes.c_double * MAXU),
        ("dhi", ctypes.c_double * MAXU),
    ]


class _Stats(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_int64),
        ("tau", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("last_delta", ctypes.c_double),
        ("converged", ctypes.c_int),
        ("alpha", ctypes.c_double * MAXD),
    ]


_lib = None
_P = ctypes.POINTER(_Problem)
_D = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.oracle_spacing.restype = ctypes.c_double
        lib.oracle_spacing.argtypes = [_P, ctypes.c_int]
        lib.oracle_node.restype = ctypes.c_double
        lib.oracle_node.argtypes = [_P, ctypes.c_int, ctypes.c_int64]
        lib.oracle_dynamics.argtypes = [_P, _D, _D, _D, _D]
        lib.oracle_hamiltonian.restype = ctypes.c_double
        lib.oracle_hamiltonian.argtypes = [_P, _D, _D]
        lib.oracle_alpha_point.argtypes = [_P, _D, _D]
        lib.oracle_alpha_dt.argtypes = [_P, ctypes.c_double, _D, _D]
        lib.oracle_one_sided.argtypes = [ctypes.c_int, _D, ctypes.c_double, _D, _D]
        lib.oracle_operator.argtypes = [_P, ctypes.c_int, _D, _D, _D]
        lib.oracle_step.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D,
                                    _D, _D, _D, ctypes.c_int, ctypes.c_double]
        lib.oracle_init.argtypes = [_P, _D, _D, _D]
        lib.oracle_solve.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int64, _D, _D,
                                     _D, ctypes.POINTER(_Stats), _D, ctypes.c_int64,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_double]
        lib.oracle_control_at.argtypes = [_P, _D, _D, _D, _D]
        lib.oracle_optimal_control.argtypes = [_P, ctypes.c_int, _D, _D, _D]
        lib.oracle_gradient.argtypes = [_P, ctypes.c_int, _D, _D]
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_ghost_width.argtypes = [ctypes.c_int]
        lib.oracle_ghost_width.restype = ctypes.c_int
        _lib = lib
    return _lib


def library_path():
    _load()
    return _build.LIB


def _ptr(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def problem(grid: dict, dyn: dict) -> _Problem:
    """Build the oracle's problem struct from a grid dict and a dynamics dict.

    grid: {"n": [...], "lo": [...], "hi": [...], "periodic": [...] (optional)}
    dyn:  {"c": n, "A": n x n, "G": n x m, "E": n x q, "ulo"/"uhi": m,
           "dlo"/"dhi": q, "terms": [(row, axis, fn, w), ...]}  (all optional
           but G/ulo/uhi; missing entries are zero / empty)."""
    P = _Problem()
    n = len(grid["n"])
    if not 1 <= n <= MAXD:
        raise ValueError("ndim out of range")
    P.ndim = n
    per = grid.get("periodic", [0] * n)
    for a in range(n):
        P.n[a] = int(grid["n"][a])
        P.lo[a] = float(grid["lo"][a])
        P.hi[a] = float(grid["hi"][a])
        P.periodic[a] = int(bool(per[a]))
    c = np.zeros(n) if dyn.get("c") is None else np.asarray(dyn["c"], float)
    A = np.zeros((n, n)) if dyn.get("A") is None else np.asarray(dyn["A"], float)
    G = np.zeros((n, 0)) if dyn.get("G") is None else np.asarray(dyn["G"], float).reshape(n, -1)
    E = np.zeros((n, 0)) if dyn.get("E") is None else np.asarray(dyn["E"], float).reshape(n, -1)
    m, q = G.shape[1], E.shape[1]
    if m > MAXU or q > MAXU:
        raise ValueError("too many inputs")
    P.m, P.q = m, q
    for i in range(n):
        P.c[i] = c[i]
        for j in range(n):
            P.A[i * MAXD + j] = A[i, j]
        for j in range(m):
            P.G[i * MAXU + j] = G[i, j]
        for k in range(q):
            P.E[i * MAXU + k] = E[i, k]
    ulo = np.asarray(dyn.get("ulo", []), float).reshape(-1)
    uhi = np.asarray(dyn.get("uhi", []), float).reshape(-1)
    dlo = np.asarray(dyn.get("dlo", []), float).reshape(-1)
    dhi = np.asarray(dyn.get("dhi", []), float).reshape(-1)
    for j in range(m):
        P.ulo[j], P.uhi[j] = ulo[j], uhi[j]
    for k in range(q):
        P.dlo[k], P.dhi[k] = dlo[k], dhi[k]
    terms = dyn.get("terms", [])
    if len(terms) > MAXT:
        raise ValueError("too many terms")
    P.nterms = len(terms)
    for t, (row, axis, fn, w) in enumerate(terms):
        P.term_row[t] = int(row)
        P.term_axis[t] = int(axis)
        P.term_fn[t] = FNS[fn] if isinstance(fn, str) else int(fn)
        P.term_w[t] = float(w)
    return P


def spacing(P, axis):
    return _load().oracle_spacing(ctypes.byref(P), axis)


def nodes(P, axis):
    lib = _load()
    return np.array([lib.oracle_node(ctypes.byref(P), axis, i) for i in range(P.n[axis])])


def dynamics(P, x, u, d):
    lib = _load()
    x, u, d = _f64(x), _f64(np.atleast_1d(u) if len(u) else np.zeros(1)), \
        _f64(np.atleast_1d(d) if len(d) else np.zeros(1))
    f = np.zeros(P.ndim)
    lib.oracle_dynamics(ctypes.byref(P), _ptr(x), _ptr(u), _ptr(d), _ptr(f))
    return f


def hamiltonian(P, x, p):
    x, p = _f64(x), _f64(p)
    return _load().oracle_hamiltonian(ctypes.byref(P), _ptr(x), _ptr(p))


def alpha_point(P, x):
    x = _f64(x)
    out = np.zeros(MAXD)
    _load().oracle_alpha_point(ctypes.byref(P), _ptr(x), _ptr(out))
    return out[: P.ndim]


def alpha_dt(P, cfl):
    alpha = np.zeros(MAXD)
    dt = ctypes.c_double(0.0)
    rc = _load().oracle_alpha_dt(ctypes.byref(P), float(cfl), _ptr(alpha), ctypes.byref(dt))
    if rc != 0:
        raise ValueError("dynamics vanish on the grid: no finite CFL step")
    return alpha[: P.ndim].copy(), dt.value


def ghost_width(scheme):
    return _load().oracle_ghost_width(SCHEMES[scheme])


def one_sided(scheme, line, dx):
    """(p-, p+) at the centre of a stencil line of 2g+1 values."""
    line = _f64(line)
    g = ghost_width(scheme)
    if line.shape != (2 * g + 1,):
        raise ValueError("stencil line must have %d values" % (2 * g + 1))
    pm, pp = ctypes.c_double(), ctypes.c_double()
    _load().oracle_one_sided(SCHEMES[scheme], _ptr(line), float(dx), ctypes.byref(pm),
                             ctypes.byref(pp))
    return pm.value, pp.value


def _alpha_arr(alpha):
    a = np.zeros(MAXD)
    a[: len(alpha)] = alpha
    return a


def operator(P, scheme, alpha, W):
    W = _f64(W)
    L = np.empty_like(W)
    a = _alpha_arr(alpha)
    _load().oracle_operator(ctypes.byref(P), SCHEMES[scheme], _ptr(a), _ptr(W), _ptr(L))
    return L


def init(P, l, k=None):
    l = _f64(l)
    V = np.empty_like(l)
    kk = None if k is None else _f64(k)
    _load().oracle_init(ctypes.byref(P), _ptr(l), None if kk is None else _ptr(kk), _ptr(V))
    return V


BRS, LOCAL_LF = 1, 2


def _flags(brs, local_lf):
    return (BRS if brs else 0) | (LOCAL_LF if local_lf else 0)


def step(P, scheme, rk, dt, alpha, l, V, brs=False, local_lf=False, discount=0.0):
    """One Runge-Kutta step + min(., l) (none with brs: Eq. (5) alone); with
    0 < discount < 1, min(l, discount * step) (Sec. II-C).
    Returns (V_next, max|dV|)."""
    l, V = _f64(l), _f64(V)
    out = np.empty_like(V)
    delta = ctypes.c_double()
    a = _alpha_arr(alpha)
    rc = _load().oracle_step(ctypes.byref(P), SCHEMES[scheme], int(rk), float(dt), _ptr(a),
                             _ptr(l), _ptr(V), _ptr(out), ctypes.byref(delta),
                             _flags(brs, local_lf), float(discount))
    if rc != 0:
        raise MemoryError("oracle_step")
    return out, delta.value


def solve(P, l, k=None, scheme="eno2", rk=2, cfl=0.5, tol=1e-6, horizon=0.0, max_steps=0,
          history=0, tol_rate=0.0, interval=0.0, interval_tol=0.0, brs=False, local_lf=False,
          discount=0.0):
    """March to convergence: max|dV| of one step < tol + tol_rate dt, or (with
    interval > 0) the change of V over K = round(interval / dt) steps below
    interval_tol (Sec. V); every step discounted by 0 < discount < 1
    (Sec. II-C).  Returns (V, stats dict[, history array])."""
    l = _f64(l)
    V = np.empty_like(l)
    kk = None if k is None else _f64(k)
    st = _Stats()
    hist = np.zeros(max(int(history), 1))
    rc = _load().oracle_solve(ctypes.byref(P), SCHEMES[scheme], int(rk), float(cfl), float(tol),
                              float(horizon), int(max_steps), _ptr(l),
                              None if kk is None else _ptr(kk), _ptr(V), ctypes.byref(st),
                              _ptr(hist), int(history), float(tol_rate), float(interval),
                              float(interval_tol), _flags(brs, local_lf), float(discount))
    if rc < 0:
        raise ValueError("oracle_solve rejected its input")
    stats = {"steps": st.steps, "tau": st.tau, "dt": st.dt, "last_delta": st.last_delta,
             "converged": bool(st.converged), "alpha": np.array(st.alpha[: P.ndim])}
    if history:
        return V, stats, hist[: min(int(history), st.steps)]
    return V, stats


def control_at(P, x, p):
    """Eq. (9) at one state for the gradient p: (u*, d*)."""
    x, p = _f64(x), _f64(p)
    u = np.zeros(MAXU)
    d = np.zeros(MAXU)
    _load().oracle_control_at(ctypes.byref(P), _ptr(x), _ptr(p), _ptr(u), _ptr(d))
    return u[: P.m].copy(), d[: P.q].copy()


def optimal_control(P, scheme, V):
    """Eq. (9) at every node of V: arrays u* of shape (m,) + V.shape and d*
    of shape (q,) + V.shape."""
    V = _f64(V)
    u = np.zeros((max(P.m, 1),) + V.shape)
    d = np.zeros((max(P.q, 1),) + V.shape)
    _load().oracle_optimal_control(ctypes.byref(P), SCHEMES[scheme], _ptr(V), _ptr(u), _ptr(d))
    return u[: P.m], d[: P.q]


def gradient(P, scheme, V):
    """(p- + p+)/2 at every node: shape (ndim,) + V.shape."""
    V = _f64(V)
    g = np.zeros((P.ndim,) + V.shape)
    _load().oracle_gradient(ctypes.byref(P), SCHEMES[scheme], _ptr(V), _ptr(g))
    return g


def max_threads():
    return _load().oracle_max_threads()


def set_threads(n):
    _load().oracle_set_threads(int(n))
