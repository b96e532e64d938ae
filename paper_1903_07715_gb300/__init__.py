"""Python binding of the GB300 HJI reachability solver (include/hji.h).

Every step of the solve runs in the CUDA library ``_hji.so`` (built in-tree
by ``paper_1903_07715_gb300.build``).  This module only marshals arguments:
the functions ``hji_grid_create``, ``hji_dynamics_set``, ``hji_solve``,
``hji_batch_solve``, ``hji_value_get``, ... carry the C names and call them
through ctypes.  There is no CPU fallback: if the library is missing,
``load()`` raises.

PyTorch is used for device memory and streams only: ``torch_allocator()``
routes the library's device allocations through torch's caching allocator,
and the ``Grid`` convenience class accepts numpy arrays (host) or CUDA
tensors (device) and runs on torch's current stream.
"""
import ctypes
import os

import numpy as np

from . import build as _build

HJI_MAX_DIM, HJI_MAX_INPUTS, HJI_MAX_TERMS = 4, 4, 8
HJI_TILE_VARIANTS = 3

HJI_OK, HJI_E_INVALID, HJI_E_NOMEM, HJI_E_CUDA = 0, 1, 2, 3
HJI_E_NOT_CONVERGED, HJI_E_TIMEOUT, HJI_E_STATE, HJI_E_NONFINITE, HJI_E_CHECK = 4, 5, 6, 7, 8
HJI_F64, HJI_F32 = 0, 1
HJI_ENO1, HJI_ENO2, HJI_WENO5 = 1, 2, 5
HJI_INIT_STANDARD, HJI_INIT_USER_K, HJI_INIT_RESIDENT = 0, 1, 2
HJI_FN = {"tan": 0, "sin": 1, "cos": 2}
SCHEMES = {"eno1": HJI_ENO1, "eno2": HJI_ENO2, "weno5": HJI_WENO5}

EXPORTS = ["hji_grid_create", "hji_grid_destroy", "hji_dynamics_set", "hji_solve",
           "hji_batch_solve", "hji_value_get", "hji_value_transfer", "hji_grid_info",
           "hji_status_string", "hji_last_error", "hji_solve_noalloc", "hji_noalloc_last_error",
           "hji_engine_create", "hji_engine_submit", "hji_engine_step", "hji_engine_poll",
           "hji_engine_destroy", "hji_engine_last_error", "hji_autotune",
           "hji_stage_times", "hji_selftest_bounded_wait", "hji_peak_fma",
           "hji_peak_last_error", "hji_optimal_control", "hji_selftest_index_check"]

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class hji_allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", ctypes.c_void_p)]


class hji_dynamics(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("q", ctypes.c_int), ("nterms", ctypes.c_int),
                ("c", ctypes.POINTER(ctypes.c_double)), ("A", ctypes.POINTER(ctypes.c_double)),
                ("G", ctypes.POINTER(ctypes.c_double)), ("E", ctypes.POINTER(ctypes.c_double)),
                ("term_row", ctypes.POINTER(ctypes.c_int)),
                ("term_axis", ctypes.POINTER(ctypes.c_int)),
                ("term_fn", ctypes.POINTER(ctypes.c_int)),
                ("term_w", ctypes.POINTER(ctypes.c_double)),
                ("ulo", ctypes.POINTER(ctypes.c_double)), ("uhi", ctypes.POINTER(ctypes.c_double)),
                ("dlo", ctypes.POINTER(ctypes.c_double)), ("dhi", ctypes.POINTER(ctypes.c_double))]


class hji_solve_opts(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int), ("rk_order", ctypes.c_int), ("cfl", ctypes.c_double),
                ("tol", ctypes.c_double), ("horizon", ctypes.c_double),
                ("check_every", ctypes.c_int), ("max_steps", ctypes.c_int64),
                ("init", ctypes.c_int), ("tile_variant", ctypes.c_int),
                ("tol_rate", ctypes.c_double), ("march", ctypes.c_int),
                ("interval", ctypes.c_double), ("interval_tol", ctypes.c_double),
                ("brs", ctypes.c_int), ("local_lf", ctypes.c_int),
                ("discount", ctypes.c_double)]


class hji_solve_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("tau", ctypes.c_double), ("dt", ctypes.c_double),
                ("final_max_dV", ctypes.c_double), ("wall_ms", ctypes.c_double),
                ("alpha", ctypes.c_double * HJI_MAX_DIM), ("converged", ctypes.c_int),
                ("kernel_launches", ctypes.c_int64)]


_lib = None


def library_path():
    """_hji.so, or the bounds-checked debug build _hji_checked.so when the
    environment variable HJI_CHECKED_BUILD is "1"."""
    return _build.CHECKED_LIB if os.environ.get("HJI_CHECKED_BUILD") == "1" else _build.LIB


def load(build_if_missing=False):
    """Load the library (library_path()).  Raises if it is missing (no
    fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build(checked=path == _build.CHECKED_LIB)
        else:
            raise RuntimeError("CUDA library %s is missing: run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    lib = ctypes.CDLL(path)
    vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.hji_grid_create.argtypes = [ctypes.c_int, i64p, dp, dp, ctypes.POINTER(ctypes.c_int),
                                    ctypes.c_int, ctypes.POINTER(hji_allocator),
                                    ctypes.POINTER(vp)]
    lib.hji_grid_destroy.argtypes = [vp]
    lib.hji_dynamics_set.argtypes = [vp, ctypes.POINTER(hji_dynamics)]
    lib.hji_solve.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.POINTER(hji_solve_opts), vp,
                              ctypes.POINTER(hji_solve_stats)]
    lib.hji_batch_solve.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                    ctypes.POINTER(vp), ctypes.c_int,
                                    ctypes.POINTER(hji_solve_opts), vp,
                                    ctypes.POINTER(hji_solve_stats)]
    lib.hji_value_get.argtypes = [vp, vp, ctypes.c_int, vp]
    lib.hji_value_transfer.argtypes = [vp, vp, vp]
    lib.hji_grid_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), i64p, i64p]
    lib.hji_status_string.argtypes = [ctypes.c_int]
    lib.hji_status_string.restype = ctypes.c_char_p
    lib.hji_last_error.argtypes = [vp]
    lib.hji_last_error.restype = ctypes.c_char_p
    lib.hji_solve_noalloc.argtypes = [ctypes.c_int, i64p, dp, dp, ctypes.POINTER(ctypes.c_int),
                                      ctypes.c_int, ctypes.POINTER(hji_dynamics), vp, vp, vp,
                                      ctypes.POINTER(hji_solve_opts), vp,
                                      ctypes.POINTER(hji_solve_stats)]
    lib.hji_noalloc_last_error.argtypes = []
    lib.hji_noalloc_last_error.restype = ctypes.c_char_p
    ip = ctypes.POINTER(ctypes.c_int)
    lib.hji_engine_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(hji_solve_opts),
                                      ctypes.c_int, ctypes.c_size_t, vp,
                                      ctypes.POINTER(hji_allocator), ctypes.POINTER(vp)]
    lib.hji_engine_submit.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64]
    lib.hji_engine_step.argtypes = [vp, ip, ip]
    lib.hji_engine_poll.argtypes = [vp, i64p, ctypes.POINTER(hji_solve_stats), ip, ctypes.c_int, ip]
    lib.hji_engine_destroy.argtypes = [vp]
    lib.hji_autotune.argtypes = [vp, vp, ctypes.c_int, ctypes.POINTER(hji_solve_opts),
                                 ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_double)]
    lib.hji_engine_last_error.argtypes = [vp]
    lib.hji_engine_last_error.restype = ctypes.c_char_p
    lib.hji_selftest_bounded_wait.argtypes = [ctypes.c_int64, vp]
    lib.hji_selftest_index_check.argtypes = [vp, ip, ip, ip, i64p, i64p]
    lib.hji_stage_times.argtypes = [vp, vp, ctypes.c_int, ctypes.POINTER(hji_solve_opts),
                                    ctypes.c_int, vp, ctypes.POINTER(ctypes.c_double)]
    lib.hji_peak_fma.argtypes = [ctypes.c_int, ctypes.c_double, vp, dp, dp]
    lib.hji_optimal_control.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int, vp]
    lib.hji_peak_last_error.argtypes = []
    lib.hji_peak_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("hji_status_string", "hji_last_error", "hji_noalloc_last_error",
                        "hji_engine_last_error", "hji_peak_last_error"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


# ---- the C entry points under their own names (marshalling only) ----

def hji_grid_create(ndim, n, lo, hi, periodic, prec, alloc, out):
    return load().hji_grid_create(ndim, n, lo, hi, periodic, prec, alloc, out)


def hji_grid_destroy(g):
    return load().hji_grid_destroy(g)


def hji_dynamics_set(g, dyn):
    return load().hji_dynamics_set(g, dyn)


def hji_solve(g, l, k, ptr_is_device, opts, stream, stats):
    return load().hji_solve(g, l, k, ptr_is_device, opts, stream, stats)


def hji_batch_solve(count, grids, l, k, ptr_is_device, opts, stream, stats):
    return load().hji_batch_solve(count, grids, l, k, ptr_is_device, opts, stream, stats)


def hji_value_get(g, out, ptr_is_device, stream):
    return load().hji_value_get(g, out, ptr_is_device, stream)


def hji_value_transfer(dst, src, stream):
    return load().hji_value_transfer(dst, src, stream)


def hji_grid_info(g, ndim, n, num_nodes):
    return load().hji_grid_info(g, ndim, n, num_nodes)


def hji_selftest_bounded_wait(limit_ns, stream):
    return load().hji_selftest_bounded_wait(limit_ns, stream)


def hji_selftest_index_check(stream, checked, count, site, index, extent):
    return load().hji_selftest_index_check(stream, checked, count, site, index, extent)


def hji_solve_noalloc(ndim, n, lo, hi, periodic, prec, dyn, l, k, v_out, opts, stream, stats):
    return load().hji_solve_noalloc(ndim, n, lo, hi, periodic, prec, dyn, l, k, v_out, opts,
                                    stream, stats)


def hji_noalloc_last_error():
    return load().hji_noalloc_last_error().decode()


def hji_autotune(g, l, ptr_is_device, opts, steps, stream, chosen, ms_per_step):
    return load().hji_autotune(g, l, ptr_is_device, opts, steps, stream, chosen, ms_per_step)


def hji_stage_times(g, l, ptr_is_device, opts, steps, stream, ms_per_stage):
    return load().hji_stage_times(g, l, ptr_is_device, opts, steps, stream, ms_per_stage)


def hji_optimal_control(g, scheme, u_out, d_out, ptr_is_device, stream):
    return load().hji_optimal_control(g, scheme, u_out, d_out, ptr_is_device, stream)


def hji_peak_fma(prec, target_ms, stream, tflops, ms_per_launch):
    return load().hji_peak_fma(prec, target_ms, stream, tflops, ms_per_launch)


def hji_peak_last_error():
    return load().hji_peak_last_error().decode()


def peak_fma(precision="f32", target_ms=20.0, stream=None):
    """Measured FMA rate of the current GPU (TFLOP/s, one FMA = 2 flops) and
    the duration of the fastest timed launch (ms)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    st = None if stream is None else ctypes.c_void_p(stream)
    rc = hji_peak_fma(HJI_F32 if precision == "f32" else HJI_F64, float(target_ms), st,
                      ctypes.byref(tf), ctypes.byref(ms))
    if rc != HJI_OK:
        raise HJIError(rc, hji_peak_last_error())
    return tf.value, ms.value


def hji_engine_create(ndim, prec, opts, max_slots, budget_bytes, stream, alloc, out):
    return load().hji_engine_create(ndim, prec, opts, max_slots, budget_bytes, stream, alloc, out)


def hji_engine_submit(e, g, l, k, ptr_is_device, init, tag):
    return load().hji_engine_submit(e, g, l, k, ptr_is_device, init, tag)


def hji_engine_step(e, active, queued):
    return load().hji_engine_step(e, active, queued)


def hji_engine_poll(e, tags, stats, status, cap, count):
    return load().hji_engine_poll(e, tags, stats, status, cap, count)


def hji_engine_destroy(e):
    return load().hji_engine_destroy(e)


def hji_engine_last_error(e):
    return load().hji_engine_last_error(e).decode()


def hji_status_string(s):
    return load().hji_status_string(s).decode()


def hji_last_error(g):
    return load().hji_last_error(g).decode()


class HJIError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (hji_status_string(status), msg))
        self.status = status


# ---- convenience layer: numpy / torch in, the same C calls underneath ----

_TORCH_ALLOC = None


def torch_allocator():
    """An hji_allocator drawing device memory from torch's caching allocator."""
    global _TORCH_ALLOC
    if _TORCH_ALLOC is None:
        import torch

        def _alloc(nbytes, stream, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
            except Exception:  # out of memory: report NULL to the library
                return None

        def _free(ptr, stream, ctx):
            torch.cuda.caching_allocator_delete(int(ptr))

        fa, ff = _ALLOC_FN(_alloc), _FREE_FN(_free)
        _TORCH_ALLOC = (hji_allocator(fa, ff, None), fa, ff)
    return _TORCH_ALLOC[0]


def _darr(vals, n=None):
    a = (ctypes.c_double * max(1, len(vals) if n is None else n))()
    for i, v in enumerate(vals):
        a[i] = float(v)
    return a


def _iarr(vals):
    a = (ctypes.c_int * max(1, len(vals)))()
    for i, v in enumerate(vals):
        a[i] = int(v)
    return a


def dynamics_struct(dyn, ndim):
    """hji_dynamics from a plain dict (the same dict the workloads produce).
    Returns (struct, keepalive)."""
    n = ndim
    c = np.zeros(n) if dyn.get("c") is None else np.asarray(dyn["c"], float).reshape(n)
    A = np.zeros((n, n)) if dyn.get("A") is None else np.asarray(dyn["A"], float).reshape(n, n)
    G = np.zeros((n, 0)) if dyn.get("G") is None else np.asarray(dyn["G"], float).reshape(n, -1)
    E = np.zeros((n, 0)) if dyn.get("E") is None else np.asarray(dyn["E"], float).reshape(n, -1)
    terms = dyn.get("terms", [])
    keep = [_darr(c), _darr(A.ravel()), _darr(G.ravel()), _darr(E.ravel()),
            _iarr([t[0] for t in terms]), _iarr([t[1] for t in terms]),
            _iarr([HJI_FN[t[2]] if isinstance(t[2], str) else t[2] for t in terms]),
            _darr([t[3] for t in terms]),
            _darr(np.asarray(dyn.get("ulo", []), float).ravel()),
            _darr(np.asarray(dyn.get("uhi", []), float).ravel()),
            _darr(np.asarray(dyn.get("dlo", []), float).ravel()),
            _darr(np.asarray(dyn.get("dhi", []), float).ravel())]
    s = hji_dynamics(G.shape[1], E.shape[1], len(terms), *keep)
    return s, keep


def _check(status, g=None):
    if status != HJI_OK:
        raise HJIError(status, hji_last_error(g))


def _stats_dict(st):
    return {"steps": int(st.steps), "tau": st.tau, "dt": st.dt, "last_delta": st.final_max_dV,
            "wall_ms": st.wall_ms, "alpha": list(st.alpha), "converged": bool(st.converged),
            "kernel_launches": int(st.kernel_launches)}


MARCH = {"auto": 0, "per_stage": 1, "multi_step": 2}


def solve_opts(scheme="eno2", rk=2, cfl=0.5, tol=1e-6, horizon=0.0, max_steps=0,
               check_every=32, init=HJI_INIT_STANDARD, tile_variant=0, tol_rate=0.0,
               march="auto", interval=0.0, interval_tol=0.0, brs=False, local_lf=False,
               discount=0.0):
    return hji_solve_opts(SCHEMES[scheme] if isinstance(scheme, str) else scheme, rk, cfl, tol,
                          horizon, check_every, max_steps, init, tile_variant, tol_rate,
                          MARCH[march] if isinstance(march, str) else march, interval,
                          interval_tol, int(brs), int(local_lf), float(discount))


class Grid:
    """One grid handle.  `gd` is a grid dict ({"n","lo","hi","periodic"});
    precision "f64" or "f32"; allocator: "torch" (default), "cuda" or None
    (the library's own cudaMallocAsync), or an hji_allocator structure (kept
    alive by the caller for the grid's lifetime)."""

    def __init__(self, gd, precision="f64", allocator="torch"):
        self._h = ctypes.c_void_p()
        nd = len(gd["n"])
        self.ndim = nd
        self.shape = tuple(int(v) for v in gd["n"])
        self.dtype = np.float64 if precision == "f64" else np.float32
        self.prec = HJI_F64 if precision == "f64" else HJI_F32
        n = (ctypes.c_int64 * nd)(*self.shape)
        per = _iarr(gd.get("periodic", [0] * nd))
        if isinstance(allocator, hji_allocator):
            alloc = allocator
        else:
            alloc = torch_allocator() if allocator == "torch" else None
        _check(hji_grid_create(nd, n, _darr(gd["lo"]), _darr(gd["hi"]), per, self.prec,
                               ctypes.byref(alloc) if alloc is not None else None,
                               ctypes.byref(self._h)))
        self._keep = None

    @property
    def handle(self):
        return self._h

    def set_dynamics(self, dyn):
        s, keep = dynamics_struct(dyn, self.ndim)
        _check(hji_dynamics_set(self._h, ctypes.byref(s)), self._h)
        self._mq = (s.m, s.q)

    def optimal_control(self, scheme="eno2", stream=None):
        """Eq. (9) at every node of the current value: numpy arrays u* of
        shape (m,) + grid shape and d* of shape (q,) + grid shape."""
        m, q = self._mq
        u = np.zeros((max(m, 1),) + self.shape, dtype=self.dtype)
        d = np.zeros((max(q, 1),) + self.shape, dtype=self.dtype)
        _check(hji_optimal_control(self._h, SCHEMES[scheme], u.ctypes.data,
                                   d.ctypes.data if q else None, 0, self._stream(stream)),
               self._h)
        return u[:m], d[:q]

    def _ptr(self, a):
        """(pointer, is_device, keepalive) for a numpy array or CUDA tensor."""
        if a is None:
            return None, 0, None
        if isinstance(a, np.ndarray):
            a = np.ascontiguousarray(a, dtype=self.dtype)
            if a.shape != self.shape:
                raise ValueError("array shape %s != grid %s" % (a.shape, self.shape))
            return a.ctypes.data, 0, a
        import torch
        if not (isinstance(a, torch.Tensor) and a.is_cuda):
            raise TypeError("expected a numpy array or a CUDA tensor")
        want = torch.float64 if self.prec == HJI_F64 else torch.float32
        if a.dtype != want or not a.is_contiguous() or tuple(a.shape) != self.shape:
            raise ValueError("CUDA tensor must be contiguous %s of shape %s" % (want, self.shape))
        return a.data_ptr(), 1, a

    @staticmethod
    def _stream(stream):
        if stream is not None:
            return ctypes.c_void_p(int(stream))
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None

    def solve(self, l, k=None, init=None, stream=None, raise_on_cap=False, **opts):
        lp, ldev, lkeep = self._ptr(l)
        kp, kdev, kkeep = self._ptr(k)
        if k is not None and kdev != ldev:
            raise ValueError("l and k must both be host or both be device arrays")
        if init is None:
            init = HJI_INIT_USER_K if k is not None else HJI_INIT_STANDARD
        o = solve_opts(init=init, **opts)
        st = hji_solve_stats()
        rc = hji_solve(self._h, lp, kp, ldev, ctypes.byref(o), self._stream(stream),
                       ctypes.byref(st))
        if rc not in (HJI_OK, HJI_E_NOT_CONVERGED) or (raise_on_cap and rc != HJI_OK):
            raise HJIError(rc, hji_last_error(self._h))
        return _stats_dict(st)

    def value(self, out=None, stream=None):
        if out is None:
            out = np.empty(self.shape, dtype=self.dtype)
        p, dev, keep = self._ptr(out)
        _check(hji_value_get(self._h, p, dev, self._stream(stream)), self._h)
        if isinstance(out, np.ndarray) and keep is not out:
            out[...] = keep
        return out

    def autotune(self, l, steps=20, stream=None, **opts):
        """hji_autotune: time each tile shape on this grid, remember the
        fastest for its class; returns (chosen, ms per step per variant)."""
        lp, ldev, keep = self._ptr(l)
        o = solve_opts(**opts)
        chosen = ctypes.c_int()
        ms = (ctypes.c_double * HJI_TILE_VARIANTS)()
        _check(hji_autotune(self._h, lp, ldev, ctypes.byref(o), int(steps), self._stream(stream),
                            ctypes.byref(chosen), ms), self._h)
        return chosen.value, list(ms)

    def stage_times(self, l, steps=20, stream=None, **opts):
        """hji_stage_times: march `steps` steps from V0 = l launching each RK
        stage kernel between two CUDA events; returns the mean kernel
        duration in ms of each stage (the last entry is the fused last
        stage)."""
        lp, ldev, keep = self._ptr(l)
        o = solve_opts(**opts)
        ms = (ctypes.c_double * 3)()
        _check(hji_stage_times(self._h, lp, ldev, ctypes.byref(o), int(steps), self._stream(stream), ms),
               self._h)
        return list(ms)[:o.rk_order]

    def take_value(self, other, stream=None):
        """Make `other`'s current value this grid's resident value (device-side
        precision conversion); follow with solve(..., init=HJI_INIT_RESIDENT)."""
        _check(hji_value_transfer(self._h, other.handle, self._stream(stream)), self._h)

    def close(self):
        if self._h:
            hji_grid_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_solve(grids, ls, ks=None, init=None, stream=None, **opts):
    """hji_batch_solve over Grid objects; returns a list of stats dicts."""
    count = len(grids)
    ptrs, keep, dev = [], [], None
    kps = []
    for i, g in enumerate(grids):
        p, d, kp_ = g._ptr(ls[i])
        keep.append(kp_)
        ptrs.append(p)
        dev = d if dev is None else dev
        if ks is not None and ks[i] is not None:
            kp, kd, kk = g._ptr(ks[i])
            keep.append(kk)
            kps.append(kp)
        else:
            kps.append(None)
    if init is None:
        init = HJI_INIT_USER_K if ks is not None else HJI_INIT_STANDARD
    o = solve_opts(init=init, **opts)
    stats = (hji_solve_stats * count)()
    ha = (ctypes.c_void_p * count)(*[g.handle.value for g in grids])
    la = (ctypes.c_void_p * count)(*ptrs)
    ka = (ctypes.c_void_p * count)(*kps)
    rc = hji_batch_solve(count, ha, la, ka, dev, ctypes.byref(o), Grid._stream(stream), stats)
    if rc not in (HJI_OK, HJI_E_NOT_CONVERGED):
        raise HJIError(rc, hji_last_error(grids[0].handle))
    return [_stats_dict(s) for s in stats], rc


class Engine:
    """Continuous-batching engine (hji_engine_*): requests are admitted into
    slots while others march; see include/hji.h."""

    def __init__(self, ndim, precision="f32", max_slots=64, budget_bytes=0, stream=None,
                 allocator="torch", **opts):
        self._h = ctypes.c_void_p()
        self.prec = HJI_F64 if precision == "f64" else HJI_F32
        o = solve_opts(**opts)
        if isinstance(allocator, hji_allocator):
            alloc = allocator
        else:
            alloc = torch_allocator() if allocator == "torch" else None
        rc = hji_engine_create(ndim, self.prec, ctypes.byref(o), max_slots, budget_bytes,
                               Grid._stream(stream),
                               ctypes.byref(alloc) if alloc is not None else None,
                               ctypes.byref(self._h))
        if rc != HJI_OK:
            raise HJIError(rc, hji_engine_last_error(None))
        self._keep = {}

    def submit(self, grid, l, k=None, init=None, tag=0):
        lp, ldev, lk = grid._ptr(l)
        kp, kdev, kk = grid._ptr(k)
        if init is None:
            init = HJI_INIT_USER_K if k is not None else HJI_INIT_STANDARD
        rc = hji_engine_submit(self._h, grid.handle, lp, kp, ldev, init, int(tag))
        if rc != HJI_OK:
            raise HJIError(rc, hji_engine_last_error(self._h))
        self._keep[int(tag)] = (lk, kk)

    def step(self):
        a, q = ctypes.c_int(), ctypes.c_int()
        rc = hji_engine_step(self._h, ctypes.byref(a), ctypes.byref(q))
        if rc != HJI_OK:
            raise HJIError(rc, hji_engine_last_error(self._h))
        return a.value, q.value

    def poll(self, cap=256):
        tags = (ctypes.c_int64 * cap)()
        stats = (hji_solve_stats * cap)()
        status = (ctypes.c_int * cap)()
        n = ctypes.c_int()
        rc = hji_engine_poll(self._h, tags, stats, status, cap, ctypes.byref(n))
        if rc != HJI_OK:
            raise HJIError(rc, hji_engine_last_error(self._h))
        out = []
        for i in range(n.value):
            self._keep.pop(int(tags[i]), None)
            out.append((int(tags[i]), _stats_dict(stats[i]), int(status[i])))
        return out

    def drain(self):
        done = []
        while True:
            a, q = self.step()
            done += self.poll()
            if a == 0 and q == 0:
                return done + self.poll()

    def close(self):
        if self._h:
            hji_engine_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
