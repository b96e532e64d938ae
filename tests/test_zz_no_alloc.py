"""hji_solve_noalloc: the allocation-free solve for callers that may not
allocate device memory (their device memory belongs to a host framework, or
they run where allocator calls are forbidden).  It keeps its scratch in one
static device array, so two calls in a row must each give what the
allocating entry point hji_solve gives for the same problem, and a grid too
large for the array must be refused before any device work.

Both arms march with the same tile shape and the same launch form: the
allocating solve is given tile_variant=1 (shape 0, the one hji_solve_noalloc
takes by default) and march="per_stage" (hji_solve_noalloc launches one
kernel per RK stage), so the comparison rests neither on an autotuned choice
made earlier in the session nor on how the compiler fused the multi-step
kernel's multiply-adds.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the FP64 per-step parity tolerance used by the other GPU tests


def _grid_args(gd):
    nd = len(gd["n"])
    n = (ctypes.c_int64 * nd)(*gd["n"])
    lo = (ctypes.c_double * nd)(*gd["lo"])
    hi = (ctypes.c_double * nd)(*gd["hi"])
    per = (ctypes.c_int * nd)(*gd["periodic"])
    return nd, n, lo, hi, per


def _noalloc(hji, torch, gd, dyn, l, k, prec, resident=None, **opts):
    """One hji_solve_noalloc call; `resident` (optional) is the previous value
    placed in v_out for an HJI_INIT_RESIDENT start."""
    nd, n, lo, hi, per = _grid_args(gd)
    tdt = torch.float64 if prec == "f64" else torch.float32
    lt = torch.as_tensor(l, dtype=tdt, device="cuda").contiguous()
    kt = None if k is None else torch.as_tensor(k, dtype=tdt, device="cuda").contiguous()
    if resident is not None:
        out = torch.as_tensor(resident, dtype=tdt, device="cuda").contiguous().clone()
        init = hji.HJI_INIT_RESIDENT
    else:
        out = torch.empty_like(lt)
        init = hji.HJI_INIT_USER_K if k is not None else hji.HJI_INIT_STANDARD
    dstruct, keep = hji.dynamics_struct(dyn, nd)
    o = hji.solve_opts(init=init, **opts)
    st = hji.hji_solve_stats()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = hji.hji_solve_noalloc(nd, n, lo, hi, per, hji.HJI_F64 if prec == "f64" else hji.HJI_F32,
                               ctypes.byref(dstruct), lt.data_ptr(),
                               None if kt is None else kt.data_ptr(), out.data_ptr(),
                               ctypes.byref(o), stream, ctypes.byref(st))
    torch.cuda.synchronize()
    return rc, out.cpu().numpy(), st


def _allocating(hji, gd, dyn, l, k, prec, **opts):
    g = hji.Grid(gd, prec)
    g.set_dynamics(dyn)
    st = g.solve(l, k, tile_variant=1, march="per_stage", **opts)
    V = g.value()
    g.close()
    return V, st


def test_noalloc_matches_hji_solve_two_calls_in_a_row(hji_lib):
    import torch
    assert torch.cuda.is_available()
    hji = hji_lib
    # Call 1: FP64, ENO2/RK2, standard start (the 101^2 double integrator).
    gd, dyn, l = W.di_config(101)
    opts = dict(scheme="eno2", rk=2, cfl=0.5, tol=1e-6, max_steps=20000)
    rc1, V1, s1 = _noalloc(hji, torch, gd, dyn, l, None, "f64", **opts)
    assert rc1 == hji.HJI_OK, hji.hji_noalloc_last_error()
    R1, r1 = _allocating(hji, gd, dyn, l, None, "f64", **opts)
    assert s1.steps == r1["steps"]
    assert np.abs(V1 - R1).max() <= TOL
    # Call 2 reuses the same scratch with another layout: FP32, WENO5/RK3,
    # a warm start from call 1's value on a disturbed problem.
    _, dyn2, _ = W.di_config(101, dmax=0.2)
    k = V1.astype(np.float32)
    l32 = l.astype(np.float32)
    opts2 = dict(scheme="weno5", rk=3, cfl=0.5, tol=1e-6, max_steps=20000)
    rc2, V2, s2 = _noalloc(hji, torch, gd, dyn2, l32, k, "f32", **opts2)
    assert rc2 == hji.HJI_OK, hji.hji_noalloc_last_error()
    R2, r2 = _allocating(hji, gd, dyn2, l32, k, "f32", **opts2)
    assert s2.steps == r2["steps"]
    assert np.abs(V2.astype(np.float64) - R2.astype(np.float64)).max() <= TOL


def test_noalloc_refuses_grids_beyond_its_scratch(hji_lib):
    import torch
    hji = hji_lib
    gd, dyn, _ = W.di_config(3001)  # 9 M nodes x 3 FP64 fields > 32 MiB
    l = torch.zeros((3001, 3001), dtype=torch.float64, device="cuda")
    nd, n, lo, hi, per = _grid_args(gd)
    dstruct, keep = hji.dynamics_struct(dyn, nd)
    o = hji.solve_opts(scheme="eno2", rk=2)
    rc = hji.hji_solve_noalloc(nd, n, lo, hi, per, hji.HJI_F64, ctypes.byref(dstruct),
                               l.data_ptr(), None, l.data_ptr(), ctypes.byref(o), None, None)
    assert rc == hji.HJI_E_INVALID
    assert "scratch" in hji.hji_noalloc_last_error()


def test_noalloc_4d_and_resident_start_match_hji_solve(hji_lib):
    """A 4-D grid (21^4 quadrotor subsystem, FP32, ENO2/RK2: the N-D tensor
    maps and strides of the scratch layout) and then an HJI_INIT_RESIDENT
    call that starts from the value left in v_out.  An FP32 resident start
    through hji_solve_noalloc begins from the float values alone, which is
    what hji_solve does for a user warm start k holding those floats."""
    import torch
    assert torch.cuda.is_available()
    hji = hji_lib
    gd, dyn, l = W.quad4d_config(21, dmax=0.1)
    l32 = l.astype(np.float32)
    opts = dict(scheme="eno2", rk=2, cfl=0.5, tol=0.0, max_steps=40)
    rc, V1, s1 = _noalloc(hji, torch, gd, dyn, l32, None, "f32", **opts)
    assert rc == hji.HJI_OK or rc == hji.HJI_E_NOT_CONVERGED, hji.hji_noalloc_last_error()
    R1, r1 = _allocating(hji, gd, dyn, l32, None, "f32", **opts)
    assert s1.steps == r1["steps"] == 40
    assert np.abs(V1.astype(np.float64) - R1.astype(np.float64)).max() <= TOL
    _, dyn2, _ = W.quad4d_config(21, dmax=0.2)
    rc2, V2, s2 = _noalloc(hji, torch, gd, dyn2, l32, None, "f32", resident=V1, **opts)
    assert rc2 == hji.HJI_OK or rc2 == hji.HJI_E_NOT_CONVERGED, hji.hji_noalloc_last_error()
    R2, r2 = _allocating(hji, gd, dyn2, l32, V1, "f32", **opts)
    assert s2.steps == r2["steps"] == 40
    assert np.abs(V2.astype(np.float64) - R2.astype(np.float64)).max() <= TOL


def test_noalloc_rejects_bad_options_before_device_work(hji_lib):
    import torch
    hji = hji_lib
    gd, dyn, l = W.di_config(21)
    lt = torch.as_tensor(l, device="cuda")
    nd, n, lo, hi, per = _grid_args(gd)
    dstruct, keep = hji.dynamics_struct(dyn, nd)
    for bad in (dict(tol_rate=-1.0), dict(tol_rate=float("nan")), dict(tile_variant=7)):
        o = hji.solve_opts(scheme="eno2", rk=2, **bad)
        rc = hji.hji_solve_noalloc(nd, n, lo, hi, per, hji.HJI_F64, ctypes.byref(dstruct),
                                   lt.data_ptr(), None, lt.data_ptr(), ctypes.byref(o), None, None)
        assert rc == hji.HJI_E_INVALID, bad
