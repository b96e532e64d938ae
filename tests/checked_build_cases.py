"""Cases for the bounds-checked debug build (_hji_checked.so), run in a child
process by tests/test_gpu_checked_build.py with HJI_CHECKED_BUILD=1 so that
the binding loads that library.  Every index the stage kernels' tile and
halo code forms is checked there; a failed check makes the solve return
HJI_E_CHECK.  The cases are the grids where that code has the most edge
logic: minimal grids (n = 2g + 1 on every axis), grids of 5-9 nodes per
axis, periodic axes, ragged multi-tile 2-D grids in every tile shape,
1-D to 4-D, every scheme and precision, both launch forms, each march
option, a batch of uneven grids, the serving engine and the allocation-free
entry point.  Each result is also compared with the FP64 oracle (FP64:
1e-10; FP32 compensated: 1e-5 max|l|) after the same number of steps.

Prints one JSON line per case and a summary line; exits 0 when every case
ran.  Not collected by pytest (no test_ prefix)."""
import json
import os
import sys
import traceback

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as orc  # noqa: E402
import paper_1903_07715_gb300 as hji  # noqa: E402
import workloads as W  # noqa: E402

SCHEMES = [("eno1", 1), ("eno2", 2), ("weno5", 3)]
GHOST = {"eno1": 1, "eno2": 2, "weno5": 3}


def _dyn(nd, rng):
    """Control-affine dynamics with a linear part, a nonlinear term, two
    inputs and a disturbance (every part of the stage kernel's Hamiltonian)."""
    dyn = {"A": rng.normal(size=(nd, nd)) * 0.4, "c": rng.normal(size=nd) * 0.2,
           "G": rng.normal(size=(nd, 2)), "ulo": [-1.0, -0.5], "uhi": [0.8, 0.6],
           "E": rng.normal(size=(nd, 1)) * 0.3, "dlo": [-0.2], "dhi": [0.3],
           "terms": [(nd - 1, 0, "sin", 0.5)]}
    if nd >= 2:
        dyn["terms"].append((0, nd - 1, "cos", 0.3))
    return dyn


def _target(gd):
    X = W.mesh(gd)
    if not isinstance(X, (list, tuple)):
        X = [X]
    r = np.sqrt(sum((x * (1.0 + 0.1 * a)) ** 2 for a, x in enumerate(X)))
    return r - 0.6


def _compare(name, gd, dyn, l, prec, steps=3, k=None, **opts):
    """One solve of `steps` steps on the checked library against the oracle."""
    dt = np.float64 if prec == "f64" else np.float32
    g = hji.Grid(gd, prec)
    try:
        g.set_dynamics(dyn)
        st = g.solve(l.astype(dt), None if k is None else k.astype(dt), tol=0.0,
                     max_steps=steps, **opts)
        V = g.value().astype(np.float64)
    finally:
        g.close()
    oopts = {key: v for key, v in opts.items() if key not in ("march", "tile_variant",
                                                             "check_every")}
    Vo, so = orc.solve(orc.problem(gd, dyn), l, k=k, tol=0.0, max_steps=steps, **oopts)
    err = float(np.abs(V - Vo).max())
    tol = 1e-10 if prec == "f64" else 1e-5 * max(1.0, float(np.abs(l).max()))
    return {"case": name, "prec": prec, "steps": [st["steps"], so["steps"]], "err": err,
            "tol": tol, "ok": st["steps"] == so["steps"] and err <= tol}


def grid_cases():
    rng = np.random.Generator(np.random.PCG64(2024))
    for prec in ("f64", "f32"):
        for nd in (1, 2, 3, 4):
            dyn = _dyn(nd, rng)
            for scheme, rk in SCHEMES:
                g = GHOST[scheme]
                shapes = [("minimal", [2 * g + 1] * nd, [0] * nd),
                          ("small", [max(2 * g + 1, v) for v in (9, 7, 8, 9)[:nd]], [0] * nd),
                          ("periodic", [max(2 * g + 1, v) for v in (8, 9, 7, 9)[:nd]],
                           [1] + [0] * (nd - 2) + [1] if nd >= 2 else [1])]
                for label, n, per in shapes:
                    gd = W.grid(n, [-1.0] * nd, [1.1] * nd, periodic=per)
                    l = _target(gd)
                    marches = ("per_stage", "multi_step") if nd <= 2 else ("per_stage",)
                    for march in marches:
                        yield _compare("%dd_%s_%s_rk%d_%s_%s" % (nd, label, scheme, rk, march,
                                                                  "x".join(map(str, n))),
                                       gd, dyn, l, prec, scheme=scheme, rk=rk, march=march,
                                       check_every=2)
            if nd == 2:
                # ragged multi-tile grids in every tile shape (31x32, 15x64, 63x16)
                for scheme, rk in SCHEMES:
                    for tv in (1, 2, 3):
                        gd = W.grid([70, 135], [-1.0, -1.5], [1.1, 1.2], periodic=[0, 1])
                        yield _compare("2d_ragged_%s_tile%d" % (scheme, tv), gd, dyn,
                                       _target(gd), prec, scheme=scheme, rk=rk, tile_variant=tv,
                                       march="per_stage")
                gd = W.grid([70, 135], [-1.0, -1.5], [1.1, 1.2])
                yield _compare("2d_ragged_weno5_multi_step", gd, dyn, _target(gd), prec,
                               scheme="weno5", rk=3, march="multi_step", check_every=2)
            if nd >= 3:
                n = [13, 11, 37] if nd == 3 else [6, 9, 7, 40]
                per = [0] * nd
                per[0] = 1
                gd = W.grid(n, [-1.0] * nd, [1.1] * nd, periodic=per)
                for scheme, rk in SCHEMES:
                    if min(n) >= 2 * GHOST[scheme] + 1:
                        yield _compare("%dd_ragged_%s" % (nd, scheme), gd, dyn, _target(gd), prec,
                                       scheme=scheme, rk=rk)


def option_cases():
    rng = np.random.Generator(np.random.PCG64(77))
    for prec in ("f64", "f32"):
        dyn = _dyn(2, rng)
        gd = W.grid([9, 41], [-1.0, -1.0], [1.1, 1.2])
        l = _target(gd)
        # an interval of one step: every step compares with the snapshot
        yield _compare("interval", gd, dyn, l, prec, steps=12, scheme="weno5", rk=3,
                       interval=1e-9, interval_tol=1e-12)
        yield _compare("local_lf", gd, dyn, l, prec, scheme="weno5", rk=3, local_lf=True)
        yield _compare("brs", gd, dyn, l, prec, scheme="eno2", rk=2, brs=True)
        yield _compare("discount", gd, dyn, l, prec, scheme="eno2", rk=2, discount=0.97)
        yield _compare("warm_k", gd, dyn, l, prec, k=l - 0.3 + 0.1 * np.cos(3 * l),
                       scheme="eno2", rk=2)
        for nd in (3, 4):
            dyn_n = _dyn(nd, rng)
            gd_n = W.grid([5] + [7] * (nd - 1), [-1.0] * nd, [1.1] * nd)
            yield _compare("local_lf_%dd" % nd, gd_n, dyn_n, _target(gd_n), prec,
                           scheme="eno2", rk=2, local_lf=True)


def batch_engine_noalloc_cases():
    import torch
    rng = np.random.Generator(np.random.PCG64(5))
    for prec in ("f64", "f32"):
        dt = np.float64 if prec == "f64" else np.float32
        dyn = _dyn(2, rng)
        shapes = [[7, 7], [9, 40], [33, 65], [5, 131]]
        gds = [W.grid(n, [-1.0, -1.0], [1.1, 1.2]) for n in shapes]
        ls = [_target(gd) for gd in gds]
        grids = []
        for gd in gds:
            g = hji.Grid(gd, prec)
            g.set_dynamics(dyn)
            grids.append(g)
        sts, _ = hji.batch_solve(grids, [x.astype(dt) for x in ls], scheme="eno2", rk=2,
                                 tol=0.0, max_steps=3)
        errs = []
        for g, gd, l, st in zip(grids, gds, ls, sts):
            Vo, _ = orc.solve(orc.problem(gd, dyn), l, scheme="eno2", rk=2, tol=0.0, max_steps=3)
            errs.append(float(np.abs(g.value().astype(np.float64) - Vo).max()))
            g.close()
        tol = 1e-10 if prec == "f64" else 1e-5 * 2.0
        yield {"case": "batch", "prec": prec, "err": max(errs), "tol": tol,
               "ok": max(errs) <= tol and all(s["steps"] == 3 for s in sts)}
        # the serving engine: two requests of different sizes
        eng = hji.Engine(2, prec, max_slots=2, scheme="eno2", rk=2, tol=0.0, max_steps=3,
                         check_every=2)
        egrids = []
        for i, gd in enumerate(gds[:2]):
            g = hji.Grid(gd, prec)
            g.set_dynamics(dyn)
            egrids.append(g)
            eng.submit(g, ls[i].astype(dt), tag=i)
        done = eng.drain()
        errs = []
        for g, gd, l in zip(egrids, gds[:2], ls[:2]):
            Vo, _ = orc.solve(orc.problem(gd, dyn), l, scheme="eno2", rk=2, tol=0.0, max_steps=3)
            errs.append(float(np.abs(g.value().astype(np.float64) - Vo).max()))
            g.close()
        eng.close()
        codes = sorted(rc for _, _, rc in done)
        yield {"case": "engine", "prec": prec, "err": max(errs), "tol": tol, "codes": codes,
               "ok": max(errs) <= tol and all(c in (hji.HJI_OK, hji.HJI_E_NOT_CONVERGED)
                                              for c in codes) and len(codes) == 2}
    # the allocation-free entry point
    from test_zz_no_alloc import _noalloc
    for prec in ("f64", "f32"):
        dt = np.float64 if prec == "f64" else np.float32
        gd = W.grid([7, 70], [-1.0, -1.0], [1.1, 1.2])
        dyn = _dyn(2, rng)
        l = _target(gd)
        rc, out, st = _noalloc(hji, torch, gd, dyn, l.astype(dt), None, prec, scheme="weno5",
                               rk=3, tol=0.0, max_steps=3)
        Vo, _ = orc.solve(orc.problem(gd, dyn), l, scheme="weno5", rk=3, tol=0.0, max_steps=3)
        err = float(np.abs(out.astype(np.float64) - Vo).max())
        tol = 1e-10 if prec == "f64" else 1e-5 * max(1.0, float(np.abs(l).max()))
        yield {"case": "noalloc", "prec": prec, "rc": rc, "err": err, "tol": tol,
               "ok": rc in (hji.HJI_OK, hji.HJI_E_NOT_CONVERGED) and err <= tol}


def stencil_wider_than_grid():
    """A grid with fewer nodes than the stencil needs is refused before any
    device work."""
    gd = W.grid([5, 9], [-1.0, -1.0], [1.0, 1.0])
    g = hji.Grid(gd, "f64")
    g.set_dynamics(_dyn(2, np.random.Generator(np.random.PCG64(1))))
    try:
        g.solve(_target(gd), scheme="weno5", rk=3, tol=0.0, max_steps=1)
        ok, status = False, 0
    except hji.HJIError as e:
        ok, status = e.status == hji.HJI_E_INVALID, e.status
    g.close()
    return {"case": "n_below_stencil", "status": status, "ok": ok}


def main():
    import ctypes
    import torch
    assert torch.cuda.is_available()
    assert hji.library_path().endswith("_hji_checked.so"), hji.library_path()
    hji.load(build_if_missing=True)
    checked, count, site = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    index, extent = ctypes.c_int64(), ctypes.c_int64()
    rc = hji.hji_selftest_index_check(None, ctypes.byref(checked), ctypes.byref(count),
                                      ctypes.byref(site), ctypes.byref(index), ctypes.byref(extent))
    print(json.dumps({"case": "selftest", "rc": rc, "checked": checked.value, "count": count.value,
                      "site": site.value, "index": index.value, "extent": extent.value,
                      "ok": rc == 0 and checked.value == 1 and count.value == 3}), flush=True)
    n = bad = 0
    for gen in (grid_cases(), option_cases(), batch_engine_noalloc_cases()):
        while True:
            try:
                r = next(gen)
            except StopIteration:
                break
            except hji.HJIError as e:
                r = {"case": "error", "status": e.status, "msg": str(e), "ok": False}
            except Exception:  # noqa: BLE001
                r = {"case": "exception", "trace": traceback.format_exc()[-2000:], "ok": False}
                print(json.dumps(r), flush=True)
                bad += 1
                break
            n += 1
            bad += 0 if r["ok"] else 1
            print(json.dumps(r), flush=True)
    r = stencil_wider_than_grid()
    n += 1
    bad += 0 if r["ok"] else 1
    print(json.dumps(r), flush=True)
    print(json.dumps({"summary": True, "cases": n, "failed": bad}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
