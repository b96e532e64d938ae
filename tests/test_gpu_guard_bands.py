"""Guard bands around every device buffer of the library (the plan that
stands in for a memory checker, which this GPU pool does not offer): a test
allocator, handed to the library through the hji_allocator hook, places each
allocation between two bands of a known byte pattern and checks both bands
when the library frees the buffer.  Solves over ragged, periodic, 1-D to
4-D grids, both precisions, both launch forms and every option must leave
every band intact (no kernel writes past the end or before the start of a
field, the tile list, the descriptors, the state or the tables)."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

GUARD = 4096  # bytes on each side; keeps the library's 512-byte alignment


class GuardedAllocator:
    def __init__(self, hji, torch):
        self.torch = torch
        self.live = {}
        self.checked = 0
        self.violations = []

        def _alloc(nbytes, stream, ctx):
            n = int(nbytes)
            t = torch.empty(n + 2 * GUARD, dtype=torch.uint8, device="cuda")
            t[:GUARD].fill_(0xA5)
            t[GUARD + n:].fill_(0x5A)
            torch.cuda.synchronize()
            ptr = t.data_ptr() + GUARD
            self.live[ptr] = (t, n)
            return ptr

        def _free(ptr, stream, ctx):
            torch.cuda.synchronize()
            t, n = self.live.pop(int(ptr))
            lo_ok = bool((t[:GUARD] == 0xA5).all().item())
            hi_ok = bool((t[GUARD + n:] == 0x5A).all().item())
            self.checked += 1
            if not (lo_ok and hi_ok):
                self.violations.append((n, lo_ok, hi_ok))

        self._fa = hji._ALLOC_FN(_alloc)
        self._ff = hji._FREE_FN(_free)
        self.struct = hji.hji_allocator(self._fa, self._ff, None)


def _runs():
    rng = np.random.Generator(np.random.PCG64(9))
    g1 = W.grid([263], [-2.0], [2.0])
    d1 = {"c": [0.3], "G": [[1.0]], "ulo": [-0.5], "uhi": [1.0], "terms": [(0, 0, "sin", 0.4)]}
    g2, d2, _ = W.di_config(37, dmax=0.2)
    g3 = W.grid([13, 19, 35], [-1.0, -2.0, -1.5], [1.0, 2.0, 1.5], periodic=[1, 0, 0])
    d3 = {"A": rng.normal(size=(3, 3)) * 0.5, "G": [[1.0], [0.0], [0.5]], "ulo": [-1],
          "uhi": [1], "terms": [(2, 0, "cos", 0.7)]}
    g4, d4, _ = W.quad4d_config(13, dmax=0.3)
    out = []
    for gd, dyn in ((g1, d1), (g2, d2), (g3, d3), (g4, d4)):
        X = W.mesh(gd)
        l = np.sqrt(sum(x ** 2 for x in X)) - 0.6
        out.append((gd, dyn, l))
    return out


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_no_kernel_writes_outside_its_buffers(hji_lib, prec):
    import torch
    assert torch.cuda.is_available()
    hji = hji_lib
    ga = GuardedAllocator(hji, torch)
    dt = np.float64 if prec == "f64" else np.float32
    variants = [dict(scheme="eno2", rk=2, march="per_stage"),
                dict(scheme="weno5", rk=3, march="multi_step", interval=0.02, interval_tol=1e-9),
                dict(scheme="eno1", rk=1, brs=True),
                dict(scheme="eno2", rk=2, local_lf=True, interval=0.02, interval_tol=1e-9)]
    for gd, dyn, l in _runs():
        for opts in variants:
            g = hji.Grid(gd, prec, allocator=ga.struct)
            g.set_dynamics(dyn)
            g.solve(l.astype(dt), tol=0.0, max_steps=11, check_every=4, **opts)
            g.solve(l.astype(dt), init=hji.HJI_INIT_RESIDENT, tol=0.0, max_steps=5, **opts)
            if len(gd["n"]) == 2:
                g.optimal_control(opts["scheme"])
            g.value()
            g.close()
    # a batch of uneven grids led by the first one (its tile list and descriptors)
    insts = W.batch_instances(count=4, seed=3, side=(41, 77))
    grids = [hji.Grid(i["grid"], prec, allocator=ga.struct) for i in insts]
    for g, i in zip(grids, insts):
        g.set_dynamics(i["dyn"])
    hji.batch_solve(grids, [W.instance_target(i).astype(dt) for i in insts], scheme="eno2",
                    rk=2, tol=0.0, max_steps=9)
    for g in grids:
        g.close()
    assert not ga.live
    assert ga.checked > 50
    assert not ga.violations, ga.violations


def test_engine_buffers_and_its_grids_stay_inside_their_bands(hji_lib):
    """The serving engine's own buffers (descriptors, counters, tile list)
    come from its allocator too; requests arriving while others march."""
    import torch
    assert torch.cuda.is_available()
    hji = hji_lib
    ga = GuardedAllocator(hji, torch)
    insts = W.batch_instances(count=5, seed=8, side=(31, 90))
    grids = []
    for i in insts:
        g = hji.Grid(i["grid"], "f32", allocator=ga.struct)
        g.set_dynamics(i["dyn"])
        grids.append(g)
    eng = hji.Engine(2, "f32", max_slots=2, allocator=ga.struct, scheme="eno2", rk=2,
                     tol=0.0, max_steps=20, check_every=4)
    for t, (g, i) in enumerate(zip(grids, insts)):
        eng.submit(g, W.instance_target(i).astype(np.float32), tag=t)
    done = eng.drain()
    eng.close()
    for g in grids:
        g.close()
    assert sorted(t for t, _, _ in done) == list(range(len(insts)))
    assert not ga.live and ga.checked > 10
    assert not ga.violations, ga.violations
