"""Within-grid sharding (slabs along axis 0, g halo rows exchanged per
Runge-Kutta stage, one all-reduce of max|dV| per step) on CPU gloo ranks,
with the FP64 oracle's spatial operator as each rank's stage operator.

The march split over 2 and 3 ranks must reproduce the single-grid oracle
march bit for bit: every owned row's stencil reads only true grid values
(its halo rows come from the neighbour), rows at a true grid edge see the
same ghost nodes as on the whole grid, and the stage combinations and the
projection onto V <= l are the same operations in the same order.  The set-
up reductions (alpha by all-reduce max, dt by all-reduce min over the ranks'
owned rows) must also give the whole grid's values exactly.

The grid is dyadic (64 and 32 intervals on [-2, 2]) so that a slab's node
coordinates and spacing equal the whole grid's exactly.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STEPS = 6


def _problem():
    sys.path.insert(0, ROOT)
    import workloads as W
    gd = W.grid([65, 33], [-2.0, -2.0], [2.0, 2.0])
    dyn = W.double_integrator(umax=1.0, dmax=0.2)
    X1, X2 = W.mesh(gd)
    l = 1.0 - np.abs(X1) + 0.05 * np.sin(3.0 * X2)  # not constant along axis 1
    return gd, dyn, l


def _worker(rank, world, port, scheme, rk, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1903_07715_gb300 import slabs
    oracle.set_threads(2)
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        gd, dyn, l = _problem()
        g = oracle.ghost_width(scheme)
        bounds = slabs.slab_bounds(gd["n"][0], world, g)
        # Set-up: each rank over its owned rows, then the two reductions.
        P_own = oracle.problem(slabs.owned_grid(gd, bounds, rank), dyn)
        a_loc, dt_loc = oracle.alpha_dt(P_own, 0.5)
        alpha, dt = slabs.reduce_alpha_dt(a_loc, dt_loc, dist, torch)
        ea, eb = slabs.extended_bounds(bounds, rank, g)
        P_ext = oracle.problem(slabs.slab_grid(gd, bounds, rank, g), dyn)

        def operator(W):
            return torch.from_numpy(oracle.operator(P_ext, scheme, alpha, W.numpy()))

        l_ext = torch.from_numpy(np.ascontiguousarray(l[ea:eb]))
        V = l_ext.clone()
        deltas = []
        for _ in range(STEPS):
            V, d = slabs.slab_step(V, l_ext, operator, dt, rk, bounds, rank, g, dist, torch)
            deltas.append(d)
        whole = slabs.gather_owned(V, bounds, rank, g, dist, torch)
        if rank == 0:
            out["V"] = whole.numpy().tobytes()
            out["shape"] = tuple(whole.shape)
        out[rank] = (list(alpha), dt, deltas)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("scheme,rk", [("eno2", 2), ("weno5", 3), ("eno1", 1)])
def test_slab_march_equals_single_grid_march(orc, world, scheme, rk):
    gd, dyn, l = _problem()
    P = orc.problem(gd, dyn)
    alpha, dt = orc.alpha_dt(P, 0.5)
    V = orc.init(P, l)
    want_d = []
    for _ in range(STEPS):
        V, d = orc.step(P, scheme, rk, dt, alpha, l, V)
        want_d.append(d)
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, scheme, rk, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    got = np.frombuffer(out["V"], dtype=np.float64).reshape(out["shape"])
    assert got.shape == V.shape
    assert np.array_equal(got, V)
    for r in range(world):
        a_r, dt_r, d_r = out[r]
        assert a_r == list(alpha) and dt_r == dt
        assert d_r == want_d


def test_slab_bounds_partition():
    sys.path.insert(0, ROOT)
    from paper_1903_07715_gb300 import slabs
    for n0, world, g in [(65, 2, 2), (65, 3, 3), (10, 5, 2), (101, 8, 3), (7, 1, 3)]:
        b = slabs.slab_bounds(n0, world, g)
        assert b[0][0] == 0 and b[-1][1] == n0
        sizes = [e - s for s, e in b]
        assert all(s >= g for s in sizes) and max(sizes) - min(sizes) <= 1
        assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
        for r in range(world):
            ea, eb = slabs.extended_bounds(b, r, g)
            assert ea == max(0, b[r][0] - g) and eb == min(n0, b[r][1] + g)
    with pytest.raises(ValueError):
        slabs.slab_bounds(5, 3, 2)
