"""Within-grid sharding of one march across ranks: the host side of the
multi-GPU design for a single grid too large for one device.

The grid is cut into slabs along axis 0 (the slowest, so each slab is one
contiguous block of every field).  Rank r owns rows [a_r, b_r) and keeps an
extended copy of rows [a_r - g, b_r + g) clipped to the grid, g being the
stencil's ghost width (2 for ENO2, 3 for WENO5).  Every Runge-Kutta stage of
the march of Sec. II-B, Eq. (7), then takes three steps:

  1. halo exchange: the first g owned rows go to rank r - 1 and the last g
     to rank r + 1, each received into the neighbour's halo rows (two
     send/receive pairs per interior rank, no collective);
  2. the stage operator L(W) on the extended slab.  A row's derivatives
     reach g rows along axis 0, so every owned row sees only true grid
     values; rows at a true grid edge get their ghost nodes exactly as on
     the whole grid, and the halo rows' own results (whose ghost nodes are
     extrapolated across the cut) are discarded;
  3. the stage combination of the TVD Runge-Kutta scheme on the owned rows.

After the last stage each rank projects onto V <= l (Eq. (7)-(8)) and forms
its share of max|V^{n+1} - V^n|; one all-reduce (max) per step gives every
rank the same convergence decision (Sec. IV).  The dissipation coefficients
and dt are maxima over the whole grid, reduced once per solve the same way.

The stage operator is passed in as a callable.  On a GPU rank it would be
the library's stage kernel run over the rank's extended slab; the C ABI has
no single-stage call, and every GPU run of this build uses one GPU, so this
within-grid form is a design whose host logic (partition, halo exchange,
reductions, stage combination) is tested on the CPU with gloo ranks and the
FP64 oracle as the operator.  Communication uses torch.distributed
point-to-point calls on the caller's process group (NCCL between GPUs,
gloo on the CPU); halos land in each rank's own memory, nothing is
multicast.
"""


def rk_stage(rk, i, V, W, L, dt):
    """Stage i (0-based) of the TVD Runge-Kutta step of order rk, from the
    stage input W and its operator value L = L(W), with the Euler stage
    E(W) = W + dt L:
      rk 1: V' = E(V);
      rk 2: W1 = E(V), V' = V/2 + E(W1)/2;
      rk 3: W1 = E(V), W2 = 3V/4 + E(W1)/4, V' = V/3 + 2 E(W2)/3."""
    euler = W + dt * L
    if i == 0:
        return euler
    if rk == 2:
        return 0.5 * V + 0.5 * euler
    if i == 1:
        return 0.75 * V + 0.25 * euler
    return V / 3.0 + 2.0 * euler / 3.0


def slab_bounds(n0, world, g):
    """Owned rows [start, stop) of axis 0 for each of `world` ranks:
    contiguous, sizes differing by at most one, each at least g rows so that
    a rank's halo comes from its two neighbours alone."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if g < 1:
        raise ValueError("ghost width must be >= 1")
    if n0 < world * g:
        raise ValueError("%d rows cannot give %d ranks %d rows each" % (n0, world, g))
    base, extra = divmod(n0, world)
    out, start = [], 0
    for r in range(world):
        size = base + (1 if r < extra else 0)
        out.append((start, start + size))
        start += size
    return out


def extended_bounds(bounds, rank, g):
    """Rows [start, stop) of rank's extended slab (owned rows plus up to g
    halo rows on each side, clipped to the grid)."""
    n0 = bounds[-1][1]
    a, b = bounds[rank]
    return max(0, a - g), min(n0, b + g)


def exchange_halos(W, bounds, rank, g, dist, group=None):
    """Fill the halo rows of rank's extended slab W (a tensor whose axis 0
    holds rows extended_bounds(...)) with its neighbours' owned rows."""
    world = len(bounds)
    a, b = bounds[rank]
    ea, eb = extended_bounds(bounds, rank, g)
    own0, own1 = a - ea, b - ea  # owned rows within W
    reqs = []
    recv_lo = recv_hi = None
    if rank > 0:
        send = W[own0:own0 + g].contiguous()
        recv_lo = W[own0 - g:own0].contiguous()
        reqs.append(dist.isend(send, rank - 1, group=group, tag=1))
        reqs.append(dist.irecv(recv_lo, rank - 1, group=group, tag=2))
    if rank < world - 1:
        send = W[own1 - g:own1].contiguous()
        recv_hi = W[own1:own1 + g].contiguous()
        reqs.append(dist.isend(send, rank + 1, group=group, tag=2))
        reqs.append(dist.irecv(recv_hi, rank + 1, group=group, tag=1))
    for r in reqs:
        r.wait()
    if recv_lo is not None:
        W[own0 - g:own0] = recv_lo
    if recv_hi is not None:
        W[own1:own1 + g] = recv_hi
    return W


def allreduce_max(value, dist, torch, group=None):
    """The maximum of a float over all ranks (FP64)."""
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def reduce_alpha_dt(alpha, dt, dist, torch, group=None):
    """Whole-grid dissipation coefficients and CFL step from each rank's
    values over its owned rows: alpha_a is a maximum over nodes (all-reduce
    max), dt = cfl / max(rate) is the smallest of the ranks' steps
    (all-reduce min; rounding is monotone, so this is the whole-grid dt)."""
    a = torch.tensor([float(v) for v in alpha], dtype=torch.float64)
    dist.all_reduce(a, op=dist.ReduceOp.MAX, group=group)
    t = torch.tensor([float(dt)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    return a.tolist(), float(t.item())


def owned_grid(gd, bounds, rank):
    """The rank's owned rows as a grid description (for its share of the
    set-up reductions)."""
    a, b = bounds[rank]
    n0, lo0, hi0 = gd["n"][0], gd["lo"][0], gd["hi"][0]
    dx0 = (hi0 - lo0) / (n0 - 1)
    out = {k: list(v) for k, v in gd.items()}
    out["n"][0] = b - a
    out["lo"][0] = lo0 + a * dx0
    out["hi"][0] = lo0 + (b - 1) * dx0
    return out


def slab_step(V, l, operator, dt, rk, bounds, rank, g, dist, torch, group=None):
    """One full Runge-Kutta step of the march on rank's extended slab.

    V, l: FP64 tensors of the extended slab (V^n's owned rows current; halo
    rows are refreshed here).  operator(W) returns L(W) on the extended
    slab.  Returns (V^{n+1} on the extended slab with its owned rows valid,
    max|V^{n+1} - V^n| over the whole grid)."""
    if rk not in (1, 2, 3):
        raise ValueError("rk must be 1, 2 or 3")
    a, b = bounds[rank]
    ea, _ = extended_bounds(bounds, rank, g)
    own = slice(a - ea, b - ea)
    exchange_halos(V, bounds, rank, g, dist, group)
    W = V
    for i in range(rk):
        if i > 0:
            exchange_halos(W, bounds, rank, g, dist, group)
        W = rk_stage(rk, i, V, W, operator(W), dt)
    Vn = torch.minimum(W, l)
    delta_local = float((Vn[own] - V[own]).abs().max().item()) if b > a else 0.0
    return Vn, allreduce_max(delta_local, dist, torch, group)


def gather_owned(V, bounds, rank, g, dist, torch, group=None):
    """Rank 0 receives every rank's owned rows (for checks and output);
    returns the whole grid on rank 0 and None elsewhere."""
    a, b = bounds[rank]
    ea, _ = extended_bounds(bounds, rank, g)
    mine = V[a - ea:b - ea].contiguous()
    if rank != 0:
        dist.send(mine, 0, group=group, tag=3)
        return None
    parts = [mine]
    for r in range(1, len(bounds)):
        ra, rb = bounds[r]
        buf = torch.empty((rb - ra,) + tuple(V.shape[1:]), dtype=V.dtype)
        dist.recv(buf, r, group=group, tag=3)
        parts.append(buf)
    return torch.cat(parts, 0)


def slab_grid(gd, bounds, rank, g):
    """The extended slab as a grid description: lo and hi are the
    coordinates of its first and last rows, so its spacing is the grid's
    (exactly so when the spacing and the node coordinates are representable,
    e.g. a power-of-two number of intervals on a dyadic interval; otherwise
    to rounding)."""
    ea, eb = extended_bounds(bounds, rank, g)
    n0, lo0, hi0 = gd["n"][0], gd["lo"][0], gd["hi"][0]
    dx0 = (hi0 - lo0) / (n0 - 1)
    out = {k: list(v) for k, v in gd.items()}
    out["n"][0] = eb - ea
    out["lo"][0] = lo0 + ea * dx0
    out["hi"][0] = lo0 + (eb - 1) * dx0
    return out


__all__ = ["rk_stage", "slab_bounds", "extended_bounds", "exchange_halos", "allreduce_max",
           "reduce_alpha_dt", "owned_grid", "slab_step", "gather_owned", "slab_grid"]
