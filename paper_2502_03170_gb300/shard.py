"""Partitioning of the PSF work across ranks (one process per GPU).

Every unit of the hot path is independent: the planes of one Fourier stack,
the emitters of a Bessel batch, the elements of an adjoint batch.  A rank
takes a contiguous range of units and writes its own slab; no data moves
between ranks on the forward path.  The one real exchange is the adjoint of a
single pupil whose planes are spread over ranks: dL/dW_0 and dL/dc are sums
over planes (Eq. 15 chain rule), so the per-rank partial gradients are summed
with one all-reduce.

Host logic only; the collective goes through torch.distributed (NCCL on GPUs,
gloo on CPU).
"""


def split_even(n_units, rank, world):
    """Contiguous range [lo, hi) of rank `rank` out of `world` for n_units
    equal units (the first n_units % world ranks take one more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    base, extra = divmod(int(n_units), world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def split_weighted(offsets, rank, world):
    """Emitter range [e_lo, e_hi) of `rank` for a packed batch whose emitter e
    owns slices offsets[e] .. offsets[e+1]: the cut points are the emitter
    boundaries closest to equal shares of slices, so every rank gets whole
    emitters and about the same number of output slices."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    offs = [int(v) for v in offsets]
    n_em, total = len(offs) - 1, offs[-1]

    def cut(k):
        if k <= 0:
            return 0
        if k >= world:
            return n_em
        goal = total * k / world
        lo, hi = 0, n_em
        while lo < hi:                      # first boundary with offs >= goal
            mid = (lo + hi) // 2
            if offs[mid] < goal:
                lo = mid + 1
            else:
                hi = mid
        if lo > 0 and goal - offs[lo - 1] < offs[lo] - goal:
            lo -= 1
        return lo

    return cut(rank), max(cut(rank), cut(rank + 1))


def local_batch(offsets, z, e_lo, e_hi):
    """Offsets (rebased to 0) and z list of emitters [e_lo, e_hi)."""
    a, b = int(offsets[e_lo]), int(offsets[e_hi])
    return [int(v) - a for v in offsets[e_lo:e_hi + 1]], z[a:b]


def allreduce_sum_(tensor, group=None):
    """In-place sum over ranks of a partial gradient (no-op on one rank)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(tensor, op=dist.ReduceOp.SUM, group=group)
    return tensor


def max_over_ranks(values, device=None):
    """Element-wise maximum over ranks of a list of floats (the step time of
    a multi-GPU run is that of the slowest rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]
