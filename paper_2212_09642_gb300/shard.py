"""Probe-column sharding of one Hutchinson estimate over a process group.

The quadratic forms v_l^T f(A) v_l of a trace estimate are independent of one
another (each probe builds its own Krylov space; Section 4, remark after the
rational Krylov matrix-function approximation), so the N probes of one
estimate split into contiguous ranges of the seeded Rademacher stream, one
range per rank.  Rank r evaluates its range on its own GPU with no exchange
during the Krylov iterations; at the end the ranks add two scalars each (the
sum of their psi values, then the sum of squared deviations from the common
mean).  The union of the ranges is exactly the probe set of a single run
with the same seed, so the sharded estimate is the single-run estimate up to
the order of the final additions.
"""
from __future__ import annotations

import math

import numpy as np


def probe_range(total: int, world: int, rank: int) -> tuple[int, int]:
    """(first probe, count) of `rank` when `total` probes split over `world`
    ranks: contiguous ranges whose sizes differ by at most one, the larger
    ones first; ranks beyond `total` get an empty range."""
    if total < 0 or world < 1 or not 0 <= rank < world:
        raise ValueError("need total >= 0, world >= 1 and 0 <= rank < world")
    base, extra = divmod(total, world)
    count = base + (1 if rank < extra else 0)
    begin = rank * base + min(rank, extra)
    return begin, count


def _allreduce_sum(values, group):
    import torch
    import torch.distributed as dist
    dev = "cpu"
    if dist.get_backend(group) == "nccl":
        dev = f"cuda:{torch.cuda.current_device()}"
    t = torch.tensor(values, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().tolist()


def combine(local_psi, group=None) -> tuple[float, float, int]:
    """Mean, standard error and count of the psi values of all ranks.

    Every rank calls this with its own psi values (possibly none) and gets the
    same result.  Two scalar all-reduces: the sum and count, then the sum of
    squared deviations from the mean (two passes, no cancellation)."""
    import torch.distributed as dist
    psi = np.asarray(local_psi, dtype=np.float64).ravel()
    if dist.is_available() and dist.is_initialized():
        s, n = _allreduce_sum([math.fsum(psi), float(psi.size)], group)
    else:
        s, n = math.fsum(psi), float(psi.size)
    count = int(round(n))
    if count == 0:
        raise ValueError("no probes on any rank")
    mean = s / count
    dev = math.fsum((psi - mean) ** 2)
    if dist.is_available() and dist.is_initialized():
        (dev,) = _allreduce_sum([dev], group)
    var = dev / (count - 1) if count > 1 else 0.0
    return mean, math.sqrt(var / count), count


def hutchinson(ctx, mat, num_vectors: int, krylov_steps: int, seed: int, opt=None, group=None):
    """Hutchinson estimate of S(rho) with the probes split over the ranks of
    `group` (the default group when torch.distributed is initialised, else a
    single rank).  Returns (estimate, standard error, probes on this rank)."""
    import torch.distributed as dist

    from . import vne
    if dist.is_available() and dist.is_initialized():
        world, rank = dist.get_world_size(group), dist.get_rank(group)
    else:
        world, rank = 1, 0
    begin, count = probe_range(num_vectors, world, rank)
    psi = np.zeros(0)
    if count > 0:
        o = vne.vne_options.from_buffer_copy(opt) if opt is not None else vne.options()
        o.probe_offset = int(o.probe_offset) + begin
        _, _, psi = vne.vne_entropy_hutchinson(ctx, mat, count, krylov_steps, seed, opt=o, want_psi=True)
    mean, se, _ = combine(psi, group)
    return mean, se, count
