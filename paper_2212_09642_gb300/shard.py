"""Probe-column sharding of one Hutchinson or Hutch++ estimate over a process
group.

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

Hutch++ (eq. Hutch++_formula) has one exchange step in the middle: every
rank computes its range of the sketch columns f(A) omega_j (stage 1), the
ranks all-gather the sketch, every rank forms the same Q = orth(Y) and
G' = (I - Q Q^T) G from the whole sketch (deterministic kernels, identical
inputs) and evaluates its range of the N_r + N_H quadratic forms of
[Q | G'] (stage 2); two scalars are all-reduced at the end.
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


def _all_gather_columns(Y, total_cols, group):
    """Concatenate the ranks' column blocks [n, k_r] (in rank order) into the
    whole [n, total_cols] block on every rank.  Blocks are padded to the
    largest k_r so that every rank sends the same shape."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    kmax = max(probe_range(total_cols, world, r)[1] for r in range(world))
    nccl = dist.get_backend(group) == "nccl"
    dev = f"cuda:{torch.cuda.current_device()}" if nccl else "cpu"
    t = torch.as_tensor(Y, device=dev)
    n = t.shape[0]
    pad = torch.zeros((n, kmax), dtype=t.dtype, device=dev)
    if t.shape[1]:
        pad[:, :t.shape[1]] = t
    outs = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(outs, pad, group=group)
    cols = [outs[r][:, :probe_range(total_cols, world, r)[1]] for r in range(world)]
    return torch.cat(cols, dim=1).contiguous()


def hutchpp(ctx, mat, sketch_cols: int, hutch_vectors: int, krylov_steps: int, seed: int, fp64: bool, opt=None,
            group=None, sketch_fn=None, project_fn=None):
    """Hutch++ estimate of S(rho) split over the ranks of `group` (the default
    group when torch.distributed is initialised, else one rank).

    Stage 1: this rank's range of the N_r sketch columns; all-gather; stage 2:
    this rank's range of the N_r + N_H quadratic forms; all-reduce of the
    low-rank and residual sums.  ``sketch_fn(c0, k)`` and
    ``project_fn(Y, c0, k)`` default to the library's stages
    (vne_hutchpp_sketch, vne_hutchpp_project); they can be replaced by another
    evaluator with the same contract.  Returns (estimate, rank of Q, the
    quadratic forms this rank evaluated)."""
    import torch.distributed as dist

    from . import vne
    if dist.is_available() and dist.is_initialized():
        world, rank = dist.get_world_size(group), dist.get_rank(group)
    else:
        world, rank = 1, 0
    Nr, NH = int(sketch_cols), int(hutch_vectors)
    if sketch_fn is None:
        def sketch_fn(c0, k):
            if k == 0:
                return np.zeros((vne.vne_matrix_info(mat)[0], 0), dtype=np.float64 if fp64 else np.float32)
            return vne.vne_hutchpp_sketch(ctx, mat, c0, k, krylov_steps, seed, fp64, opt=opt)
    if project_fn is None:
        def project_fn(Y, c0, k):
            return vne.vne_hutchpp_project(ctx, mat, Y, Nr, NH, krylov_steps, seed, col_begin=c0, ncols=k, opt=opt)
    c0, k = probe_range(Nr, world, rank)
    Y = sketch_fn(c0, k)  # [n, k]
    if world > 1:
        Yall = _all_gather_columns(Y, Nr, group)
        Yall = Yall if Yall.is_cuda else Yall.numpy()
    else:
        Yall = Y
    q0, qk = probe_range(Nr + NH, world, rank)
    psi, piv, r = project_fn(Yall, q0, qk)
    psi = np.asarray(psi, dtype=np.float64)
    idx = np.arange(q0, q0 + qk)
    low = math.fsum(psi[idx < r])
    res = math.fsum(psi[idx >= Nr])
    if world > 1:
        low, res = _allreduce_sum([low, res], group)
    est = low + (res / NH if NH > 0 else 0.0)
    return est, int(r), psi
