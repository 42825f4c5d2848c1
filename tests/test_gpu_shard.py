"""Probe ranges on the GPU: the psi values of probe ranges evaluated
separately (as ranks of a sharded estimate would, one after another here)
are bit-identical to the same probes of one full run, for both precisions;
the single-rank sharded driver returns the full-run estimate."""
import numpy as np
import pytest

from paper_2212_09642_gb300 import graphs, shard, vne

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fp64", [False, True])
def test_probe_ranges_bit_identical(vctx, fp64):
    g = graphs.barabasi_albert(5000, 3, 21)
    total, m, seed = 37, 20, 123
    mat = vne.matrix_from_graph(vctx, g, fp64=fp64)
    try:
        _, _, full = vne.vne_entropy_hutchinson(vctx, mat, total, m, seed, want_psi=True)
        parts = []
        for rank in range(3):
            b, c = shard.probe_range(total, 3, rank)
            _, _, psi = vne.vne_entropy_hutchinson(vctx, mat, c, m, seed, opt=vne.options(probe_offset=b),
                                                   want_psi=True)
            parts.append(psi)
        est, se, n = shard.hutchinson(vctx, mat, total, m, seed)
        ref_est, ref_se = vne.vne_entropy_hutchinson(vctx, mat, total, m, seed)
    finally:
        vne.vne_matrix_destroy(mat)
    assert np.array_equal(np.concatenate(parts), full)
    assert n == total
    assert abs(est - ref_est) <= 1e-14 * abs(ref_est)
    assert abs(se - ref_se) <= 1e-10 * ref_se


def test_negative_probe_offset_rejected(vctx):
    g = graphs.erdos_renyi(500, 0.02, 1)
    mat = vne.matrix_from_graph(vctx, g)
    try:
        with pytest.raises(vne.VneError):
            vne.vne_entropy_hutchinson(vctx, mat, 4, 5, 1, opt=vne.options(probe_offset=-1))
    finally:
        vne.vne_matrix_destroy(mat)


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _hpp_rank(rank, world, port, fp64, out):
    import os

    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ctx = vne.vne_ctx_create(0)
    try:
        g = graphs.barabasi_albert(5000, 3, 21)
        mat = vne.matrix_from_graph(ctx, g, fp64=fp64)
        try:
            o = vne.options(reorth=1 if fp64 else 0)
            est, r, psi = shard.hutchpp(ctx, mat, 16, 20, 24, 9, fp64, opt=o)
        finally:
            vne.vne_matrix_destroy(mat)
        out[rank] = (est, r, psi.tolist())
    finally:
        vne.vne_ctx_destroy(ctx)
        dist.destroy_process_group()


@pytest.mark.parametrize("fp64", [False, True])
def test_hutchpp_two_gloo_ranks_reproduce_one_call(vctx, fp64):
    """Two ranks (processes) on this GPU, each with its own context: each
    computes its range of the sketch columns, the sketch is all-gathered over
    gloo, each evaluates its range of the quadratic forms, two scalars are
    all-reduced.  The ranks' quadratic forms are the one-call values bit for
    bit, and the estimate is the one-call estimate up to the order of the
    final sums.  The ranks' kernels never wait on one another."""
    import torch.multiprocessing as mp
    g = graphs.barabasi_albert(5000, 3, 21)
    mat = vne.matrix_from_graph(vctx, g, fp64=fp64)
    o = vne.options(reorth=1 if fp64 else 0)
    try:
        ref, parts = vne.vne_entropy_hutchpp(vctx, mat, 16, 20, 24, 9, opt=o)
        Y = vne.vne_hutchpp_sketch(vctx, mat, 0, 16, 24, 9, fp64, opt=o)
        psi_all, _, r_all = vne.vne_hutchpp_project(vctx, mat, Y, 16, 20, 24, 9, opt=o)
        single, _, _ = shard.hutchpp(vctx, mat, 16, 20, 24, 9, fp64, opt=o)
    finally:
        vne.vne_matrix_destroy(mat)
    assert abs(single - ref) <= 1e-14 * abs(ref)
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_hpp_rank, args=(2, _free_port(), fp64, out), nprocs=2, start_method="spawn", join=True)
    (e0, r0, p0), (e1, r1, p1) = out[0], out[1]
    assert r0 == r1 == r_all == int(parts[2])
    assert np.array_equal(np.array(p0 + p1), psi_all)
    assert e0 == e1 and abs(e0 - ref) <= 1e-14 * abs(ref)
