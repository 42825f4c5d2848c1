"""Probe-column sharding over ranks (host logic, CPU): world_size-2 gloo
process groups, each rank evaluating its probe range with the FP64 oracle.
The combined estimate must equal the single-process estimate over all probes
(the ranges partition the seeded probe stream exactly)."""
import math
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2212_09642_gb300 import graphs, shard


def test_probe_range_partitions():
    for total in [0, 1, 2, 7, 100, 101]:
        for world in [1, 2, 3, 8]:
            ranges = [shard.probe_range(total, world, r) for r in range(world)]
            assert sum(c for _, c in ranges) == total
            pos = 0
            for b, c in ranges:
                assert b == pos and c >= 0
                pos += c
            counts = [c for _, c in ranges]
            assert max(counts) - min(counts) <= 1
    with pytest.raises(ValueError):
        shard.probe_range(5, 2, 2)


def test_combine_single_process():
    x = np.array([1.0, 2.0, 4.0, 7.0])
    mean, se, n = shard.combine(x)
    assert n == 4 and mean == 3.5
    assert math.isclose(se, np.std(x, ddof=1) / 2.0, rel_tol=1e-15)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, total, seed, m, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import density, estimators
        g = graphs.erdos_renyi(300, 0.03, 5)
        A, _ = density.density_matrix(g)
        begin, count = shard.probe_range(total, world, rank)
        psi = []
        if count:
            _, psi = estimators.hutchinson(A, count, m, seed, reorth="full", col_begin=begin)
        mean, se, n = shard.combine(psi)
        out[rank] = (mean, se, n, begin, count)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("total", [9, 1])
def test_gloo_two_ranks_match_single_run(total):
    from oracle import density, estimators
    world, seed, m = 2, 31, 12
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), total, seed, m, out), nprocs=world,
                       start_method="spawn", join=True)
    g = graphs.erdos_renyi(300, 0.03, 5)
    A, _ = density.density_matrix(g)
    ref, psi = estimators.hutchinson(A, total, m, seed, reorth="full")
    ref_se = np.std(psi, ddof=1) / math.sqrt(total) if total > 1 else 0.0
    res = [out[r] for r in range(world)]
    for mean, se, n, _, _ in res:
        assert n == total
        assert abs(mean - ref) <= 1e-14 * abs(ref)
        assert abs(se - ref_se) <= 1e-10 * max(ref_se, 1e-300)
    assert res[0][2] == res[1][2] and res[0][0] == res[1][0]  # same result on every rank
    assert res[0][4] + res[1][4] == total


# ---- Hutch++ split over ranks: the host logic with the oracle as evaluator ----

def _oracle_stages(A, Nr, NH, m, seed):
    """Stage functions with the contract of the library's two stages, written
    with the oracle: the sketch columns f(A) omega_j, and from the whole
    sketch Q = orth(Y), G' and the quadratic forms of a column range."""
    from oracle import density, estimators, krylov, rng
    nA = density.gershgorin_norm(A)
    n = A.shape[0]

    def sketch(c0, k):
        X = rng.rademacher(seed, n, c0, k)
        cols = [krylov.lanczos_fmatvec(A, X[:, j], m, reorth="full", norm_A=nA) for j in range(k)]
        return np.column_stack(cols) if k else np.zeros((n, 0))

    def project(Y, c0, k):
        Y = np.asarray(Y, dtype=np.float64)
        Q, piv = estimators.orthonormal_range(Y, return_pivots=True)
        r = Q.shape[1]
        G = rng.rademacher(seed, n, Nr, NH)
        Gp = G - Q @ (Q.T @ G)
        psi = []
        for i in range(c0, c0 + k):
            if i < Nr:
                psi.append(krylov.lanczos_quadform(A, Q[:, i], m, reorth="full", norm_A=nA)[0] if i < r else 0.0)
            else:
                psi.append(krylov.lanczos_quadform(A, Gp[:, i - Nr], m, reorth="full", norm_A=nA)[0])
        pv = np.full(Nr, -1, dtype=np.int32)
        pv[:r] = piv
        return np.array(psi), pv, r

    return sketch, project


def _hpp_worker(rank, world, port, Nr, NH, seed, m, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import density
        g = graphs.barabasi_albert(400, 3, 8)
        A, _ = density.density_matrix(g)
        sk, pr = _oracle_stages(A, Nr, NH, m, seed)
        est, r, psi = shard.hutchpp(None, None, Nr, NH, m, seed, True, sketch_fn=sk, project_fn=pr)
        out[rank] = (est, r, len(psi))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,Nr,NH", [(2, 8, 6), (3, 2, 4)])
def test_gloo_hutchpp_matches_single_run(world, Nr, NH):
    """world-size 2 and 3 gloo groups (with 3 ranks and N_r = 2 one rank has
    no sketch column): the sketch gathered from the ranks' column ranges, the
    quadratic forms split over the ranks and the two sums all-reduced give the
    oracle's one-process Hutch++ estimate."""
    from oracle import density, estimators
    seed, m = 17, 14
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_hpp_worker, args=(world, _free_port(), Nr, NH, seed, m, out), nprocs=world,
                       start_method="spawn", join=True)
    g = graphs.barabasi_albert(400, 3, 8)
    A, _ = density.density_matrix(g)
    ref, rp = estimators.hutchpp(A, Nr, NH, m, seed=seed, reorth="full", return_parts=True)
    res = [out[r] for r in range(world)]
    for est, r, _ in res:
        assert r == rp["Q"].shape[1]
        assert abs(est - ref) <= 1e-13 * abs(ref)
    assert sum(c for _, _, c in res) == Nr + NH
    assert len({e for e, _, _ in res}) == 1  # the same estimate on every rank
