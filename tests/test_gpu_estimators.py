"""Trace-estimator parity: GPU (C ABI) vs the FP64 oracle on identical probes."""
import math

import numpy as np
import pytest

from oracle import coloring, density, entropy, estimators, rng
from paper_2212_09642_gb300 import graphs, vne

pytestmark = pytest.mark.gpu


def test_c1_hutchinson_fp64_parity(vctx):
    # ER G(2000, 0.005) seed 1, 100 Rademacher vectors, 50 Lanczos steps, FP64
    g = graphs.erdos_renyi(2000, 0.005, 1)
    A, _ = density.density_matrix(g)
    mat = vne.matrix_from_graph(vctx, g, fp64=True)
    try:
        est, se, psi = vne.vne_entropy_hutchinson(vctx, mat, 100, 50, seed=2, want_psi=True)
    finally:
        vne.vne_matrix_destroy(mat)
    ref_est, ref_psi = estimators.hutchinson(A, 100, 50, seed=2, reorth="full")
    assert np.max(np.abs(psi - ref_psi) / np.abs(ref_psi)) <= 1e-10
    assert abs(est - ref_est) <= 1e-10 * abs(ref_est)
    S = entropy.dense_entropy(A)
    assert abs(est - S) <= 5 * se + 1e-12


@pytest.mark.parametrize("fp64,tol", [(True, 1e-10), (False, 1e-5)])
def test_hutchpp_parity(vctx, fp64, tol):
    g = graphs.barabasi_albert(3000, 3, 4)
    A, _ = density.density_matrix(g)
    mat = vne.matrix_from_graph(vctx, g, fp64=fp64)
    reorth = 1 if fp64 else 0
    try:
        est, parts = vne.vne_entropy_hutchpp(vctx, mat, 16, 24, 30, seed=5, opt=vne.options(reorth=reorth))
    finally:
        vne.vne_matrix_destroy(mat)
    ref, rp = estimators.hutchpp(A, 16, 24, 30, seed=5, reorth="full" if fp64 else "none", return_parts=True)
    assert int(parts[2]) == rp["Q"].shape[1]
    assert abs(est - ref) <= tol * abs(ref), (est, ref)
    assert abs(parts[0] - rp["low_rank"]) <= tol * abs(ref)


def test_hutchpp_full_sketch_is_exact(vctx):
    g = graphs.erdos_renyi(24, 0.3, 5)
    A, _ = density.density_matrix(g)
    mat = vne.matrix_from_graph(vctx, g, fp64=True)
    try:
        est, parts = vne.vne_entropy_hutchpp(vctx, mat, 24, 8, 24, seed=3)
    finally:
        vne.vne_matrix_destroy(mat)
    assert int(parts[2]) == 23
    assert abs(est - entropy.dense_entropy(A)) <= 1e-10 * entropy.dense_entropy(A)


@pytest.mark.parametrize("fp64", [True, False])
def test_probing_parity_and_lower_bound(vctx, fp64):
    g = graphs.grid2d(30, 40)
    A, _ = density.density_matrix(g)
    S = entropy.dense_entropy(A)
    col = coloring.greedy_distance_coloring(g, 2)
    mat = vne.matrix_from_graph(vctx, g, fp64=fp64)
    try:
        est, s = vne.vne_entropy_probing(vctx, mat, None, 2, 40, opt=vne.options(reorth=1 if fp64 else 0))
        est2, s2 = vne.vne_entropy_probing(vctx, mat, col, 0, 40, opt=vne.options(reorth=1 if fp64 else 0))
    finally:
        vne.vne_matrix_destroy(mat)
    assert s == s2 == col.max() + 1
    ref, _ = estimators.probing(A, col, 40, reorth="full" if fp64 else "none")
    tol = 1e-10 if fp64 else 1e-5
    assert abs(est - ref) <= tol * ref and abs(est2 - ref) <= tol * ref
    assert est <= S * (1 + 1e-6)  # probing is a lower bound for graph entropy


def test_batched_equals_alone_and_oracle(vctx):
    gs = [graphs.erdos_renyi(1500, 8 / 1499, 11), graphs.barabasi_albert(2500, 3, 12),
          graphs.watts_strogatz(1200, 6, 0.1, 13), graphs.barabasi_albert(700, 3, 14),
          graphs.erdos_renyi(4000, 8 / 3999, 15)]
    opt = vne.options(reorth=0, panel=8)
    mats = [vne.matrix_from_graph(vctx, g, fp64=False) for g in gs]
    try:
        est, se = vne.vne_batch_hutchinson(vctx, mats, 64, 40, 21, opt=opt)
        alone = [vne.vne_entropy_hutchinson(vctx, m, 64, 40, 21, opt=opt)[0] for m in mats]
    finally:
        for m in mats:
            vne.vne_matrix_destroy(m)
    assert np.array_equal(est, np.array(alone))  # bit-identical alone and in the batch
    for g, e in zip(gs, est):
        A, _ = density.density_matrix(g)
        ref, _ = estimators.hutchinson(A, 64, 40, seed=21, reorth="none")
        assert abs(e - ref) <= 1e-5 * ref
