"""Parity at the headline's full size: the BA graph with n = 10^6, m = 4
(seed 3), FP32, the schedule the autotuner picks (as the benchmark times it),
60 Lanczos steps.  The oracle evaluates a few sampled quadratic forms one by
one (FP64 Lanczos with the same breakdown rule and no reorthogonalisation,
as the FP32 path), and the FP32 Hutch++ estimate is compared with the FP64
device run on identical vectors (the accuracy the headline is quoted at)."""
import numpy as np
import pytest

from oracle import density, krylov, rng
from paper_2212_09642_gb300 import graphs, vne

pytestmark = pytest.mark.gpu

N, M_BA, SEED, STEPS = 1_000_000, 4, 3, 60


@pytest.fixture(scope="module")
def headline_graph():
    return graphs.barabasi_albert(N, M_BA, SEED)


def test_sampled_quadforms_at_full_size(vctx, headline_graph):
    g = headline_graph
    mat = vne.matrix_from_graph(vctx, g, fp64=False, reorder=True)
    try:
        vne.vne_autotune(vctx, mat, 112, 8)
        # probes 100..111: the first Hutchinson columns of the headline's Hutch++
        opt = vne.options(reorth=0, probe_offset=100)
        _, _, psi = vne.vne_entropy_hutchinson(vctx, mat, 12, STEPS, 7, opt=opt, want_psi=True)
    finally:
        vne.vne_matrix_destroy(mat)
    A, _ = density.density_matrix(g)
    nA = density.gershgorin_norm(A)
    X = rng.rademacher(7, g.n, 100, 3)
    for j in range(3):
        ref = krylov.lanczos_quadform(A, X[:, j], STEPS, reorth="none", norm_A=nA)[0]
        assert abs(psi[j] - ref) <= 1e-5 * abs(ref), (j, psi[j], ref)


def test_hutchpp_fp32_against_fp64_at_full_size(vctx, headline_graph):
    """The headline's metric is quoted at a relative error of 1e-4 of the
    mixed-precision estimate against the FP64 run on identical vectors."""
    g = headline_graph
    ests = {}
    for fp64 in (False, True):
        mat = vne.matrix_from_graph(vctx, g, fp64=fp64, reorder=True)
        try:
            ests[fp64] = vne.vne_entropy_hutchpp(vctx, mat, 100, 100, STEPS, 11, opt=vne.options(reorth=0))[0]
        finally:
            vne.vne_matrix_destroy(mat)
    assert abs(ests[False] - ests[True]) <= 1e-4 * abs(ests[True]), ests


def test_hutchpp_parts_against_oracle_at_full_size(vctx, headline_graph):
    """The headline's Hutch++ path (FP32, degree relabelling, the tuned
    schedule, 60 steps) at n = 10^6 on a sketch small enough for the oracle:
    N_r = 6 sketch columns and N_H = 4 projected vectors, against the FP64
    oracle (no reorthogonalisation on either side).  The quadratic forms
    psi(q_i) and psi(g'_j) to 1e-5; the pivot order exactly; the sketch
    columns, vectors recovered from 61 FP32 Lanczos slots, to 5e-5 of their
    norm (the mixed path's vector tolerance)."""
    from oracle import estimators
    g = headline_graph
    Nr, NH, seed = 6, 4, 13
    mat = vne.matrix_from_graph(vctx, g, fp64=False, reorder=True)
    try:
        vne.vne_autotune(vctx, mat, 112, 8)
        opt = vne.options(reorth=0)
        Y = vne.vne_hutchpp_sketch(vctx, mat, 0, Nr, STEPS, seed, False, opt=opt)
        psi, piv, r = vne.vne_hutchpp_project(vctx, mat, Y, Nr, NH, STEPS, seed, opt=opt)
    finally:
        vne.vne_matrix_destroy(mat)
    A, _ = density.density_matrix(g)
    _, rp = estimators.hutchpp(A, Nr, NH, STEPS, seed=seed, reorth="none", return_parts=True)
    assert r == rp["Q"].shape[1] == Nr
    assert np.array_equal(piv, rp["pivots"])
    assert np.max(np.abs(psi[:Nr] - rp["psi_q"]) / np.abs(rp["psi_q"])) <= 1e-5
    assert np.max(np.abs(psi[Nr:] - rp["psi_g"]) / np.abs(rp["psi_g"])) <= 1e-5
    Yr = rp["Y"]
    for j in range(Nr):
        assert np.linalg.norm(Y[:, j] - Yr[:, j]) <= 5e-5 * np.linalg.norm(Yr[:, j]), j
