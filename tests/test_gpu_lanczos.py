"""Lanczos quadrature parity: GPU (C ABI) vs the FP64 oracle on identical
vectors and step counts.  FP64 path (full reorthogonalisation on both sides):
relative error <= 1e-10.  Mixed path (FP32 vectors, FP64 scalars, plain
recurrence on both sides): relative error <= 1e-5."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import density, entropy, krylov, rng
from paper_2212_09642_gb300 import graphs, vne

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-10, 1e-5


def _cases():
    return [
        ("ER3000", graphs.erdos_renyi(3000, 0.003, 2)),
        ("BA20000", graphs.barabasi_albert(20000, 4, 3)),      # > 4 row tiles, long rows
        ("star+WS", graphs.disjoint_union([graphs.star(900), graphs.watts_strogatz(1100, 6, 0.2, 1)])),
        ("grid", graphs.grid2d(40, 50)),
    ]


def _oracle_psi(A, X, m, reorth):
    nA = density.gershgorin_norm(A)
    out = []
    for j in range(X.shape[1]):
        psi, a, b = krylov.lanczos_quadform(A, X[:, j], m, reorth=reorth, norm_A=nA)
        out.append((psi, a, b))
    return out


@pytest.mark.parametrize("name,g", _cases())
@pytest.mark.parametrize("m", [1, 7, 30])
def test_fp64_full_reorth_parity(vctx, name, g, m):
    A, _ = density.density_matrix(g)
    k = 13  # ragged: 2 panels of 8 with 3 padding columns
    X = rng.rademacher(5, g.n, 0, k)
    X[:, 3] = np.random.default_rng(1).standard_normal(g.n)  # one Gaussian column
    mat = vne.matrix_from_graph(vctx, g, fp64=True)
    try:
        psi, ab = vne.vne_quadform_batch(vctx, mat, X, m, opt=vne.options(reorth=1, item_nnz=64),
                                         want_alpha_beta=True)
    finally:
        vne.vne_matrix_destroy(mat)
    ref = _oracle_psi(A, X, m, "full")
    for j in range(k):
        assert abs(psi[j] - ref[j][0]) <= TOL64 * abs(ref[j][0]), (j, psi[j], ref[j][0])
        kk = len(ref[j][1])
        assert np.allclose(ab[j, :kk], ref[j][1], rtol=1e-10, atol=1e-13 * np.abs(ref[j][1]).max())


@pytest.mark.parametrize("name,g", _cases())
@pytest.mark.parametrize("panel", [8, 16, 32])
def test_fp32_mixed_parity(vctx, name, g, panel):
    A, _ = density.density_matrix(g)
    k, m = 21, 30
    X = rng.rademacher(8, g.n, 0, k)
    mat = vne.matrix_from_graph(vctx, g, fp64=False)
    try:
        psi = vne.vne_quadform_batch(vctx, mat, X, m, opt=vne.options(reorth=0, panel=panel))
    finally:
        vne.vne_matrix_destroy(mat)
    ref = np.array([r[0] for r in _oracle_psi(A, X, m, "none")])
    rel = np.abs(psi - ref) / np.abs(ref)
    assert rel.max() <= TOL32, rel.max()


@pytest.mark.parametrize("reorder,g", [
    (True, graphs.barabasi_albert(5000, 3, 7)),
    ("rcm", graphs.random_geometric(4000, graphs.rgg_radius_for_degree(4000, 6.0), 2)),
    ("rcm", graphs.disjoint_union([graphs.barabasi_albert(1500, 2, 1), graphs.grid2d(30, 40), graphs.star(50)])),
])
def test_reordering_leaves_quadforms_unchanged(vctx, reorder, g):
    A, _ = density.density_matrix(g)
    X = rng.rademacher(2, g.n, 0, 8)
    mat = vne.matrix_from_graph(vctx, g, fp64=True, reorder=reorder)
    try:
        psi = vne.vne_quadform_batch(vctx, mat, X, 20, opt=vne.options(reorth=1))
    finally:
        vne.vne_matrix_destroy(mat)
    ref = np.array([r[0] for r in _oracle_psi(A, X, 20, "full")])
    assert np.max(np.abs(psi - ref) / np.abs(ref)) <= TOL64


@pytest.mark.parametrize("fp64", [True, False])
def test_breakdown_cases_are_exact(vctx, fp64):
    tol = 1e-10 if fp64 else 1e-6
    # K_n: one Lanczos step spans an invariant subspace
    g = graphs.complete(64)
    A, _ = density.density_matrix(g)
    X = rng.rademacher(3, 64, 0, 4)
    mat = vne.matrix_from_graph(vctx, g, fp64=fp64)
    try:
        psi = vne.vne_quadform_batch(vctx, mat, X, 10, opt=vne.options(reorth=1 if fp64 else 0))
    finally:
        vne.vne_matrix_destroy(mat)
    F = entropy.dense_matrix_function(A)
    want = np.einsum("ij,ij->j", X, F @ X)
    assert np.max(np.abs(psi - want) / np.abs(want)) <= tol
    # hypercube Q_6: 7 distinct eigenvalues -> exact after 7 steps
    g = graphs.hypercube(6)
    A, _ = density.density_matrix(g)
    X = rng.rademacher(4, g.n, 0, 5)
    mat = vne.matrix_from_graph(vctx, g, fp64=fp64)
    try:
        psi = vne.vne_quadform_batch(vctx, mat, X, 25, opt=vne.options(reorth=1 if fp64 else 0))
    finally:
        vne.vne_matrix_destroy(mat)
    F = entropy.dense_matrix_function(A)
    want = np.einsum("ij,ij->j", X, F @ X)
    assert np.max(np.abs(psi - want) / np.abs(want)) <= tol


def test_edge_cases(vctx):
    # single column, tiny graph, a zero column, isolated nodes
    g = graphs.from_edges(7, np.array([0, 1, 2]), np.array([1, 2, 0]))  # triangle + 4 isolated nodes
    A, _ = density.density_matrix(g)
    X = np.zeros((7, 3))
    X[:, 0] = rng.rademacher(1, 7, 0, 1)[:, 0]
    X[:, 2] = 1.0  # constant vector: desingularised to zero
    mat = vne.matrix_from_graph(vctx, g, fp64=True)
    try:
        psi = vne.vne_quadform_batch(vctx, mat, X, 5, opt=vne.options(reorth=1))
        one = vne.vne_quadform_batch(vctx, mat, X[:, :1], 5, opt=vne.options(reorth=1))
    finally:
        vne.vne_matrix_destroy(mat)
    F = entropy.dense_matrix_function(A)
    want = np.einsum("ij,ij->j", X, F @ X)
    assert abs(psi[0] - want[0]) <= 1e-10 * abs(want[0])
    assert psi[1] == 0.0 and psi[2] == 0.0
    assert one[0] == psi[0]


@pytest.mark.parametrize("fp64", [True, False])
def test_valued_matrix_path(vctx, fp64):
    # general symmetric PSD matrix with explicit values (no desingularisation):
    # a diagonal matrix with Chebyshev-point eigenvalues, shuffled by a sparse
    # symmetric perturbation-free permutation (values path of the SpMM)
    n = 2000
    lam = 0.5 * (1e-3 + 1.0) + 0.5 * (1.0 - 1e-3) * np.cos(np.pi * (2 * np.arange(n) + 1) / (2 * n))
    lam /= lam.sum()
    W = graphs.watts_strogatz(n, 4, 0.1, 3)
    L = density.laplacian(W)
    M = (sp.diags(lam * 50) + 1e-4 * L / L.diagonal().max()).tocsr()
    M.sort_indices()
    A = M / M.diagonal().sum()
    X = rng.rademacher(6, n, 0, 9)
    mat = vne.vne_create_density_matrix(vctx, n, M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data,
                                        (vne.VNE_FP64 if fp64 else vne.VNE_FP32) | vne.VNE_NORMALIZE_TRACE)
    try:
        psi = vne.vne_quadform_batch(vctx, mat, X, 25, opt=vne.options(reorth=1 if fp64 else 0))
    finally:
        vne.vne_matrix_destroy(mat)
    ref = np.array([krylov.lanczos_quadform(A, X[:, j], 25, reorth="full" if fp64 else "none", desing=False)[0]
                    for j in range(9)])
    assert np.max(np.abs(psi - ref) / np.abs(ref)) <= (TOL64 if fp64 else TOL32)


def test_invalid_inputs_raise(vctx):
    g = graphs.path(5)
    with pytest.raises(vne.VneError):  # no precision flag
        vne.vne_create_density_matrix(vctx, g.n, g.rowptr, g.col, None, 0)
    bad = g.col.copy()
    bad[0] = 99
    with pytest.raises(vne.VneError):  # column out of range
        vne.vne_create_density_matrix(vctx, g.n, g.rowptr, bad, None, vne.VNE_FP32)
    empty = graphs.from_edges(4, np.zeros(0, np.int64), np.zeros(0, np.int64))
    with pytest.raises(vne.VneError):  # zero trace
        vne.vne_create_density_matrix(vctx, empty.n, empty.rowptr, empty.col, None, vne.VNE_FP32)
    asym = graphs.Graph(3, np.array([0, 1, 1, 1], np.int64), np.array([1], np.int32))
    with pytest.raises(vne.VneError):
        vne.vne_create_density_matrix(vctx, 3, asym.rowptr, asym.col, None, vne.VNE_FP32 | vne.VNE_CHECK_SYMMETRY)
    mat = vne.matrix_from_graph(vctx, g)
    try:
        with pytest.raises(vne.VneError):
            vne.vne_entropy_hutchinson(vctx, mat, 4, 0, 1)  # zero steps
    finally:
        vne.vne_matrix_destroy(mat)


def test_device_validation_reports_first_offender(vctx):
    """Column range and self-loops are checked on the device over many rows;
    the error names the first offending entry and the context stays usable."""
    g = graphs.erdos_renyi(200000, 4e-5, 9)
    k_late, k_early = g.nnz - 3, g.nnz // 2
    bad = g.col.copy()
    bad[k_late] = -1
    bad[k_early] = g.n
    with pytest.raises(vne.VneError, match="out of range") as ei:
        vne.vne_create_density_matrix(vctx, g.n, g.rowptr, bad, None, vne.VNE_FP32 | vne.VNE_REORDER)
    row = int(np.searchsorted(g.rowptr, k_early, side="right") - 1)
    assert f"row {row}" in str(ei.value)
    loop = g.col.copy()
    r = int(np.searchsorted(g.rowptr, k_late, side="right") - 1)
    loop[k_late] = r
    with pytest.raises(vne.VneError, match="self-loop"):
        vne.vne_create_density_matrix(vctx, g.n, g.rowptr, loop, None, vne.VNE_FP32)
    # the context is still usable
    mat = vne.matrix_from_graph(vctx, g, reorder=True)
    try:
        est, _ = vne.vne_entropy_hutchinson(vctx, mat, 8, 5, 1)
        assert np.isfinite(est)
    finally:
        vne.vne_matrix_destroy(mat)


def test_autotuned_schedule_keeps_parity(vctx):
    g = graphs.barabasi_albert(30000, 4, 21)
    A, _ = density.density_matrix(g)
    X = rng.rademacher(3, g.n, 0, 10)
    mat = vne.matrix_from_graph(vctx, g, fp64=False, reorder=True)
    try:
        chosen, ms = vne.vne_autotune(vctx, mat, 16, 4)
        assert chosen.panel in (8, 16, 32) and chosen.item_nnz in (128, 256, 512, 1024)
        assert 0 <= chosen.step_variant < 14 and ms > 0
        psi = vne.vne_quadform_batch(vctx, mat, X, 30, opt=vne.options(reorth=0))
        # a second matrix of the same shape inherits the tuned schedule
        mat2 = vne.matrix_from_graph(vctx, g, fp64=False, reorder=True)
        try:
            psi2 = vne.vne_quadform_batch(vctx, mat2, X, 30, opt=vne.options(reorth=0))
        finally:
            vne.vne_matrix_destroy(mat2)
    finally:
        vne.vne_matrix_destroy(mat)
    assert np.array_equal(psi, psi2)
    ref = np.array([r[0] for r in _oracle_psi(A, X, 30, "none")])
    assert np.max(np.abs(psi - ref) / np.abs(ref)) <= TOL32


@pytest.mark.parametrize("variant", list(range(14)))
def test_every_step_variant_matches_oracle_and_is_deterministic(vctx, variant):
    # item_nnz = 64 splits every row longer than 64 into chunks (many long rows)
    g = graphs.barabasi_albert(20000, 4, 3)
    A, _ = density.density_matrix(g)
    X = rng.rademacher(8, g.n, 0, 12)
    mat = vne.matrix_from_graph(vctx, g, fp64=False)
    try:
        opt = vne.options(reorth=0, step_variant=variant, item_nnz=64)
        psi = vne.vne_quadform_batch(vctx, mat, X, 30, opt=opt)
        again = [vne.vne_quadform_batch(vctx, mat, X, 30, opt=opt) for _ in range(3)]
    finally:
        vne.vne_matrix_destroy(mat)
    for a in again:
        assert np.array_equal(a, psi)  # bit-reproducible run to run
    ref = np.array([r[0] for r in _oracle_psi(A, X, 30, "none")])
    assert np.max(np.abs(psi - ref) / np.abs(ref)) <= TOL32


@pytest.mark.parametrize("variant,ipw", [(4, 2), (10, 2), (12, 4), (0, 4)])
def test_items_per_warp_match_oracle_and_are_deterministic(vctx, variant, ipw):
    # a warp takes ipw work items in turn (long rows split at item_nnz = 64)
    g = graphs.barabasi_albert(20000, 4, 3)
    A, _ = density.density_matrix(g)
    X = rng.rademacher(8, g.n, 0, 12)
    mat = vne.matrix_from_graph(vctx, g, fp64=False, reorder=True)
    try:
        opt = vne.options(reorth=0, step_variant=variant, item_nnz=64, items_per_warp=ipw)
        psi = vne.vne_quadform_batch(vctx, mat, X, 30, opt=opt)
        again = vne.vne_quadform_batch(vctx, mat, X, 30, opt=opt)
    finally:
        vne.vne_matrix_destroy(mat)
    assert np.array_equal(again, psi)
    ref = np.array([r[0] for r in _oracle_psi(A, X, 30, "none")])
    assert np.max(np.abs(psi - ref) / np.abs(ref)) <= TOL32
