"""Pins for the oracle's trace estimators and colouring (Section 3)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import coloring, density, entropy, estimators, bounds
from paper_2212_09642_gb300 import graphs as G


def _rho(g):
    return density.density_matrix(g)[0]


def test_hutchpp_with_full_sketch_is_exact():
    # N_r >= rank f(A): Q spans range f(A), tr(Q^T B Q) = tr B, residual part 0
    g = G.erdos_renyi(24, 0.3, 5)
    A = _rho(g)
    S = entropy.dense_entropy(A)
    est, parts = estimators.hutchpp(A, 24, 6, 24, seed=3, return_parts=True)
    assert parts["Q"].shape[1] == 23  # f(A) 1 = 0 removes one direction
    assert math.isclose(est, S, rel_tol=1e-9)
    assert abs(parts["resid"]) < 1e-9


def test_hutchpp_unbiased_statistically():
    g = G.watts_strogatz(60, 4, 0.3, 1)
    A = _rho(g)
    S = entropy.dense_entropy(A)
    ests = [estimators.hutchpp(A, 4, 8, 30, seed=s) for s in range(60)]
    se = np.std(ests) / math.sqrt(len(ests))
    assert abs(np.mean(ests) - S) < 4 * se + 1e-12


def test_hutchinson_variance_matches_rademacher_formula():
    # Var[x^T B x] = 2 (||B||_F^2 - sum_i B_ii^2) for Rademacher x
    g = G.erdos_renyi(80, 0.08, 2)
    A = _rho(g)
    F = entropy.dense_matrix_function(A)
    S = float(np.trace(F))
    est, psi = estimators.hutchinson(A, 400, 80, seed=8)
    var = 2 * (np.sum(F * F) - np.sum(np.diag(F) ** 2))
    assert abs(np.var(psi) / var - 1) < 0.25
    assert abs(est - S) < 4 * math.sqrt(var / 400)


def test_probing_exact_when_all_colours_distinct():
    g = G.path(12)
    A = _rho(g)
    col = coloring.greedy_distance_coloring(g, 11)
    assert len(set(col.tolist())) == 12
    T, _ = estimators.probing(A, col, 12)
    assert math.isclose(T, entropy.dense_entropy(A), rel_tol=1e-11)


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_probing_lower_bound_and_error_identity(d):
    # Proposition probing-graph-entropy-lower-bound and eq. probing_error_identity
    g = G.barabasi_albert(150, 2, 9)
    A = _rho(g)
    F = entropy.dense_matrix_function(A)
    S = float(np.trace(F))
    col = coloring.greedy_distance_coloring(g, d)
    T_exact = estimators.probing_exact(F, col)
    assert T_exact <= S + 1e-13
    off = 0.0
    for l in range(col.max() + 1):
        idx = np.where(col == l)[0]
        blk = F[np.ix_(idx, idx)]
        off += blk.sum() - np.trace(blk)
    assert math.isclose(S - T_exact, -off, rel_tol=1e-9, abs_tol=1e-13)
    T_kry, _ = estimators.probing(A, col, 150)
    assert math.isclose(T_kry, T_exact, rel_tol=1e-9)


def test_probing_corollary_bound():
    g = G.grid2d(12, 12)
    A = _rho(g)
    lam = np.linalg.eigvalsh(A.toarray())
    S = entropy.dense_entropy(A)
    F = entropy.dense_matrix_function(A)
    for d in (2, 3, 5):
        col = coloring.greedy_distance_coloring(g, d)
        err = abs(S - estimators.probing_exact(F, col))
        assert err <= bounds.probing_bound(g.n, d, 0.0, lam[-1])
        assert err <= bounds.probing_bound(g.n, d, lam[1], lam[-1])


@pytest.mark.parametrize("d", [1, 2, 3])
def test_greedy_coloring_valid_and_greedy(d):
    # Brute force via the pattern of (I + W)^d (the paper's alternative
    # construction of the distance-d neighbourhoods): the colouring is a
    # distance-d colouring and each node has the smallest colour not used by
    # its earlier-visited d-neighbours (Algorithm greedy_coloring).
    g = G.random_geometric(200, 0.12, 3)
    col = coloring.greedy_distance_coloring(g, d)
    W = sp.csr_matrix((np.ones(g.nnz), g.col, g.rowptr), shape=(g.n, g.n))
    P = sp.identity(g.n, format="csr") + W
    R = sp.identity(g.n, format="csr")
    for _ in range(d):
        R = (R @ P).tocsr()
        R.data[:] = 1.0
    R = R.toarray() > 0
    order = coloring.greedy_order(g)
    rank = np.empty(g.n, dtype=int)
    rank[order] = np.arange(g.n)
    for i in range(g.n):
        nb = np.where(R[i])[0]
        nb = nb[nb != i]
        assert np.all(col[nb] != col[i])
        earlier = {int(col[j]) for j in nb if rank[j] < rank[i]}
        assert col[i] == min(set(range(len(earlier) + 1)) - earlier)
    assert coloring.is_distance_coloring(g, col, d)


def test_grid_colors_at_least_the_optimum():
    # the optimal distance-d colouring of a 2D grid has ceil((d+1)^2/2) colours
    g = G.grid2d(20, 20)
    for d in (1, 2, 3):
        col = coloring.greedy_distance_coloring(g, d)
        assert col.max() + 1 >= math.ceil((d + 1) ** 2 / 2)


# ---- orth() of eq. Hutch++_formula: column-pivoted QR ----

def _brute_force_pivots(Y, r):
    """Greedy column choice by explicit least squares: at every step the
    column with the largest residual after fitting it by the chosen ones."""
    chosen = []
    for _ in range(r):
        best, bi = -1.0, -1
        for c in range(Y.shape[1]):
            if c in chosen:
                continue
            y = Y[:, c]
            if chosen:
                B = Y[:, chosen]
                coef = np.linalg.lstsq(B, y, rcond=None)[0]
                res = np.linalg.norm(y - B @ coef)
            else:
                res = np.linalg.norm(y)
            if res > best:
                best, bi = res, c
        chosen.append(bi)
    return np.array(chosen)


def test_orth_is_column_pivoted_qr():
    rs = np.random.default_rng(11)
    Y = rs.standard_normal((60, 9)) * np.array([3.0, 0.2, 5.0, 1.0, 0.7, 2.5, 0.1, 4.0, 1.5])
    Q, piv = estimators.orthonormal_range(Y, return_pivots=True)
    assert Q.shape == (60, 9)
    assert np.array_equal(piv, _brute_force_pivots(Y, 9))
    assert np.allclose(Q.T @ Q, np.eye(9), atol=1e-14)
    R = Q.T @ Y[:, piv]
    assert np.allclose(np.tril(R, -1), 0.0, atol=1e-13)
    assert np.all(np.diag(R) > 0.0)
    assert np.all(np.diff(np.abs(np.diag(R))) <= 1e-12)
    assert np.allclose(Q @ R, Y[:, piv], atol=1e-13)


def test_orth_rank_of_low_rank_sketch():
    rs = np.random.default_rng(12)
    Y = rs.standard_normal((50, 3)) @ rs.standard_normal((3, 7))
    Q = estimators.orthonormal_range(Y)
    assert Q.shape[1] == 3
    U = np.linalg.svd(Y, full_matrices=False)[0][:, :3]
    assert np.allclose(Q @ Q.T, U @ U.T, atol=1e-13)


def test_hutchpp_parts_consistent():
    # the low-rank part is the sum of the quadratures of the pivoted Q's
    # columns; G' is orthogonal to Q
    g = G.barabasi_albert(200, 3, 4)
    A = _rho(g)
    est, p = estimators.hutchpp(A, 6, 5, 20, seed=5, return_parts=True)
    assert p["Q"].shape[1] == 6 and len(p["pivots"]) == 6
    assert math.isclose(p["low_rank"], float(np.sum(p["psi_q"])), rel_tol=1e-15)
    assert math.isclose(est, p["low_rank"] + p["resid"], rel_tol=1e-15)
