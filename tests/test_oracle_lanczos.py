"""Pins for the oracle's Lanczos quadrature (Section 4)."""
import itertools
import math

import numpy as np
import pytest

from oracle import density, entropy, krylov, rng, bounds
from paper_2212_09642_gb300 import graphs as G


def _rho(g):
    return density.density_matrix(g)[0]


@pytest.mark.parametrize("m", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("reorth", ["full", "none"])
def test_polynomial_exactness(m, reorth):
    # Lemma exactness-rational-krylov-quadform with all poles at infinity:
    # psi_m is exact for polynomials of degree <= 2m - 1.
    A = _rho(G.erdos_renyi(150, 0.06, 3))
    b = rng.rademacher(5, 150, 0, 1)[:, 0]
    c = krylov.desingularize(b)
    Ad = A.toarray()
    for p in range(0, 2 * m):
        exact = float(c @ np.linalg.matrix_power(Ad, p) @ c)
        got = krylov.lanczos_quadform(A, b, m, reorth=reorth, f=lambda x, p=p: x ** p)[0]
        assert math.isclose(got, exact, rel_tol=1e-9, abs_tol=1e-14 * abs(exact) + 1e-300)
    # and not exact one degree higher (the pin would miss a wrong step count otherwise)
    p = 2 * m
    exact = float(c @ np.linalg.matrix_power(Ad, p) @ c)
    got = krylov.lanczos_quadform(A, b, m, reorth=reorth, f=lambda x: x ** p)[0]
    assert abs(got - exact) > 1e-11 * abs(exact)


def test_alpha_beta_match_explicit_projection():
    # A_m = V_m^T A V_m is the tridiagonal built from alpha, beta
    A = _rho(G.watts_strogatz(200, 6, 0.2, 1))
    c = krylov.desingularize(rng.rademacher(1, 200, 0, 1)[:, 0])
    alpha, beta, V = krylov.lanczos(A, c, 12, reorth="full", keep_basis=True)
    T = np.diag(alpha) + np.diag(beta[:-1], 1) + np.diag(beta[:-1], -1)
    assert np.allclose(V.T @ V, np.eye(12), atol=1e-13)
    assert np.allclose(V.T @ (A @ V), T, atol=1e-15)
    assert np.allclose(V[:, 0], c / np.linalg.norm(c))


def test_invariant_subspace_gives_exact_quadform():
    # Q_5 has 6 distinct Laplacian eigenvalues: Lanczos breaks down by m = 6
    g = G.hypercube(5)
    A = _rho(g)
    F = entropy.dense_matrix_function(A)
    b = rng.rademacher(2, g.n, 0, 1)[:, 0]
    c = krylov.desingularize(b)
    psi, alpha, beta = krylov.lanczos_quadform(A, b, 20, reorth="full")
    assert len(alpha) <= 6 and beta[-1] == 0.0
    assert math.isclose(psi, float(b @ F @ b), rel_tol=1e-12)
    assert math.isclose(psi, float(c @ F @ c), rel_tol=1e-12)


def test_complete_graph_breaks_down_after_one_step():
    A = _rho(G.complete(40))
    b = rng.rademacher(3, 40, 0, 1)[:, 0]
    psi, alpha, beta = krylov.lanczos_quadform(A, b, 10)
    c = krylov.desingularize(b)
    assert len(alpha) == 1
    lam = 40.0 / (40 * 39)
    assert math.isclose(psi, float(c @ c) * (-lam * math.log(lam)), rel_tol=1e-13)


def test_full_dimension_equals_dense_quadform():
    g = G.erdos_renyi(60, 0.1, 7)
    A = _rho(g)
    F = entropy.dense_matrix_function(A)
    for j in range(3):
        b = rng.rademacher(11, 60, j, 1)[:, 0]
        psi = krylov.lanczos_quadform(A, b, 60, reorth="full")[0]
        assert math.isclose(psi, float(b @ F @ b), rel_tol=1e-10)


def test_fmatvec_full_dimension_equals_dense():
    g = G.barabasi_albert(50, 2, 7)
    A = _rho(g)
    F = entropy.dense_matrix_function(A)
    b = rng.rademacher(4, 50, 0, 1)[:, 0]
    y = krylov.lanczos_fmatvec(A, b, 50, reorth="full")
    assert np.allclose(y, F @ b, atol=1e-12 * np.linalg.norm(F @ b))


def test_hutchinson_brute_force_over_all_sign_vectors():
    # E[x x^T] = I holds exactly when averaging over all 2^n sign vectors, so the
    # average of the quadratic forms equals tr f(A) = S (eq. hutchinson...).
    g = G.path(5)
    g2 = G.from_edges(9, np.array([0, 1, 2, 3, 5, 6, 7, 2, 4]), np.array([1, 2, 3, 4, 6, 7, 8, 6, 8]))
    for graph in (g, g2):
        A = _rho(graph)
        n = graph.n
        S = entropy.dense_entropy(A)
        tot = 0.0
        for signs in itertools.product((-1.0, 1.0), repeat=n):
            tot += krylov.lanczos_quadform(A, np.array(signs), n, reorth="full")[0]
        assert math.isclose(tot / 2 ** n, S, rel_tol=1e-10)


def test_apriori_bound_holds():
    # Proposition 4.2 (poles at infinity) + Theorem 2.2 on [lambda_2, lambda_n]
    g = G.erdos_renyi(300, 0.04, 2)
    A = _rho(g)
    lam = np.linalg.eigvalsh(A.toarray())
    l2, ln = lam[1], lam[-1]
    assert l2 > 1e-10  # connected
    F = entropy.dense_matrix_function(A)
    b = rng.rademacher(9, 300, 0, 1)[:, 0]
    c = krylov.desingularize(b)
    exact = float(c @ F @ c)
    for m in (2, 4, 6, 10, 14):
        psi = krylov.lanczos_quadform(A, b, m, reorth="full")[0]
        assert abs(psi - exact) <= bounds.lanczos_apriori_bound(float(c @ c), m, l2, ln)


def test_posterior_bounds_bracket_the_error():
    # Theorem 4.4, polynomial Krylov case
    g = G.watts_strogatz(400, 6, 0.3, 4)
    A = _rho(g)
    lam = np.linalg.eigvalsh(A.toarray())
    l2, ln = lam[1], lam[-1]
    F = entropy.dense_matrix_function(A)
    b = rng.rademacher(6, 400, 0, 1)[:, 0]
    c = krylov.desingularize(b)
    exact = float(c @ F @ c)
    for m in (3, 6, 10, 16):
        psi, alpha, beta = krylov.lanczos_quadform(A, b, m, reorth="full")
        lo, hi, est = bounds.posterior_bounds(alpha, beta, float(c @ c), l2, ln, grid=20000)
        err = abs(psi - exact)
        assert lo <= err * (1 + 1e-6) + 1e-300
        assert err <= hi * (1 + 1e-6)
        assert lo <= est <= hi


# ---- partial reorthogonalisation (Simon's omega recurrence) ----

def _pro_case():
    A = _rho(G.erdos_renyi(400, 0.05, 3))
    c = krylov.desingularize(rng.rademacher(1, 400, 0, 1)[:, 0])
    return A, c


@pytest.mark.parametrize("eps", [2.0 ** -53, 2.0 ** -24])
def test_partial_reorth_keeps_semi_orthogonality(eps):
    # plain Lanczos loses orthogonality completely within 150 steps here;
    # partial reorthogonalisation keeps |v_i . v_k| at the sqrt(eps) level it
    # promises, reorthogonalising in pairs of steps and far less often than
    # every step
    A, c = _pro_case()
    _, _, Vn = krylov.lanczos(A, c, 150, reorth="none", keep_basis=True)
    assert np.max(np.abs(Vn.T @ Vn - np.eye(Vn.shape[1]))) > 0.1
    st = {}
    _, _, V = krylov.lanczos(A, c, 150, reorth="partial", keep_basis=True, eps=eps, stats=st)
    off = np.abs(V.T @ V - np.eye(V.shape[1]))
    assert np.max(off) <= 10 * math.sqrt(eps)
    steps = st["reorth_steps"]
    assert 2 <= len(steps) < 150 / 2
    assert all(b == a + 1 for a, b in zip(steps[0::2], steps[1::2]))  # each trigger is followed by its pair


def test_partial_reorth_estimates_track_the_loss():
    # omega_{j+1,k} estimates v_{j+1} . v_k: the measured inner products stay
    # within a modest factor of the estimates at every step
    A, c = _pro_case()
    st = {}
    _, _, V = krylov.lanczos(A, c, 150, reorth="partial", keep_basis=True, stats=st)
    for j, om in enumerate(st["omega"]):
        if j + 1 >= V.shape[1]:
            break
        actual = np.abs(V[:, : j + 1].T @ V[:, j + 1])
        assert np.all(actual <= 100.0 * np.abs(om[: j + 1]) + 1e-15), j


@pytest.mark.parametrize("m", [2, 5, 8])
def test_partial_reorth_polynomial_exactness(m):
    # Lemma exactness-rational-krylov-quadform holds with the partial policy too
    A = _rho(G.erdos_renyi(150, 0.06, 3))
    b = rng.rademacher(5, 150, 0, 1)[:, 0]
    c = krylov.desingularize(b)
    Ad = A.toarray()
    for p in range(0, 2 * m):
        exact = float(c @ np.linalg.matrix_power(Ad, p) @ c)
        got = krylov.lanczos_quadform(A, b, m, reorth="partial", eps=2.0 ** -24, f=lambda x, p=p: x ** p)[0]
        assert math.isclose(got, exact, rel_tol=1e-9, abs_tol=1e-14 * abs(exact) + 1e-300)
