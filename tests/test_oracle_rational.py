"""Pins for the oracle's rational Krylov quadrature (Sections 4, 4.2)."""
import math

import numpy as np
import pytest

from oracle import density, entropy, krylov, rational, rng
from paper_2212_09642_gb300 import graphs as G


def _setup(n=120):
    g = G.watts_strogatz(n, 6, 0.2, 2)
    A = density.density_matrix(g)[0]
    shifts = rational.default_shifts(A, count=4, decades=3.0)
    b = rng.rademacher(4, n, 0, 1)[:, 0]
    c = krylov.desingularize(b)
    return A, shifts, b, c


def _dense_quadform(A, c, fn):
    lam, U = np.linalg.eigh(A.toarray())
    y = U.T @ c
    return float(np.sum(y * y * fn(lam)))


def test_exactness_for_rational_functions():
    # Lemma exactness-rational-krylov-quadform: exact for p_{2m-1} / q_{m-1}^2.
    # Here m = 1 + 2 + 4 = 7 and q_6 has the 4 finite poles -s_k.
    A, s, b, c = _setup()
    tests = [
        lambda x: 1.0 / (x + s[0]),
        lambda x: 1.0 / (x + s[1]) ** 2,
        lambda x: x ** 5,
        lambda x: x ** 3 / ((x + s[2]) * (x + s[3])),
        lambda x: 1.0 / ((x + s[0]) ** 2 * (x + s[3]) ** 2),
    ]
    for fn in tests:
        got = rational.rational_quadform(A, b, s, n_inf=2, f=fn)
        want = _dense_quadform(A, c, fn)
        assert math.isclose(got, want, rel_tol=1e-8), (got, want)


def test_rational_beats_polynomial_of_same_dimension():
    A, s8, b, c = _setup(400)
    s = rational.default_shifts(A)
    exact = _dense_quadform(A, c, entropy.f_entropy)
    rat = rational.rational_quadform(A, b, s, n_inf=2)
    poly = krylov.lanczos_quadform(A, b, 11)[0]
    assert abs(rat - exact) < abs(poly - exact)


def test_complete_graph_exact():
    A = density.density_matrix(G.complete(30))[0]
    b = rng.rademacher(1, 30, 0, 1)[:, 0]
    c = krylov.desingularize(b)
    lam = 1.0 / 29
    got = rational.rational_quadform(A, b, rational.default_shifts(A))
    assert math.isclose(got, float(c @ c) * (-lam * math.log(lam)), rel_tol=1e-12)


def test_cg_solves_match_dense():
    A, s, b, c = _setup(300)
    Xd = rational.shifted_solves(A, c, s, method="dense")
    Xc = rational.shifted_solves(A, c, s, method="cg", rtol=1e-12)
    assert np.allclose(Xd, Xc, rtol=1e-8, atol=1e-10 * np.abs(Xd).max())


# ---- mixed polynomial / rational Krylov (Section 5.3 switching rule) ----

def test_switch_index_rule():
    """Switch after iteration k when err_k / err_{k-ell-1} >= c^ell (ell = 3,
    c = 0.75: 0.421875), first possible at k = ell + 2 = 5."""
    assert rational.switch_index([0.5 ** k for k in range(1, 13)]) == 12  # ratio 0.0625: never
    assert rational.switch_index([0.9 ** k for k in range(1, 13)]) == 5   # ratio 0.656 at once
    est = [1.0, 0.1, 0.01, 1e-3, 1e-4, 9e-5, 8e-5, 7e-5, 6e-5, 5e-5]
    # k = 9: 6e-5 / 1e-4 = 0.6 is the first ratio >= 0.421875 (k = 8: 7e-5 / 1e-3)
    assert rational.switch_index(est) == 9
    assert rational.switch_index([1.0, 0.2, 0.0, 0.1]) == 3  # invariant Krylov space
    ratio_at_threshold = 0.75 ** 3
    assert rational.switch_index([1.0, 1.0, 1.0, 1.0, ratio_at_threshold]) == 5


def test_mixed_without_poles_is_lanczos_quadrature():
    """With no finite poles the space is K_k(A, c): the projection equals the
    k-step Lanczos (Gauss) quadrature."""
    g = G.barabasi_albert(400, 3, 6)
    A, _ = density.density_matrix(g)
    b = rng.rademacher(3, g.n, 0, 1)[:, 0]
    for k in (3, 7, 11):
        psi, _ = rational.mixed_quadform(A, b, [], k_poly=k, k_max=12)
        ref = krylov.lanczos_quadform(A, b, k)[0]
        assert abs(psi - ref) <= 1e-12 * abs(ref), (k, psi, ref)


def test_mixed_complete_graph_exact():
    g = G.complete(30)
    A, _ = density.density_matrix(g)
    b = rng.rademacher(5, 30, 0, 1)[:, 0]
    c = krylov.desingularize(b)
    lam = 1.0 / 29
    psi, k = rational.mixed_quadform(A, b, rational.default_shifts(A))
    assert k == 1  # the Krylov space of c is invariant after one step
    assert abs(psi - float(c @ c) * (-lam * math.log(lam))) <= 1e-12


def test_mixed_matches_dense_on_small_graph():
    """K_k(A, c) + the eight pole directions: on a 300-node graph the
    quadrature agrees with c^T f(A) c from the dense spectrum to 1e-9."""
    g = G.watts_strogatz(300, 6, 0.2, 9)
    A, _ = density.density_matrix(g)
    F = entropy.dense_matrix_function(A)
    b = rng.rademacher(7, g.n, 0, 1)[:, 0]
    c = krylov.desingularize(b)
    psi, k = rational.mixed_quadform(A, b, rational.default_shifts(A))
    assert abs(psi - float(c @ F @ c)) <= 1e-9 * float(c @ F @ c)


def test_drop_rule_is_rounding_level():
    # exact rational Arnoldi drops nothing: a direction independent to 1e-9
    # is kept (its normalised remainder is the new basis vector), an exact
    # repeat is dropped
    e = np.eye(6)
    W = np.column_stack([e[:, 0], e[:, 0] + 1e-9 * e[:, 1], 2.0 * e[:, 0], e[:, 2]])
    V = rational.orthonormalize(W)
    assert V.shape[1] == 3
    assert np.allclose(np.abs(V[:, 1]), e[:, 1], atol=1e-6)
    assert np.allclose(V.T @ V, np.eye(3), atol=1e-14)


def test_repeated_pole_adds_no_direction():
    A, s, b, c = _setup()
    W1 = rational.rational_basis(A, c, s[:3], n_inf=2, method="dense")
    W2 = rational.rational_basis(A, c, np.concatenate([s[:3], s[1:2]]), n_inf=2, method="dense")
    assert rational.orthonormalize(W1).shape[1] == rational.orthonormalize(W2).shape[1] == 6
