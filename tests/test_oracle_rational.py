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
