"""Pins for the dense entropy oracle: closed-form spectra and invariants (Section 2)."""
import math

import numpy as np
import pytest

from oracle import density, entropy
from paper_2212_09642_gb300 import graphs as G

CASES = [
    (lambda: G.complete(7), lambda: entropy.spectrum_complete(7)),
    (lambda: G.path(11), lambda: entropy.spectrum_path(11)),
    (lambda: G.cycle(12), lambda: entropy.spectrum_cycle(12)),
    (lambda: G.star(9), lambda: entropy.spectrum_star(9)),
    (lambda: G.complete_bipartite(3, 5), lambda: entropy.spectrum_complete_bipartite(3, 5)),
    (lambda: G.hypercube(5), lambda: entropy.spectrum_hypercube(5)),
    (lambda: G.grid2d(6, 9), lambda: entropy.spectrum_grid(6, 9)),
    (lambda: G.grid2d(5, 8, periodic=True), lambda: entropy.spectrum_grid(5, 8, periodic=True)),
]


@pytest.mark.parametrize("mk_graph,mk_spec", CASES)
def test_dense_entropy_matches_closed_form_spectra(mk_graph, mk_spec):
    g = mk_graph()
    A, tr = density.density_matrix(g)
    spec = mk_spec()
    assert math.isclose(tr, float(np.sum(spec)), rel_tol=1e-13)
    assert np.allclose(np.sort(np.linalg.eigvalsh(A.toarray())), np.sort(spec / tr), atol=1e-13)
    assert math.isclose(entropy.dense_entropy(A), entropy.entropy_from_laplacian_spectrum(spec),
                        rel_tol=1e-12)


@pytest.mark.parametrize("n", [2, 3, 10, 64])
def test_complete_graph_entropy_is_log_n_minus_1(n):
    A, _ = density.density_matrix(G.complete(n))
    assert math.isclose(entropy.dense_entropy(A), math.log(n - 1), rel_tol=1e-12, abs_tol=1e-14)


def test_large_grid_closed_form_is_consistent():
    # the closed form for a 1024 x 1024 grid (n = 2^20, the largest size of the
    # scaling study) is finite and below log n
    S = entropy.entropy_from_laplacian_spectrum(entropy.spectrum_grid(1024, 1024))
    assert 0 < S < math.log(1024 * 1024)


def test_invariants_trace_one_and_entropy_range():
    for seed in range(4):
        g = G.erdos_renyi(120, 0.05, seed)
        A, _ = density.density_matrix(g)
        assert math.isclose(A.diagonal().sum(), 1.0, rel_tol=1e-14)
        lam = np.linalg.eigvalsh(A.toarray())
        assert lam.min() > -1e-14
        rank = int(np.sum(lam > 1e-12))
        S = entropy.dense_entropy(A)
        assert 0.0 <= S <= math.log(rank) + 1e-12


def test_pure_state_and_maximally_mixed():
    # S = 0 iff pure state; S = log n iff rho = I/n (Section 2)
    v = np.random.default_rng(1).standard_normal(6)
    P = np.outer(v, v) / (v @ v)
    assert abs(entropy.dense_entropy(P)) < 1e-13
    assert math.isclose(entropy.dense_entropy(np.eye(6) / 6), math.log(6), rel_tol=1e-14)


def test_scaling_identity():
    # eq. entropy_normalization: S(gamma A) = gamma S(A) - gamma log(gamma) tr(A)
    A, _ = density.density_matrix(G.barabasi_albert(80, 3, 2))
    L = A.toarray() * 3.7
    for gamma in (0.25, 1.0 / 3.7, 2.0):
        lhs = entropy.dense_entropy(gamma * L)
        rhs = entropy.scaled_entropy(entropy.dense_entropy(L), gamma, float(np.trace(L)))
        assert math.isclose(lhs, rhs, rel_tol=1e-12, abs_tol=1e-12)


def test_f_entropy_convention():
    x = np.array([-1e-18, 0.0, 1.0, math.exp(-1), 0.5])
    want = [0.0, 0.0, 0.0, math.exp(-1), 0.5 * math.log(2)]
    assert np.allclose(entropy.f_entropy(x), want, atol=1e-16)
