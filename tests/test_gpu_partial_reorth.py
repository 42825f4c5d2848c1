"""Partial reorthogonalisation (vne_options.reorth = 2, Simon's omega
recurrence) against the oracle running the same policy with the rounding
unit of the path's vector precision.

What the policy promises is semi-orthogonality (|v_i . v_k| <= sqrt(eps)),
which keeps the Ritz values of T_m those of a fully orthogonal run: the
converged top eigenvalue of A appears once in T_m instead of as a ghost pair.
It does not make the alpha / beta sequences of two correct implementations
agree beyond the steps before orthogonality starts to decay (rounding
differences grow from there on), so these are compared over the first 20
steps only.  Checked: psi to 1e-10 (FP64) and 1e-5 (FP32), alpha / beta over
the first 20 steps (FP64), a single copy of lambda_max in the device's T_m
(within 1e-8 of it in FP64, 1e-5 in FP32) where the plain recurrence on the
device has two or more, and run-to-run bit-identity."""
import numpy as np
import pytest

from oracle import density, krylov, rng
from paper_2212_09642_gb300 import graphs, vne

pytestmark = pytest.mark.gpu

M_STEPS = 120


def _oracle(A, X, m, reorth, eps):
    nA = density.gershgorin_norm(A)
    out = []
    for j in range(X.shape[1]):
        c = krylov.desingularize(X[:, j])
        a, b, _ = krylov.lanczos(A, c, m, reorth=reorth, norm_A=nA, eps=eps)
        out.append((krylov.gauss_quadrature(a, b[:-1], float(c @ c)), a, b))
    return out


def _copies_of_lambda_max(ab, m, lmax, rel):
    a, b = ab[:m], ab[m:2 * m]
    k = int(np.count_nonzero(a)) if np.all(b[:m - 1] > 0) else int(np.argmin(b[:m - 1] > 0)) + 1
    T = np.diag(a[:k]) + np.diag(b[:k - 1], 1) + np.diag(b[:k - 1], -1)
    th = np.linalg.eigvalsh(T)
    return int(np.sum(np.abs(th - lmax) <= rel * lmax))


@pytest.mark.parametrize("fp64", [True, False])
def test_partial_reorth_matches_oracle_and_removes_ghosts(vctx, fp64):
    g = graphs.erdos_renyi(400, 0.05, 3)
    A, _ = density.density_matrix(g)
    X = rng.rademacher(1, 400, 0, 5)
    lmax = float(np.linalg.eigvalsh(A.toarray())[-1])
    mat = vne.matrix_from_graph(vctx, g, fp64=fp64)
    try:
        psi, ab = vne.vne_quadform_batch(vctx, mat, X, M_STEPS, opt=vne.options(reorth=2), want_alpha_beta=True)
        psi2, _ = vne.vne_quadform_batch(vctx, mat, X, M_STEPS, opt=vne.options(reorth=2), want_alpha_beta=True)
        _, ab0 = vne.vne_quadform_batch(vctx, mat, X, M_STEPS, opt=vne.options(reorth=0), want_alpha_beta=True)
    finally:
        vne.vne_matrix_destroy(mat)
    assert np.array_equal(psi, psi2)
    ref = _oracle(A, X, M_STEPS, "partial", 2.0 ** -53 if fp64 else 2.0 ** -24)
    nA = density.gershgorin_norm(A)
    tol = 1e-10 if fp64 else 1e-5
    for j, (p_ref, a_ref, b_ref) in enumerate(ref):
        assert abs(psi[j] - p_ref) <= tol * abs(p_ref)
        if fp64:
            assert np.max(np.abs(ab[j, :20] - a_ref[:20])) <= 1e-10 * nA
            assert np.max(np.abs(ab[j, M_STEPS:M_STEPS + 20] - b_ref[:20])) <= 1e-10 * nA
        # within the accuracy the vector precision allows, the converged top
        # eigenvalue appears once with the policy and as ghost copies without
        win = 1e-8 if fp64 else 1e-5
        assert _copies_of_lambda_max(ab[j], M_STEPS, lmax, win) == 1
        assert _copies_of_lambda_max(ab0[j], M_STEPS, lmax, win) >= 2


def test_partial_reorth_fp32_at_larger_size(vctx):
    g = graphs.barabasi_albert(20000, 4, 3)
    A, _ = density.density_matrix(g)
    X = rng.rademacher(2, g.n, 0, 6)
    mat = vne.matrix_from_graph(vctx, g, fp64=False, reorder=True)
    try:
        psi = vne.vne_quadform_batch(vctx, mat, X, 60, opt=vne.options(reorth=2))
    finally:
        vne.vne_matrix_destroy(mat)
    ref = np.array([r[0] for r in _oracle(A, X, 60, "partial", 2.0 ** -24)])
    assert np.max(np.abs(psi - ref) / np.abs(ref)) <= 1e-5
