"""Rational Krylov quadrature by multi-shift CG (Sections 4, 4.2, 5.3): GPU
(C ABI) vs the oracle's dense-solve rational quadrature on identical
vectors and poles.

Tolerances: 1e-10 relative in the FP64 path (CG driven to 1e-13) and 1e-5
in the mixed path (FP32 vectors, CG to the default 1e-8 recursive residual).
The oracle solves the shifted systems directly and drops a spanning vector
only at the rounding level of its norm (1e-12); the GPU orthonormalises
through Gram matrices (Cholesky-QR2), which cannot resolve remainders below
the square root of the rounding unit, so it drops a pole direction whose
remainder is below 1e-6 (FP64) or 1e-3 (FP32) of its norm.  Both readings
give the same psi within these tolerances on every case here."""
import math

import numpy as np
import pytest

from oracle import coloring, density, entropy, krylov, rational, rng
from paper_2212_09642_gb300 import graphs, vne

pytestmark = pytest.mark.gpu


def _cases():
    return [("WS600", graphs.watts_strogatz(600, 6, 0.2, 2)),
            ("BA2000", graphs.barabasi_albert(2000, 3, 1)),
            ("grid", graphs.grid2d(30, 40)),
            ("RGG2000", graphs.random_geometric(2000, graphs.rgg_radius_for_degree(2000, 8), 3))]


@pytest.mark.parametrize("name,g", _cases())
@pytest.mark.parametrize("fp64", [True, False])
def test_rational_quadform_parity(vctx, name, g, fp64):
    A, _ = density.density_matrix(g)
    sh = rational.default_shifts(A)
    X = rng.rademacher(4, g.n, 0, 9)
    mat = vne.matrix_from_graph(vctx, g, fp64=fp64)
    tol_cg = 1e-13 if fp64 else 1e-8
    try:
        psi, its, res = vne.vne_quadform_rational(vctx, mat, X, sh, opt=vne.options(cg_tol=tol_cg))
    finally:
        vne.vne_matrix_destroy(mat)
    ref = np.array([rational.rational_quadform(A, X[:, j], sh) for j in range(X.shape[1])])
    rel = np.abs(psi - ref) / np.abs(ref)
    assert rel.max() <= (1e-10 if fp64 else 1e-5), rel.max()
    assert np.all(res <= tol_cg * 1.0000001)
    # larger shifts converge in fewer iterations (they are retired first)
    order = np.argsort(sh)
    assert np.all(np.diff(its[order].max(axis=1)) <= 0)


def test_rational_complete_graph_exact(vctx):
    g = graphs.complete(40)
    A, _ = density.density_matrix(g)
    X = rng.rademacher(2, 40, 0, 3)
    mat = vne.matrix_from_graph(vctx, g, fp64=True)
    try:
        psi, _, _ = vne.vne_quadform_rational(vctx, mat, X, None, num_shifts=8)
    finally:
        vne.vne_matrix_destroy(mat)
    lam = 1.0 / 39
    c = krylov.desingularize(X)
    want = np.sum(c * c, axis=0) * (-lam * math.log(lam))
    assert np.max(np.abs(psi - want) / want) <= 1e-10


@pytest.mark.parametrize("fp64", [True, False])
def test_rational_probing(vctx, fp64):
    g = graphs.grid2d(30, 40)
    A, _ = density.density_matrix(g)
    col = coloring.greedy_distance_coloring(g, 2)
    sh = rational.default_shifts(A)
    mat = vne.matrix_from_graph(vctx, g, fp64=fp64)
    try:
        est, s = vne.vne_entropy_probing(vctx, mat, None, 2, 0, shifts=sh,
                                         opt=vne.options(cg_tol=1e-13 if fp64 else 1e-8))
    finally:
        vne.vne_matrix_destroy(mat)
    V = np.zeros((g.n, col.max() + 1))
    V[np.arange(g.n), col] = 1.0
    ref = sum(rational.rational_quadform(A, V[:, l], sh) for l in range(V.shape[1]))
    assert s == V.shape[1]
    assert abs(est - ref) <= (1e-10 if fp64 else 1e-5) * ref
    assert est <= entropy.dense_entropy(A) * (1 + 1e-7)


# ---- switching rule (Section 5.3): polynomial part chosen per block ----

def _oracle_rule_k(A, X, k_max=16):
    ks = []
    for j in range(X.shape[1]):
        c = krylov.desingularize(X[:, j])
        est, _ = rational.polynomial_estimates(A, c, k_max)
        ks.append(rational.switch_index(est))
    return max(ks)


@pytest.mark.parametrize("name,g", _cases())
@pytest.mark.parametrize("fp64", [True, False])
def test_mixed_switching_parity(vctx, name, g, fp64):
    """n_inf_poles = -1: the device takes the polynomial dimension k from the
    seed CG's coefficients (CG-Lanczos relation) and its Theorem 4.4
    estimates, spans K_k(A, c) by the CG residuals and adds the pole
    directions.  FP64: k equals the oracle's (Lanczos in FP64, same rule, the
    block's largest k); both paths: psi equals the oracle's mixed quadrature
    with the device's k."""
    A, _ = density.density_matrix(g)
    sh = rational.default_shifts(A)
    X = rng.rademacher(6, g.n, 0, 7)
    mat = vne.matrix_from_graph(vctx, g, fp64=fp64)
    tol_cg = 1e-13 if fp64 else 1e-8
    try:
        psi, its, res = vne.vne_quadform_rational(vctx, mat, X, sh, opt=vne.options(cg_tol=tol_cg, n_inf_poles=-1))
        k = vne.vne_ctx_last_poly_dim(vctx)
    finally:
        vne.vne_matrix_destroy(mat)
    assert 1 <= k <= 16
    if fp64:
        assert k == _oracle_rule_k(A, X), (name, k)
    ref = np.array([rational.mixed_quadform(A, X[:, j], sh, k_poly=k, k_max=16)[0] for j in range(X.shape[1])])
    rel = np.abs(psi - ref) / np.abs(ref)
    assert rel.max() <= (1e-10 if fp64 else 1e-5), (k, rel.max())
    assert np.all(res <= tol_cg * 1.0000001)


def test_mixed_complete_graph_one_step(vctx):
    """K_n: the polynomial estimate is 0 after one step (invariant Krylov
    space), so the polynomial part is K_1 = span{c} and psi is exact."""
    g = graphs.complete(40)
    A, _ = density.density_matrix(g)
    X = rng.rademacher(3, 40, 0, 3)
    mat = vne.matrix_from_graph(vctx, g, fp64=True)
    try:
        psi, _, _ = vne.vne_quadform_rational(vctx, mat, X, None, num_shifts=8, opt=vne.options(n_inf_poles=-1))
        k = vne.vne_ctx_last_poly_dim(vctx)
    finally:
        vne.vne_matrix_destroy(mat)
    lam = 1.0 / 39
    c = krylov.desingularize(X)
    want = np.sum(c * c, axis=0) * (-lam * math.log(lam))
    assert k == 1
    assert np.allclose(psi, want, rtol=1e-10, atol=0)
