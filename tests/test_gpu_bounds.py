"""A-posteriori bounds of Theorem 4.4 on the GPU (vne_quadrature_bounds) vs
the oracle's evaluation of the same g_m over the same points, on Lanczos
tridiagonals of small graphs; and the bracket itself: the GPU bounds enclose
the exact quadrature error from the dense f(A)."""
import numpy as np
import pytest

from oracle import bounds, density, entropy, krylov, rng
from paper_2212_09642_gb300 import graphs, vne

pytestmark = pytest.mark.gpu


def _case(g, seed, ms):
    A, _ = density.density_matrix(g)
    lam = np.linalg.eigvalsh(A.toarray())
    F = entropy.dense_matrix_function(A)
    b = rng.rademacher(seed, g.n, 0, 1)[:, 0]
    c = krylov.desingularize(b)
    exact = float(c @ F @ c)
    out = []
    for m in ms:
        psi, alpha, beta = krylov.lanczos_quadform(A, b, m, reorth="full")
        out.append((m, psi, np.asarray(alpha), np.asarray(beta), float(c @ c)))
    return lam[1], lam[-1], exact, out


@pytest.mark.parametrize("name,g,seed", [
    ("WS400", graphs.watts_strogatz(400, 6, 0.3, 4), 6),
    ("BA600", graphs.barabasi_albert(600, 3, 2), 3),
])
def test_bounds_match_oracle_and_bracket(vctx, name, g, seed):
    l2, ln, exact, runs = _case(g, seed, (3, 6, 10, 16, 24))
    grid = 3000
    for m, psi, alpha, beta, nb in runs:
        if len(alpha) < m:
            continue  # breakdown: exact
        lo, hi, est = vne.vne_quadrature_bounds(vctx, alpha[None, :], beta[None, :m], np.array([nb]), 1.0,
                                                l2, ln, grid)
        rlo, rhi, rest = bounds.posterior_bounds(alpha, beta[:m], nb, l2, ln, grid=grid)
        # g_m is a sum over the Ritz values whose terms cancel to ~1e-9 of
        # their size by m = 16, so two correct evaluations (the GPU's
        # eigenpairs by bisection and twisted factorisation, the oracle's by
        # a dense solver) agree to ~1e-7 of max |g_m|; once the error itself
        # reaches rounding level (1e-12 of psi) both bounds are noise
        floor = 1e-12 * abs(psi)
        assert abs(hi[0] - rhi) <= 1e-6 * rhi + floor, (m, hi[0], rhi)
        # the minimum of |g_m| is sensitive to where the grid points fall near
        # a sign change of g_m: compare it on the scale of the maximum
        assert abs(lo[0] - rlo) <= 1e-6 * rhi + floor, (m, lo[0], rlo)
        err = abs(psi - exact)
        assert lo[0] <= err * (1 + 1e-6) + floor
        assert err <= hi[0] * (1 + 1e-6) + floor
        assert lo[0] <= est[0] <= hi[0]


def test_bounds_zero_after_breakdown(vctx):
    # K_n: the Krylov space of a desingularised vector is invariant after one step
    g = graphs.complete(30)
    A, _ = density.density_matrix(g)
    b = rng.rademacher(1, g.n, 0, 1)[:, 0]
    psi, alpha, beta = krylov.lanczos_quadform(A, b, 4, reorth="full")
    m = 4
    a = np.zeros((1, m))
    bb = np.zeros((1, m))
    a[0, :len(alpha)] = alpha
    bb[0, :min(len(beta), m)] = np.asarray(beta)[:m]
    lo, hi, est = vne.vne_quadrature_bounds(vctx, a, bb, np.array([1.0]), 1.0, 0.01, 0.1, 100)
    assert lo[0] == 0.0 and hi[0] == 0.0 and est[0] == 0.0
    with pytest.raises(vne.VneError):
        vne.vne_quadrature_bounds(vctx, a, bb, np.array([1.0]), 1.0, 0.0, 0.1, 100)


def test_adaptive_lanczos_stops_early_with_parity(vctx):
    """quad_tol > 0: the block stops at the first check where every column's
    Theorem 4.4 estimate is below quad_tol |psi|; the quadratures are then the
    oracle's at that step count, and close to the converged ones."""
    g = graphs.barabasi_albert(3000, 3, 5)
    A, _ = density.density_matrix(g)
    mat = vne.matrix_from_graph(vctx, g, fp64=True)
    try:
        opt = vne.options(quad_tol=1e-8, check_every=4)
        est, se, psi = vne.vne_entropy_hutchinson(vctx, mat, 24, 120, 17, opt=opt, want_psi=True)
        steps = vne.vne_ctx_last_steps(vctx)
        full, _, psi_full = vne.vne_entropy_hutchinson(vctx, mat, 24, 120, 17, want_psi=True)
        assert vne.vne_ctx_last_steps(vctx) == 120
    finally:
        vne.vne_matrix_destroy(mat)
    assert 4 <= steps < 120 and steps % 4 == 0, steps
    X = rng.rademacher(17, g.n, 0, 24)
    nA = density.gershgorin_norm(A)
    for j in range(24):
        ref = krylov.lanczos_quadform(A, X[:, j], steps, reorth="full", norm_A=nA)[0]
        assert abs(psi[j] - ref) <= 1e-10 * abs(ref)
        assert abs(psi[j] - psi_full[j]) <= 1e-6 * abs(psi_full[j])
