"""GPU kernel parity through the C ABI: probe generator, SpMM, quadrature."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import density, krylov, rng
from paper_2212_09642_gb300 import graphs, vne

pytestmark = pytest.mark.gpu


def _graphs():
    iso = graphs.from_edges(300, np.array([1, 2, 3, 10]), np.array([2, 3, 1, 11]))  # mostly isolated nodes
    star = graphs.star(5000)  # one row with 4999 nonzeros (split into chunks)
    return [graphs.erdos_renyi(3000, 0.003, 2), graphs.barabasi_albert(20000, 4, 3), star, iso,
            graphs.disjoint_union([graphs.star(700), graphs.watts_strogatz(900, 6, 0.2, 1)])]


def test_rademacher_bit_exact(vctx):
    import torch
    n, k, c0 = 5003, 37, 11
    out = torch.empty((n, k), dtype=torch.float64, device="cuda")
    vne.vne_rademacher(vctx, 1234, n, c0, k, out, fp64=True)
    want = rng.rademacher(1234, n, c0, k)
    assert np.array_equal(out.cpu().numpy(), want)
    out32 = torch.empty((n, k), dtype=torch.float32, device="cuda")
    vne.vne_rademacher(vctx, 99, n, 0, k, out32, fp64=False)
    assert np.array_equal(out32.cpu().numpy().astype(np.float64), rng.rademacher(99, n, 0, k))


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("reorder", [False, True, "rcm"])
def test_spmm_matches_scipy(vctx, fp64, reorder):
    import torch
    dt = torch.float64 if fp64 else torch.float32
    for g in _graphs():
        A, _ = density.density_matrix(g)
        k = 5
        X = np.random.default_rng(g.n).standard_normal((g.n, k))
        mat = vne.matrix_from_graph(vctx, g, fp64=fp64, reorder=reorder)
        try:
            Xd = torch.tensor(X, dtype=dt, device="cuda")
            Yd = torch.empty_like(Xd)
            vne.vne_spmm(vctx, mat, Xd, Yd, k)
            Y = Yd.cpu().numpy().astype(np.float64)
        finally:
            vne.vne_matrix_destroy(mat)
        ref = A @ X
        scale = np.abs(A) @ np.abs(X) + 1e-300
        tol = 1e-13 if fp64 else 1e-5
        assert np.max(np.abs(Y - ref) / scale) < tol


def test_tridiag_quadrature_matches_oracle(vctx):
    r = np.random.default_rng(3)
    count, m = 200, 60
    a = r.uniform(0, 1e-3, (count, m))
    b = r.uniform(0, 5e-4, (count, m))
    b[::7, 13] = 0.0           # truncation after row 14
    a[::11, :] = 2e-4          # clustered Toeplitz spectra
    b[::11, :] = 1e-4
    norm2 = r.uniform(1, 100, count)
    got = vne.vne_tridiag_quadrature(vctx, a, b, norm2, 3.0)
    for c in range(count):
        bb = b[c, :m - 1]
        z = np.where(bb == 0)[0]
        kk = m if len(z) == 0 else z[0] + 1
        want = krylov.gauss_quadrature(3.0 * a[c, :kk], 3.0 * bb[:kk - 1], norm2[c])
        assert abs(got[c] - want) <= 1e-12 * abs(want)


def _wilkinson_plus(k):
    n = 2 * k + 1
    return np.abs(np.arange(n) - k).astype(float) + 1.0, np.ones(n - 1)


def _ghost_tridiagonal(g, m, seed):
    """Lanczos tridiagonal without reorthogonalisation: converged Ritz values
    reappear as near-identical copies (clusters down to rounding level)."""
    A, _ = density.density_matrix(g)
    x = rng.rademacher(seed, g.n, 0, 1)[:, 0]
    _, al, be = krylov.lanczos_quadform(A, x, m, reorth="none")
    return np.asarray(al), np.asarray(be[:len(al) - 1])


def test_tridiag_quadrature_clusters_and_grading(vctx):
    """Tight eigenvalue pairs (Wilkinson W+), Lanczos ghost clusters, graded
    and nearly decoupled tridiagonals, a 1 x 1 block: the quadrature matches
    the oracle's eigendecomposition to 1e-12 relative."""
    cases = []
    for k in (10, 20, 30, 63):
        a, b = _wilkinson_plus(k)
        cases.append((a / (a.max() + 2.5), b / (a.max() + 2.5)))
    g = graphs.barabasi_albert(3000, 3, 1)
    for m, seed in ((60, 1), (100, 2), (128, 3)):
        cases.append(_ghost_tridiagonal(g, m, seed))
    r = np.random.default_rng(11)
    for _ in range(6):
        n = int(r.integers(20, 120))
        cases.append((10.0 ** r.uniform(-8, 0, n), 10.0 ** r.uniform(-10, -1, n - 1)))   # graded
        cases.append((r.random(n), r.random(n - 1) * 1e-9 + 1e-14))                      # nearly decoupled
    cases.append((np.array([0.25]), np.zeros(0)))
    m = max(len(a) for a, _ in cases)
    count = len(cases)
    A = np.zeros((count, m))
    B = np.zeros((count, m))
    for c, (a, b) in enumerate(cases):
        A[c, :len(a)] = a
        B[c, :len(b)] = b
        # rows past the block stay decoupled: beta = 0 ends it
    norm2 = np.ones(count)
    got = vne.vne_tridiag_quadrature(vctx, A, B, norm2, 1.0)
    again = vne.vne_tridiag_quadrature(vctx, A, B, norm2, 1.0)
    assert np.array_equal(got, again)
    for c, (a, b) in enumerate(cases):
        want = krylov.gauss_quadrature(a, b, 1.0)
        # eigenvalues are backward stable: an absolute floor of a few ulps of
        # ||T|| covers graded blocks whose quadrature is tiny
        tnorm = np.max(np.abs(a) + np.r_[np.abs(b), 0.0] + np.r_[0.0, np.abs(b)])
        assert abs(got[c] - want) <= 1e-12 * abs(want) + 64 * np.finfo(float).eps * tnorm, (c, len(a), got[c], want)


def test_measure_gather_probe(vctx):
    gbs = vne.vne_measure_gather(vctx, 16 << 20, 64, 1 << 20, 0, 1)
    assert gbs > 0
    with pytest.raises(vne.VneError):
        vne.vne_measure_gather(vctx, 16 << 20, 48, 1 << 20, 0, 1)
