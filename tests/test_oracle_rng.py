"""Pins for the counter-based Rademacher generator (oracle side)."""
import os

import numpy as np

from oracle import rng
from paper_2212_09642_gb300 import graphs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed1234567.txt")


def test_splitmix64_known_answer():
    want = [int(l) for l in open(GOLD) if l.strip() and not l.startswith("#")]
    got = [int(x) for x in rng.splitmix64_stream(1234567, len(want))]
    assert got == want


def test_rademacher_entries_and_balance():
    X = rng.rademacher(7, 20000, 0, 8)
    assert set(np.unique(X)) == {-1.0, 1.0}
    # each column is balanced to within 5 standard deviations
    assert np.all(np.abs(X.sum(axis=0)) < 5 * np.sqrt(20000))
    # distinct columns are nearly orthogonal (E[x x^T] = I)
    G = X.T @ X / 20000
    assert np.allclose(np.diag(G), 1.0)
    assert np.max(np.abs(G - np.eye(8))) < 5 / np.sqrt(20000)


def test_rademacher_columns_are_addressed_globally():
    A = rng.rademacher(3, 100, 0, 10)
    B = rng.rademacher(3, 100, 4, 3)
    assert np.array_equal(A[:, 4:7], B)
    C = rng.rademacher(4, 100, 0, 10)
    assert not np.array_equal(A, C)


def test_rademacher_row_relabelling():
    perm = np.random.default_rng(0).permutation(50)
    A = rng.rademacher(9, 50, 0, 4)
    B = rng.rademacher(9, 50, 0, 4, rows=perm)
    assert np.array_equal(A[perm], B)


# ---- Gaussian probes (Box-Muller on the same counters) ----

def test_gaussian_probes_are_standard_normal():
    """10^6 entries: mean, variance and the Kolmogorov-Smirnov distance to
    N(0, 1) at their sampling accuracy; columns uncorrelated; the stream is
    reproducible and the row mapping is honoured."""
    from scipy import stats
    X = rng.gaussian(123, 250_000, 5, 4)
    x = X.ravel()
    N = x.size
    assert abs(x.mean()) < 5.0 / np.sqrt(N)
    assert abs(x.var() - 1.0) < 5.0 * np.sqrt(2.0 / N)
    assert stats.kstest(x, "norm").statistic < 1.63 / np.sqrt(N) * 1.5  # well inside the 1 % level
    C = np.corrcoef(X.T)
    assert np.max(np.abs(C - np.eye(4))) < 5.0 / np.sqrt(X.shape[0])
    assert np.array_equal(X, rng.gaussian(123, 250_000, 5, 4))
    rows = np.array([7, 3, 250_001])
    sub = rng.gaussian(123, 3, 5, 4, rows=rows)
    assert np.array_equal(sub[:2], X[[7, 3]])


def test_gaussian_hutchinson_is_unbiased():
    """E[x^T B x] = tr B for standard normal x: 4000 Gaussian probes of a
    small graph's f(A) average to the dense entropy within 4 standard errors."""
    from oracle import density, entropy
    g = graphs.erdos_renyi(60, 0.15, 3)
    A, _ = density.density_matrix(g)
    F = entropy.dense_matrix_function(A)
    X = rng.gaussian(9, g.n, 0, 4000)
    q = np.einsum("ij,ij->j", X, F @ X)
    S = float(np.trace(F))
    assert abs(q.mean() - S) <= 4.0 * q.std(ddof=1) / np.sqrt(q.size)
