"""Sanity of the seeded graph inputs (symmetric simple CSR patterns)."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2212_09642_gb300 import graphs as G


def _check_simple_symmetric(g):
    assert g.rowptr.shape == (g.n + 1,) and g.rowptr[0] == 0
    assert g.col.dtype == np.int32 and g.col.size == g.nnz
    rows = np.repeat(np.arange(g.n), g.degrees)
    assert np.all(rows != g.col), "self-loop"
    for i in range(min(g.n, 500)):
        c = g.col[g.rowptr[i]:g.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0), "unsorted or duplicate columns"
    W = sp.csr_matrix((np.ones(g.nnz), g.col, g.rowptr), shape=(g.n, g.n))
    assert (W != W.T).nnz == 0


@pytest.mark.parametrize("make", [
    lambda: G.erdos_renyi(500, 0.02, 1),
    lambda: G.barabasi_albert(2000, 4, 3),
    lambda: G.watts_strogatz(1000, 6, 0.1, 5),
    lambda: G.random_geometric(3000, G.rgg_radius_for_degree(3000, 6), 4),
    lambda: G.grid2d(7, 9), lambda: G.grid2d(5, 6, periodic=True),
    lambda: G.hypercube(5), lambda: G.complete_bipartite(3, 4), lambda: G.star(9),
])
def test_generators_give_simple_symmetric_patterns(make):
    _check_simple_symmetric(make())


def test_generators_are_deterministic():
    a = G.barabasi_albert(3000, 4, 11)
    b = G.barabasi_albert(3000, 4, 11)
    assert np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.col, b.col)


def test_barabasi_albert_edge_count_and_min_degree():
    n, m = 5000, 4
    g = G.barabasi_albert(n, m, 3)
    assert g.nnz // 2 == m * (m + 1) // 2 + (n - m - 1) * m
    assert g.degrees.min() >= m


def test_erdos_renyi_edge_count_statistics():
    n, p = 400, 0.05
    counts = [G.erdos_renyi(n, p, s).nnz // 2 for s in range(40)]
    mean = p * n * (n - 1) / 2
    assert abs(np.mean(counts) - mean) < 4 * np.sqrt(mean / 40)


def test_rgg_mean_degree():
    n = 20000
    g = G.random_geometric(n, G.rgg_radius_for_degree(n, 6.0), 4)
    assert 5.4 < g.nnz / n < 6.2  # boundary effects lower the mean slightly
