"""Greedy distance-d colouring on the device (vne_matrix_coloring) against the
oracle's sequential Algorithm 1: the same colour at every node (the device
rounds colour a node once all higher-priority nodes of its d-ball have
theirs, which reproduces the sequential sweep exactly), whatever the
relabelling of the stored matrix."""
import numpy as np
import pytest

from oracle import coloring, density, estimators
from paper_2212_09642_gb300 import graphs, vne

pytestmark = pytest.mark.gpu


def _small_graphs():
    iso = graphs.from_edges(300, np.array([1, 2, 3, 10]), np.array([2, 3, 1, 11]))  # mostly isolated nodes
    return [
        ("ER500", graphs.erdos_renyi(500, 0.01, 3)),
        ("BA600", graphs.barabasi_albert(600, 3, 2)),
        ("WS400", graphs.watts_strogatz(400, 6, 0.3, 4)),
        ("RGG900", graphs.random_geometric(900, graphs.rgg_radius_for_degree(900, 6.0), 5)),
        ("grid", graphs.grid2d(17, 23)),
        ("iso", iso),
        ("K2", graphs.complete(2)),
    ]


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("reorder", [False, True, "rcm"])
def test_device_coloring_equals_algorithm_1(vctx, d, reorder):
    for name, g in _small_graphs():
        want = coloring.greedy_distance_coloring(g, d)
        mat = vne.matrix_from_graph(vctx, g, reorder=reorder)
        try:
            got, s, rounds = vne.vne_matrix_coloring(vctx, mat, g.n, d)
        finally:
            vne.vne_matrix_destroy(mat)
        assert rounds > 0, name  # every ball fits: the device path ran
        assert np.array_equal(got, want), (name, d, reorder, int(np.sum(got != want)))
        assert s == int(want.max()) + 1


def test_device_coloring_large_rgg_and_ba(vctx):
    """Thousands of nodes per round and long priority chains (the neighbours of
    a BA hub are pairwise within distance 2): same colours as the oracle."""
    for g, d in [(graphs.random_geometric(30000, graphs.rgg_radius_for_degree(30000, 6.0), 7), 2),
                 (graphs.random_geometric(20000, graphs.rgg_radius_for_degree(20000, 6.0), 8), 3),
                 (graphs.barabasi_albert(20000, 4, 9), 2)]:
        want = coloring.greedy_distance_coloring(g, d)
        mat = vne.matrix_from_graph(vctx, g, reorder=True)
        try:
            got, s, rounds = vne.vne_matrix_coloring(vctx, mat, g.n, d)
        finally:
            vne.vne_matrix_destroy(mat)
        assert rounds > 0
        assert np.array_equal(got, want), (g.n, d, int(np.sum(got != want)))


def test_ball_overflow_uses_host_sweep(vctx):
    """A star with 1700 leaves at d = 3: the hub's neighbourhood does not fit
    the per-warp table, the host sweep runs and gives Algorithm 1's colours
    (all distinct: every pair of nodes is within distance 2)."""
    g = graphs.star(1701)
    mat = vne.matrix_from_graph(vctx, g)
    try:
        got, s, rounds = vne.vne_matrix_coloring(vctx, mat, g.n, 3)
    finally:
        vne.vne_matrix_destroy(mat)
    assert rounds == 0
    assert np.array_equal(got, coloring.greedy_distance_coloring(g, 3))
    assert s == g.n


def test_probing_without_colouring_uses_algorithm_1(vctx):
    """vne_entropy_probing with coloring = NULL gives the estimate of the same
    call with the oracle's colouring passed in, bit for bit."""
    g = graphs.random_geometric(4000, graphs.rgg_radius_for_degree(4000, 6.0), 11)
    col = coloring.greedy_distance_coloring(g, 2)
    for reorder in (False, "rcm"):
        mat = vne.matrix_from_graph(vctx, g, fp64=True, reorder=reorder)
        try:
            a, sa = vne.vne_entropy_probing(vctx, mat, None, 2, 40)
            b, sb = vne.vne_entropy_probing(vctx, mat, col, 2, 40)
        finally:
            vne.vne_matrix_destroy(mat)
        assert sa == sb == int(col.max()) + 1
        assert a == b
    A, _ = density.density_matrix(g)
    ref, _ = estimators.probing(A, col, 40)
    assert abs(a - ref) <= 1e-10 * abs(ref)
