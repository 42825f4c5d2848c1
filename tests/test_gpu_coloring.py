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


def test_large_balls_searched_by_a_cta(vctx):
    """Balls too large for a warp's table (d >= 3) are searched by a whole CTA
    with a table in global memory: a star with 1700 leaves (every pair within
    distance 2, so all colours distinct) and a hub joined to 1600 nodes of a
    1800-node cycle, whose neighbours each have 1600 nodes within distance 2."""
    ring = np.arange(1, 1801)
    hub_ring = graphs.from_edges(1801, np.concatenate([np.zeros(1600, dtype=np.int64), ring]),
                                 np.concatenate([np.arange(1, 1601), np.roll(ring, 1)]))
    for g, d in [(graphs.star(1701), 3), (hub_ring, 3), (hub_ring, 4)]:
        mat = vne.matrix_from_graph(vctx, g, reorder=True)
        try:
            got, s, rounds = vne.vne_matrix_coloring(vctx, mat, g.n, d)
        finally:
            vne.vne_matrix_destroy(mat)
        want = coloring.greedy_distance_coloring(g, d)
        assert rounds > 0
        assert np.array_equal(got, want), (g.n, d, int(np.sum(got != want)))
    assert s == int(want.max()) + 1


def test_ball_beyond_the_cta_table_is_refused(vctx):
    """A hub with 200,000 neighbours at d = 3: the radius-2 ball of every leaf
    holds the whole graph, more than a CTA's table; the call reports
    EUNSUPPORTED instead of colouring (the context stays usable)."""
    g = graphs.star(200001)
    mat = vne.matrix_from_graph(vctx, g)
    try:
        with pytest.raises(vne.VneError) as e:
            vne.vne_matrix_coloring(vctx, mat, g.n, 3)
        assert e.value.status == vne.VNE_EUNSUPPORTED
        got, s, rounds = vne.vne_matrix_coloring(vctx, mat, g.n, 1)
    finally:
        vne.vne_matrix_destroy(mat)
    want = np.ones(g.n, dtype=np.int32)
    want[0] = 0  # the hub first (highest degree), then every leaf next to it
    assert s == 2 and np.array_equal(got, want)


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
