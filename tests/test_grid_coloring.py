"""The lattice colouring of the 2D grid used by the scaling study: a valid
distance-d colouring (brute-force check of every pair within distance d) with
exactly ceil((d+1)^2 / 2) colours, which no distance-d colouring can beat (the
grid contains that many nodes pairwise within distance d)."""
import numpy as np
import pytest

from oracle import coloring
from paper_2212_09642_gb300 import graphs, grid_coloring


@pytest.mark.parametrize("d", range(1, 9))
def test_lattice_coloring_valid_and_optimal(d):
    rows, cols = 30, 31
    g = graphs.grid2d(rows, cols)
    c = grid_coloring.lattice_coloring(rows, cols, d)
    assert coloring.is_distance_coloring(g, c, d)
    assert len(np.unique(c)) == grid_coloring.colors_needed(d) == c.max() + 1
    # a clique of the d-th power graph with ceil((d+1)^2/2) nodes: the L1 ball
    # of radius d/2 (d even) or its union with a shifted copy (d odd)
    r = d // 2
    ball = [(a, b) for a in range(-r, r + 2) for b in range(-r, r + 2)
            if abs(a) + abs(b) <= r or (d % 2 == 1 and abs(a - 1) + abs(b) <= r)]
    assert len(ball) == grid_coloring.colors_needed(d)
    assert all(abs(p[0] - q[0]) + abs(p[1] - q[1]) <= d for p in ball for q in ball)
