"""Probing with the heuristic choice of d on the 2D grid with the optimal
lattice colouring (the scaling study's setting), through the colouring
callback of vne_entropy_probing_auto: T_1..T_3 and the choice of d against
the oracle's run with the same colourings, and the estimate against the
grid's closed-form entropy (Cartesian-product spectrum) up to n = 2^20."""
import numpy as np
import pytest

from oracle import density, entropy, probing
from paper_2212_09642_gb300 import graphs, grid_coloring, vne

pytestmark = pytest.mark.gpu


def _closed_form(rows, cols):
    return entropy.entropy_from_laplacian_spectrum(entropy.spectrum_grid(rows, cols))


def test_grid_lattice_colouring_matches_oracle(vctx):
    side, eps = 48, 1e-3
    g = graphs.grid2d(side, side)
    colfn = lambda d: grid_coloring.lattice_coloring(side, side, d)
    A, _ = density.density_matrix(g)
    ref, rrep = probing.probing_auto(A, g, eps, 128, check=2, d_max=32, coloring=colfn)
    mat = vne.matrix_from_graph(vctx, g, fp64=True, reorder=True)
    try:
        est, rep = vne.vne_entropy_probing_auto(vctx, mat, eps, 128, 32, opt=vne.options(check_every=2),
                                                coloring=colfn)
    finally:
        vne.vne_matrix_destroy(mat)
    assert rep["colors_d"] == [grid_coloring.colors_needed(d) for d in (1, 2, 3)]
    # same stopping steps as the oracle here (no estimate near its threshold)
    assert rep["steps_d"] == [rrep["steps"][d] for d in (1, 2, 3)]
    assert np.allclose(rep["T"], rrep["T"][:3], rtol=1e-10, atol=0)
    assert (rep["d"], rep["rule"]) == (rrep["d"], rrep["rule"])
    assert abs(est - ref) <= 1e-10 * ref
    S = _closed_form(side, side)
    assert abs(est - S) <= eps * S


@pytest.mark.parametrize("side", [256, 1024])
def test_grid_probing_against_closed_form(vctx, side):
    eps = 1e-3
    mat = vne.matrix_from_graph(vctx, graphs.grid2d(side, side), fp64=False, reorder=True)
    try:
        est, rep = vne.vne_entropy_probing_auto(
            vctx, mat, eps, 128, 32, opt=vne.options(check_every=2),
            coloring=lambda d: grid_coloring.lattice_coloring(side, side, d))
    finally:
        vne.vne_matrix_destroy(mat)
    S = _closed_form(side, side)
    assert abs(est - S) <= eps * S, (side, est, S, rep)


def test_colouring_callback_failure_is_reported(vctx):
    g = graphs.grid2d(20, 20)
    mat = vne.matrix_from_graph(vctx, g)
    try:
        with pytest.raises(vne.VneError):
            vne.vne_entropy_probing_auto(vctx, mat, 1e-3, 40, 8, coloring=lambda d: np.full(7, -1))
    finally:
        vne.vne_matrix_destroy(mat)
