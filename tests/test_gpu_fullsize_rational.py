"""Rational-Krylov probing at the C3 workload's full size: the random
geometric graph n = 4e6 (radius sqrt(6 / (pi n)), seed 4), relabelled by
reverse Cuthill-McKee and coloured on the device at distance 2, with the
autotuned schedule, 8 default poles + 2 at infinity and multi-shift CG to
1e-8 in FP32, as the benchmark runs it.  Colour classes 0..3 are checked
against the FP64 oracle values in tests/golden/rgg4e6_rational_psi.txt
(written by tests/golden/make_rgg4e6_rational.py from the oracle alone:
greedy distance-2 colouring, rational Krylov with CG to 1e-10): the device's
classes are the oracle's (size and sums of node ids) and psi agrees to
1e-5 (the mixed path's tolerance)."""
import os

import numpy as np
import pytest

from paper_2212_09642_gb300 import graphs, vne

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rgg4e6_rational_psi.txt")


def _golden():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    return [(int(c), int(sz), int(s1), int(s2), float(psi)) for c, sz, s1, s2, psi in rows]


def test_rgg4e6_rational_colour_classes_against_oracle(vctx):
    n = 4_000_000
    g = graphs.random_geometric(n, graphs.rgg_radius_for_degree(n, 6), 4)
    mat = vne.matrix_from_graph(vctx, g, fp64=False, reorder="rcm")
    try:
        colors, s, _ = vne.vne_matrix_coloring(vctx, mat, n, 2)
        vne.vne_autotune(vctx, mat, s, 8)
        gold = _golden()
        X = np.zeros((n, len(gold)))
        for col, size, s1, s2, _ in gold:
            ids = np.nonzero(colors == col)[0].astype(np.int64)
            assert (ids.size, int(ids.sum()), int((ids * ids).sum())) == (size, s1, s2), col
            X[ids, col] = 1.0
        psi, _, res = vne.vne_quadform_rational(vctx, mat, X, None, num_shifts=8,
                                                opt=vne.options(cg_tol=1e-8, n_inf_poles=2))
    finally:
        vne.vne_matrix_destroy(mat)
    ref = np.array([r[4] for r in gold])
    assert np.max(np.abs(psi - ref) / ref) <= 1e-5, (psi, ref)
    assert np.all(res <= 1e-8 * 1.0000001)
