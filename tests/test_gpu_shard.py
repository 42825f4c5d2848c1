"""Probe ranges on the GPU: the psi values of probe ranges evaluated
separately (as ranks of a sharded estimate would, one after another here)
are bit-identical to the same probes of one full run, for both precisions;
the single-rank sharded driver returns the full-run estimate."""
import numpy as np
import pytest

from paper_2212_09642_gb300 import graphs, shard, vne

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fp64", [False, True])
def test_probe_ranges_bit_identical(vctx, fp64):
    g = graphs.barabasi_albert(5000, 3, 21)
    total, m, seed = 37, 20, 123
    mat = vne.matrix_from_graph(vctx, g, fp64=fp64)
    try:
        _, _, full = vne.vne_entropy_hutchinson(vctx, mat, total, m, seed, want_psi=True)
        parts = []
        for rank in range(3):
            b, c = shard.probe_range(total, 3, rank)
            _, _, psi = vne.vne_entropy_hutchinson(vctx, mat, c, m, seed, opt=vne.options(probe_offset=b),
                                                   want_psi=True)
            parts.append(psi)
        est, se, n = shard.hutchinson(vctx, mat, total, m, seed)
        ref_est, ref_se = vne.vne_entropy_hutchinson(vctx, mat, total, m, seed)
    finally:
        vne.vne_matrix_destroy(mat)
    assert np.array_equal(np.concatenate(parts), full)
    assert n == total
    assert abs(est - ref_est) <= 1e-14 * abs(ref_est)
    assert abs(se - ref_se) <= 1e-10 * ref_se


def test_negative_probe_offset_rejected(vctx):
    g = graphs.erdos_renyi(500, 0.02, 1)
    mat = vne.matrix_from_graph(vctx, g)
    try:
        with pytest.raises(vne.VneError):
            vne.vne_entropy_hutchinson(vctx, mat, 4, 5, 1, opt=vne.options(probe_offset=-1))
    finally:
        vne.vne_matrix_destroy(mat)
