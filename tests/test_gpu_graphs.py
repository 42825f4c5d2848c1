"""CUDA-graph replay of the Lanczos step loop: a loop is captured the second
time the same launch parameters are seen and replayed from then on.  Replays
must give bit-identical results to direct launches (the graph holds the same
kernels with the same arguments), on the plain FP32 path, the FP64 path with
full reorthogonalisation, Hutch++ (two blocks per call) and the batched
packing, and the replayed result must still match the FP64 oracle."""
import numpy as np
import pytest

from oracle import density, estimators
from paper_2212_09642_gb300 import graphs, vne

pytestmark = pytest.mark.gpu


def _stats(ctx):
    return np.array(vne.vne_ctx_graph_stats(ctx))


@pytest.mark.parametrize("fp64", [False, True])
def test_hutchinson_replay_bit_identical(vctx, fp64):
    g = graphs.barabasi_albert(6000, 3, 11)
    mat = vne.matrix_from_graph(vctx, g, fp64=fp64)
    try:
        direct, _ = vne.vne_entropy_hutchinson(vctx, mat, 40, 25, 77, opt=vne.options(graphs=0))
        s0 = _stats(vctx)
        runs = [vne.vne_entropy_hutchinson(vctx, mat, 40, 25, 77)[0] for _ in range(4)]
        s1 = _stats(vctx)
    finally:
        vne.vne_matrix_destroy(mat)
    assert all(r == direct for r in runs), (direct, runs)
    captured, replayed = s1 - s0
    assert captured == 1 and replayed >= 3, (captured, replayed)
    # the replayed estimate is the oracle's Hutchinson estimate on the same vectors
    A, _ = density.density_matrix(g)
    ref, _ = estimators.hutchinson(A, 40, 25, seed=77, reorth="full" if fp64 else "none")
    assert abs(runs[-1] - ref) <= (1e-10 if fp64 else 1e-5) * abs(ref)


def test_hutchpp_replay_bit_identical(vctx):
    g = graphs.erdos_renyi(5000, 0.002, 4)
    mat = vne.matrix_from_graph(vctx, g, fp64=False)
    try:
        direct = vne.vne_entropy_hutchpp(vctx, mat, 24, 16, 20, 5, opt=vne.options(graphs=0))
        s0 = _stats(vctx)
        runs = [vne.vne_entropy_hutchpp(vctx, mat, 24, 16, 20, 5) for _ in range(3)]
        s1 = _stats(vctx)
    finally:
        vne.vne_matrix_destroy(mat)
    for r in runs:
        assert r[0] == direct[0] and np.array_equal(r[1], direct[1])
    captured, replayed = s1 - s0
    assert captured == 2 and replayed >= 2, (captured, replayed)


def test_batch_replay_bit_identical(vctx):
    gs = [graphs.erdos_renyi(n, 8.0 / n, 30 + i) for i, n in enumerate([700, 1500, 400, 2600])]
    mats = [vne.matrix_from_graph(vctx, g) for g in gs]
    try:
        direct = vne.vne_batch_hutchinson(vctx, mats, 16, 20, 9, opt=vne.options(graphs=0))
        runs = [vne.vne_batch_hutchinson(vctx, mats, 16, 20, 9) for _ in range(3)]
    finally:
        for m in mats:
            vne.vne_matrix_destroy(m)
    for est, se in runs:
        assert np.array_equal(est, direct[0]) and np.array_equal(se, direct[1])


def test_profiled_calls_launch_directly(vctx):
    g = graphs.erdos_renyi(3000, 0.003, 8)
    mat = vne.matrix_from_graph(vctx, g)
    try:
        vne.vne_ctx_profile(vctx, True)
        s0 = _stats(vctx)
        for _ in range(3):
            vne.vne_entropy_hutchinson(vctx, mat, 16, 10, 3)
        s1 = _stats(vctx)
        launches, st = vne.vne_ctx_stats(vctx)
    finally:
        vne.vne_ctx_profile(vctx, False)
        vne.vne_matrix_destroy(mat)
    assert np.array_equal(s1, s0)
    assert st["step"][0] == 3 * 10
