"""The batched uneven workload at its full size, in the launch configuration
the benchmark times: 512 graphs with n log-uniform in [1e3, 2e5] (ER degree
8, BA m = 3, WS k = 6 beta = 0.1; sum n = 1.9e7), FP32 implicit Laplacians, 64
Rademacher probes x 40 plain Lanczos steps each, one packed launch sequence.

Sampled against the FP64 oracle (Hutchinson on the same probes, plain
recurrence): the smallest graph, the median one and the largest BA graph,
within the mixed-path tolerance 1e-5; those graphs run alone give the batched
numbers bit for bit; every estimate of the batch lies in [0, log n]."""
import math

import numpy as np
import pytest

from oracle import density, estimators
from paper_2212_09642_gb300 import graphs, vne

pytestmark = pytest.mark.gpu

SEED = 1


def test_batched_full_size_sampled_against_oracle(vctx):
    gs = graphs.batched_uneven_family(512, 1000, 200000, 1000)
    ns = np.array([g.n for g in gs])
    ba = [i for i in range(len(gs)) if i % 3 == 1]
    sample = sorted({int(np.argmin(ns)), int(np.argsort(ns)[len(ns) // 2]), max(ba, key=lambda i: ns[i])})
    opt = vne.options(reorth=0)
    mats = [vne.matrix_from_graph(vctx, g, fp64=False) for g in gs]
    try:
        est, se = vne.vne_batch_hutchinson(vctx, mats, 64, 40, SEED, opt=opt)
        alone = {i: vne.vne_entropy_hutchinson(vctx, mats[i], 64, 40, SEED, opt=opt)[0] for i in sample}
    finally:
        for m in mats:
            vne.vne_matrix_destroy(m)
    assert est.shape == (512,) and np.all(np.isfinite(est)) and np.all(se >= 0)
    assert np.all(est >= 0) and np.all(est <= np.log(ns) * (1 + 1e-6))
    for i in sample:
        assert est[i] == alone[i]
        A, _ = density.density_matrix(gs[i])
        ref, _ = estimators.hutchinson(A, 64, 40, SEED, reorth="none")
        assert abs(est[i] - ref) <= 1e-5 * ref, (i, gs[i].n, est[i], ref)
        assert ref <= math.log(gs[i].n)
