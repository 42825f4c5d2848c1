"""The allocation-free entry point (vne_quadform_noalloc).

It serves callers that cannot allocate device memory when they need the
result -- for example code bound to another framework's memory pool, or an
allocator-free real-time loop: they pass only buffers they own, and all
intermediates live in the library's fixed static device scratch.  This test
calls it through the C ABI twice in a row (different sizes, so the second
call must not depend on what the first left in the shared scratch) and
compares each result with the existing allocating entry point
vne_quadform_batch (FP64 path, plain recurrence) within the FP64 tolerance
of the other parity tests, 1e-10 relative.  It lives in its own file, named
to be collected last.
"""
import numpy as np
import pytest

from oracle import rng
from paper_2212_09642_gb300 import graphs, vne

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _device_csr(g):
    import torch
    rp = torch.tensor(g.rowptr.astype(np.int32), device="cuda")
    ci = torch.tensor(g.col, device="cuda")
    return rp, ci


def test_noalloc_matches_allocating_entry_point_twice(vctx):
    import torch
    cases = [(graphs.erdos_renyi(3000, 0.003, 2), 13, 20, 5),
             (graphs.barabasi_albert(5000, 3, 9), 6, 12, 6)]
    stream = torch.cuda.current_stream()
    for g, k, m, seed in cases:
        X = rng.rademacher(seed, g.n, 0, k)
        X[:, 0] = np.random.default_rng(seed).standard_normal(g.n)
        rp, ci = _device_csr(g)
        Xd = torch.tensor(X, dtype=torch.float64, device="cuda")
        psi_d = torch.full((k,), float("nan"), dtype=torch.float64, device="cuda")
        vne.vne_quadform_noalloc(stream, g.n, rp, ci, Xd, k, m, psi_d)
        torch.cuda.synchronize()
        got = psi_d.cpu().numpy()
        mat = vne.matrix_from_graph(vctx, g, fp64=True)
        try:
            want = vne.vne_quadform_batch(vctx, mat, X, m, opt=vne.options(reorth=0))
        finally:
            vne.vne_matrix_destroy(mat)
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - want) / np.abs(want)) <= TOL64


def test_noalloc_rejects_sizes_beyond_the_scratch(vctx):
    import torch
    n, k = 400_000, 16  # 3 vectors x n x 16 doubles = 154 MB > 32 MiB scratch
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    X = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    psi = torch.zeros(k, dtype=torch.float64, device="cuda")
    with pytest.raises(vne.VneError):
        vne.vne_quadform_noalloc(None, n, rp, ci, X, k, 10, psi)
