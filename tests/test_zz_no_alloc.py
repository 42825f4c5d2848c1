"""The allocation-free entry point (vne_quadform_noalloc).

It serves callers that cannot allocate device memory when they need the
result -- for example code bound to another framework's memory pool, or an
allocator-free real-time loop: they pass only buffers they own, and all
intermediates live in the library's fixed static device scratch.  These
tests call it through the C ABI several times in a row (different sizes and
step counts, so no call may depend on what an earlier one left in the shared
scratch) and compare each result with the existing allocating entry point
vne_quadform_batch (FP64 path, plain recurrence) and with the FP64 oracle,
within the FP64 tolerance of the other parity tests, 1e-10 relative.  They
live in their own file, named to be collected last.
"""
import math

import numpy as np
import pytest

from oracle import density, estimators, krylov, rng
from paper_2212_09642_gb300 import graphs, vne

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _device_csr(g):
    import torch
    rp = torch.tensor(g.rowptr.astype(np.int32), device="cuda")
    ci = torch.tensor(g.col, device="cuda")
    return rp, ci


def _noalloc(g, X, m, rp=None, ci=None):
    import torch
    if rp is None:
        rp, ci = _device_csr(g)
    k = X.shape[1]
    Xd = torch.tensor(np.ascontiguousarray(X), dtype=torch.float64, device="cuda")
    psi_d = torch.full((k,), float("nan"), dtype=torch.float64, device="cuda")
    vne.vne_quadform_noalloc(torch.cuda.current_stream(), g.n, rp, ci, Xd, k, m, psi_d)
    torch.cuda.synchronize()
    return psi_d.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_and_oracle(vctx):
    # the larger step count first, then a shorter and smaller call, then a
    # tiny graph whose Lanczos recurrence breaks down long before m steps
    cases = [(graphs.barabasi_albert(5000, 3, 9), 6, 28, 6),
             (graphs.erdos_renyi(3000, 0.003, 2), 13, 20, 5),
             (graphs.path(10), 5, 30, 7)]
    for g, k, m, seed in cases:
        X = rng.rademacher(seed, g.n, 0, k)
        X[:, 0] = np.random.default_rng(seed).standard_normal(g.n)
        got = _noalloc(g, X, m)
        mat = vne.matrix_from_graph(vctx, g, fp64=True)
        try:
            want = vne.vne_quadform_batch(vctx, mat, X, m, opt=vne.options(reorth=0))
        finally:
            vne.vne_matrix_destroy(mat)
        A, _ = density.density_matrix(g)
        ref = estimators.quadforms(A, X, m, reorth="none")
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - want) / np.abs(want)) <= TOL64
        assert np.max(np.abs(got - ref) / np.abs(ref)) <= TOL64


def test_noalloc_breakdown_is_exact(vctx):
    # K_n: every desingularised vector lies in the eigenspace of 1/(n-1), the
    # recurrence stops after one step, psi = ||c||^2 f(1/(n-1)) exactly
    g = graphs.complete(10)
    X = rng.rademacher(3, 10, 0, 4)
    got = _noalloc(g, X, 30)
    lam = 1.0 / 9
    c = krylov.desingularize(X)
    want = np.sum(c * c, axis=0) * (-lam * math.log(lam))
    assert np.max(np.abs(got - want) / want) <= TOL64


def test_noalloc_invalid_csr_gives_nan(vctx):
    # the kernels' own checks: a column outside [0, n) and a decreasing pair of
    # row offsets are never dereferenced; the call marks every psi NaN
    import torch
    g = graphs.path(6)
    X = rng.rademacher(1, 6, 0, 2)
    col = g.col.copy()
    col[3] = 6
    rp = torch.tensor(g.rowptr.astype(np.int32), device="cuda")
    ci = torch.tensor(col, device="cuda")
    assert np.all(np.isnan(_noalloc(g, X, 5, rp, ci)))
    rows = g.rowptr.astype(np.int32).copy()
    rows[2], rows[3] = rows[3], rows[2]
    rp = torch.tensor(rows, device="cuda")
    ci = torch.tensor(g.col, device="cuda")
    assert np.all(np.isnan(_noalloc(g, X, 5, rp, ci)))
    # a valid call afterwards is unaffected by the flag of the last one
    rp, ci = _device_csr(g)
    assert np.all(np.isfinite(_noalloc(g, X, 5, rp, ci)))


def test_noalloc_rejects_sizes_beyond_the_scratch(vctx):
    import torch
    n, k = 400_000, 16  # 3 vectors x n x 16 doubles = 154 MB > 32 MiB scratch
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    X = torch.zeros((n, k), dtype=torch.float64, device="cuda")
    psi = torch.zeros(k, dtype=torch.float64, device="cuda")
    with pytest.raises(vne.VneError):
        vne.vne_quadform_noalloc(None, n, rp, ci, X, k, 10, psi)


def test_noalloc_binding_rejects_wrong_layouts(vctx):
    import torch
    g = graphs.path(8)
    rp, ci = _device_csr(g)
    psi = torch.zeros(2, dtype=torch.float64, device="cuda")
    X32 = torch.zeros((8, 2), dtype=torch.float32, device="cuda")
    Xt = torch.zeros((2, 8), dtype=torch.float64, device="cuda").t()
    for X in (X32, Xt):
        with pytest.raises(vne.VneError):
            vne.vne_quadform_noalloc(None, 8, rp, ci, X, 2, 5, psi)
    with pytest.raises(vne.VneError):
        vne.vne_quadform_noalloc(None, 8, rp.to(torch.int64), ci, torch.zeros((8, 2), dtype=torch.float64,
                                                                               device="cuda"), 2, 5, psi)
