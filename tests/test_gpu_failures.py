"""Failure detection in the forms that fault no GPU.

* Host-side allocation failure: the library's allocation wrappers make the
  k-th allocation fail as if memory were exhausted.  For every k over a
  sequence that builds matrices and runs several estimators, the failing
  call returns VNE_ENOMEM, the context stays usable (the same sequence then
  gives the undisturbed results), and once everything is destroyed the
  library holds no more device or pinned buffers than before.
"""
import numpy as np
import pytest

from oracle import rng
from paper_2212_09642_gb300 import graphs, vne

pytestmark = pytest.mark.gpu


def _sequence(ctx, gs):
    """Matrices with and without relabelling, Hutch++, a rational quadrature
    and a batched estimate; returns the numbers and the matrices made."""
    mats, out = [], []
    try:
        for i, g in enumerate(gs):
            mats.append(vne.matrix_from_graph(ctx, g, fp64=False, reorder=bool(i % 2)))
        out.append(vne.vne_entropy_hutchpp(ctx, mats[0], 8, 8, 12, 3)[0])
        X = rng.rademacher(2, gs[1].n, 0, 3)
        out.extend(vne.vne_quadform_rational(ctx, mats[1], X, None, num_shifts=4)[0].tolist())
        out.extend(vne.vne_batch_hutchinson(ctx, mats, 16, 10, 5)[0].tolist())
    finally:
        for m in mats:
            vne.vne_matrix_destroy(m)
    return out


def test_allocation_failure_is_enomem_and_leaks_nothing(vctx):
    gs = [graphs.barabasi_albert(600, 3, 1), graphs.erdos_renyi(500, 0.02, 2)]
    vne.vne_debug_fail_allocation(0)
    base = vne.vne_debug_live_allocations()
    ctx = vne.vne_ctx_create(0)
    try:
        want = _sequence(ctx, gs)
    finally:
        vne.vne_ctx_destroy(ctx)
    assert vne.vne_debug_live_allocations() == base
    failures = 0
    for k in range(1, 400):
        ctx = vne.vne_ctx_create(0)
        try:
            vne.vne_debug_fail_allocation(k)
            try:
                _sequence(ctx, gs)
                hit = False
            except vne.VneError as e:
                assert e.status == vne.VNE_ENOMEM, (k, e)
                hit = True
            vne.vne_debug_fail_allocation(0)
            if hit:
                failures += 1
                got = _sequence(ctx, gs)  # the context is still usable
                assert np.allclose(got, want, rtol=1e-12, atol=0), k
        finally:
            vne.vne_debug_fail_allocation(0)
            vne.vne_ctx_destroy(ctx)
        assert vne.vne_debug_live_allocations() == base, k
        if not hit:
            break
    assert failures >= 10


def test_tensor_core_wait_timeout_is_reported():
    """The tcgen05 sketch kernels' main-loop waits are made to give up at
    once (a limit of zero polls).  Every CTA then takes the time-out path --
    error flag, a full-limit wait for the MMAs already issued, TMEM freed --
    and the calls report VNE_ETIMEOUT.  With the limit restored the same
    calls give the undisturbed results, bit for bit: the context and the
    GPU stay usable."""
    import torch
    n, ks, k = 60_000, 16, 32  # >= 3 slabs and >= 3 row tiles on every CTA
    gen = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randn(k * n, device="cuda", generator=gen)
    Y = torch.randn(k * n, device="cuda", generator=gen)
    Mh = np.random.default_rng(3).standard_normal((k, k))
    out = torch.zeros(k * n, device="cuda")
    g = graphs.barabasi_albert(20_000, 3, 4)
    ctx = vne.vne_ctx_create(0)
    mat = vne.matrix_from_graph(ctx, g, fp64=False)

    def run():
        C1 = vne.vne_block_gram(ctx, X, k, X, k, ks, n)
        C2 = vne.vne_block_gram(ctx, X, k, Y, k, ks, n)
        vne.vne_block_apply(ctx, X, k, Mh, k, Y, out, ks, n, -1.0)
        torch.cuda.synchronize()
        est = vne.vne_entropy_hutchpp(ctx, mat, 16, 16, 20, 3)[0]
        return C1, C2, out.cpu().numpy().copy(), est

    try:
        want = run()
        vne.vne_debug_tensor_wait_limit(0)
        try:
            for call in (lambda: vne.vne_block_gram(ctx, X, k, X, k, ks, n),
                         lambda: vne.vne_block_gram(ctx, X, k, Y, k, ks, n),
                         lambda: vne.vne_block_apply(ctx, X, k, Mh, k, Y, out, ks, n, -1.0),
                         lambda: vne.vne_entropy_hutchpp(ctx, mat, 16, 16, 20, 3)):
                with pytest.raises(vne.VneError) as e:
                    call()
                assert e.value.status == vne.VNE_ETIMEOUT
        finally:
            vne.vne_debug_tensor_wait_limit(-1)
        got = run()
    finally:
        vne.vne_matrix_destroy(mat)
        vne.vne_ctx_destroy(ctx)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    assert np.array_equal(got[2], want[2]) and got[3] == want[3]
