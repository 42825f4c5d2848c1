"""The tcgen05 kernels of the Hutch++ sketch (Section 3.2) against FP64
products of the same FP32 data, elementwise: the Gram C = X^T Y and the
block product Out = In2 + coef In M.  The TF32 three-product split and FP32
accumulation keep each entry within a small multiple of the FP32 unit
roundoff of the sum of the absolute products."""
import numpy as np
import pytest
import torch

from paper_2212_09642_gb300 import vne

pytestmark = pytest.mark.gpu


def panel_major(M, ks):
    """[n, k] -> device float32 [k / ks][n][ks]."""
    n, k = M.shape
    P = np.ascontiguousarray(M.reshape(n, k // ks, ks).transpose(1, 0, 2)).astype(np.float32)
    return torch.from_numpy(P).cuda()


@pytest.mark.parametrize("n,kx,ky,ks,same", [
    (1_000_000, 112, 112, 16, True), # the headline sketch's Y^T Y (n = 10^6, N_r = 100 in 7 panels)
    (100_003, 112, 112, 16, True),   # the same shape, ragged tail
    (5_000, 128, 128, 32, True),     # full 128 x 128 tile
    (77_777, 112, 112, 16, False),   # Q^T G
    (40_000, 16, 48, 8, False),      # narrow, N not a multiple of the output tile
    (33, 32, 16, 16, False),         # fewer rows than one slab per CTA
    (1, 8, 8, 8, True),              # a single row
])
def test_block_gram_tcgen05(vctx, n, kx, ky, ks, same):
    rs = np.random.default_rng(n + kx + ky)
    X = rs.standard_normal((n, kx)).astype(np.float32)
    Y = X if same else rs.standard_normal((n, ky)).astype(np.float32)
    dX = panel_major(X, ks)
    dY = dX if same else panel_major(Y, ks)
    C = vne.vne_block_gram(vctx, dX, kx, dY, ky, ks, n)
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    ref = X64.T @ Y64
    scale = np.abs(X64).T @ np.abs(Y64)
    err = np.abs(C - ref)
    assert np.all(err <= 2e-5 * scale + 1e-30), float(np.max(err / (scale + 1e-300)))


def test_block_gram_rejects_bad_sizes(vctx):
    d = torch.zeros((2, 10, 16), dtype=torch.float32, device="cuda")
    for kx, ky, ks in [(0, 16, 16), (144, 16, 16), (16, 12, 16), (16, 16, 4)]:
        with pytest.raises(vne.VneError):
            vne.vne_block_gram(vctx, d, kx, d, ky, ks, 10)


@pytest.mark.parametrize("n,kin,kout,ks,addend", [
    (1_000_000, 112, 112, 16, False),  # the headline sketch's Q = Y R^{-1}
    (100_003, 112, 112, 16, True),     # G' = G - Q C, ragged tail
    (77_777, 128, 128, 32, True),      # full 128-column blocks
    (50_000, 16, 48, 8, False),        # one K chunk, N padded to 48
    (300, 40, 8, 8, True),             # fewer rows than one tile
    (1, 8, 8, 8, False),               # a single row
])
def test_block_apply_tcgen05(vctx, n, kin, kout, ks, addend):
    rs = np.random.default_rng(n + 3 * kin + kout)
    A = rs.standard_normal((n, kin)).astype(np.float32)
    M = rs.standard_normal((kin, kout))
    coef = -1.0 if addend else 1.0
    A2 = rs.standard_normal((n, kout)).astype(np.float32) if addend else None
    dA = panel_major(A, ks)
    dA2 = panel_major(A2, ks) if addend else None
    dO = torch.empty((kout // ks, n, ks), dtype=torch.float32, device="cuda")
    vne.vne_block_apply(vctx, dA, kin, M, kout, dA2, dO, ks, n, coef)
    got = dO.cpu().numpy().transpose(1, 0, 2).reshape(n, kout).astype(np.float64)
    Mf = (coef * M).astype(np.float32).astype(np.float64)  # B is coef M rounded to FP32
    ref = A.astype(np.float64) @ Mf
    scale = np.abs(A.astype(np.float64)) @ np.abs(Mf)
    if addend:
        ref += A2.astype(np.float64)
        scale += np.abs(A2.astype(np.float64))
    err = np.abs(got - ref)
    assert np.all(err <= 2e-6 * scale + 1e-30), float(np.max(err / (scale + 1e-300)))


def test_block_apply_rejects_bad_sizes(vctx):
    d = torch.zeros((2, 10, 16), dtype=torch.float32, device="cuda")
    M = np.zeros((16, 16))
    for kin, kout, ks in [(0, 16, 16), (144, 16, 16), (16, 12, 16), (16, 16, 4)]:
        with pytest.raises(vne.VneError):
            vne.vne_block_apply(vctx, d, kin, np.zeros((max(kin, 1), max(kout, 1))), kout, None, d, ks, 10)
