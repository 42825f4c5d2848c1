"""Hutch++ (Section 3.2, eq. Hutch++_formula) part by part: GPU (C ABI) vs the
FP64 oracle on the same probes and step counts.

* the sketch Y = f(A) Omega column by column (eq.
  rational-krylov-approximation-matvec), relative to ||y_j||;
* the pivot order of orth(Y): the column-pivoted QR factor (Businger-Golub),
  which the GPU's pivoted Cholesky-QR computes;
* psi(q_i) per column of Q, in pivot order;
* psi(g'_j) per projected Hutchinson vector (these depend only on span(Q));
* the estimate.
Tolerances: 1e-10 (FP64 path, full reorthogonalisation on both sides) and
1e-5 (mixed path: FP32 vectors, no reorthogonalisation on both sides) for
every quadratic form and the estimate; the sketch columns, vectors recovered
from m + 1 Lanczos slots, to 1e-10 (FP64) and 5e-5 (FP32) of their norm.
Also: the staged entry points split over column ranges reproduce the
one-call estimate column for column."""
import numpy as np
import pytest

from oracle import density, estimators
from paper_2212_09642_gb300 import graphs, vne

pytestmark = pytest.mark.gpu

CASES = [("BA3000", lambda: graphs.barabasi_albert(3000, 3, 4), 16, 24, 30),
         ("ER2000", lambda: graphs.erdos_renyi(2000, 0.005, 1), 12, 20, 40)]


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.mark.parametrize("name,make,Nr,NH,m", CASES)
@pytest.mark.parametrize("fp64,tol", [(True, 1e-10), (False, 1e-5)])
def test_hutchpp_parts_match_oracle(vctx, name, make, Nr, NH, m, fp64, tol):
    g = make()
    A, _ = density.density_matrix(g)
    ref, rp = estimators.hutchpp(A, Nr, NH, m, seed=5, reorth="full" if fp64 else "none", return_parts=True)
    o = vne.options(reorth=1 if fp64 else 0)
    mat = vne.matrix_from_graph(vctx, g, fp64=fp64)
    try:
        est, parts = vne.vne_entropy_hutchpp(vctx, mat, Nr, NH, m, seed=5, opt=o)
        Y = vne.vne_hutchpp_sketch(vctx, mat, 0, Nr, m, 5, fp64, opt=o)
        psi, piv, r = vne.vne_hutchpp_project(vctx, mat, Y, Nr, NH, m, 5, opt=o)
    finally:
        vne.vne_matrix_destroy(mat)
    Yr = rp["Y"]
    tol_vec = 1e-10 if fp64 else 5e-5
    for j in range(Nr):
        assert np.linalg.norm(Y[:, j] - Yr[:, j]) <= tol_vec * np.linalg.norm(Yr[:, j]), j
    assert r == rp["Q"].shape[1] == int(parts[2])
    assert np.array_equal(piv[:r], rp["pivots"])
    assert np.all(piv[r:] == -1)
    assert _rel(psi[:r], rp["psi_q"]) <= tol
    assert np.all(psi[r:Nr] == 0.0)
    assert _rel(psi[Nr:], rp["psi_g"]) <= tol
    assert abs(est - ref) <= tol * abs(ref)
    assert abs(parts[0] - rp["low_rank"]) <= tol * abs(rp["low_rank"])
    # the staged result is the one-call result
    assert abs(psi[:r].sum() + psi[Nr:].mean() - est) <= 1e-14 * abs(est)


@pytest.mark.parametrize("fp64", [True, False])
def test_hutchpp_ranges_reproduce_one_call(vctx, fp64):
    """Sketch columns computed in two ranges and quadratic forms in three are
    bit-identical to the whole ranges (each column is its own recurrence)."""
    g = graphs.barabasi_albert(3000, 3, 4)
    Nr, NH, m = 16, 24, 30
    o = vne.options(reorth=1 if fp64 else 0)
    mat = vne.matrix_from_graph(vctx, g, fp64=fp64)
    try:
        Y = vne.vne_hutchpp_sketch(vctx, mat, 0, Nr, m, 5, fp64, opt=o)
        Ya = vne.vne_hutchpp_sketch(vctx, mat, 0, 5, m, 5, fp64, opt=o)
        Yb = vne.vne_hutchpp_sketch(vctx, mat, 5, Nr - 5, m, 5, fp64, opt=o)
        psi, piv, r = vne.vne_hutchpp_project(vctx, mat, Y, Nr, NH, m, 5, opt=o)
        parts = [vne.vne_hutchpp_project(vctx, mat, Y, Nr, NH, m, 5, col_begin=c0, ncols=nc, opt=o)[0]
                 for c0, nc in ((0, 7), (7, 20), (27, Nr + NH - 27))]
    finally:
        vne.vne_matrix_destroy(mat)
    assert np.array_equal(np.hstack([Ya, Yb]), Y)
    assert np.array_equal(np.concatenate(parts), psi)


def test_hutchpp_device_sketch(vctx):
    """Stage 1 into a CUDA tensor and stage 2 from it give the host results."""
    import torch
    g = graphs.erdos_renyi(2000, 0.005, 1)
    Nr, NH, m = 12, 20, 40
    mat = vne.matrix_from_graph(vctx, g, fp64=False)
    try:
        Yh = vne.vne_hutchpp_sketch(vctx, mat, 0, Nr, m, 5, False)
        Yd = torch.zeros((g.n, Nr), dtype=torch.float32, device="cuda")
        vne.vne_hutchpp_sketch(vctx, mat, 0, Nr, m, 5, False, out=Yd)
        ph = vne.vne_hutchpp_project(vctx, mat, Yh, Nr, NH, m, 5)
        pd = vne.vne_hutchpp_project(vctx, mat, Yd, Nr, NH, m, 5)
    finally:
        vne.vne_matrix_destroy(mat)
    assert np.array_equal(Yd.cpu().numpy(), Yh)
    assert np.array_equal(ph[0], pd[0]) and np.array_equal(ph[1], pd[1]) and ph[2] == pd[2]
