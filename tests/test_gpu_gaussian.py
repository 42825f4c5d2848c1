"""Gaussian probes (the paper's distribution, Section 3.2) on the device: the
entries against the oracle's Box-Muller on the same counters, and the
Hutchinson / Hutch++ estimates with Gaussian probes against the FP64 oracle
on identical vectors."""
import numpy as np
import pytest
import torch

from oracle import density, entropy, estimators, rng
from paper_2212_09642_gb300 import graphs, vne

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,col_begin,k", [(1, 0, 1), (1000, 0, 7), (4097, 13, 33)])
def test_gaussian_probe_entries(vctx, n, col_begin, k):
    out = torch.empty((n, k), dtype=torch.float64, device="cuda")
    vne.vne_gaussian_probes(vctx, 21, n, col_begin, k, out)
    ref = rng.gaussian(21, n, col_begin, k)
    got = out.cpu().numpy()
    # log and cos are each within a few ulp on both sides
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-14)


def test_gaussian_probe_moments(vctx):
    n, k = 200_000, 4
    out = torch.empty((n, k), dtype=torch.float64, device="cuda")
    vne.vne_gaussian_probes(vctx, 5, n, 0, k, out)
    x = out.cpu().numpy().ravel()
    assert abs(x.mean()) < 5 / np.sqrt(x.size)
    assert abs(x.var() - 1.0) < 5 * np.sqrt(2.0 / x.size)


def test_hutchinson_gaussian_fp64_parity(vctx):
    g = graphs.erdos_renyi(1500, 0.006, 2)
    A, _ = density.density_matrix(g)
    mat = vne.matrix_from_graph(vctx, g, fp64=True)
    try:
        est, se, psi = vne.vne_entropy_hutchinson(vctx, mat, 40, 40, seed=9, want_psi=True,
                                                  opt=vne.options(gaussian_probes=1))
        est_r = vne.vne_entropy_hutchinson(vctx, mat, 40, 40, seed=9)[0]
    finally:
        vne.vne_matrix_destroy(mat)
    ref_est, ref_psi = estimators.hutchinson(A, 40, 40, seed=9, reorth="full", dist="gaussian")
    assert np.max(np.abs(psi - ref_psi) / np.abs(ref_psi)) <= 1e-10
    assert abs(est - ref_est) <= 1e-10 * abs(ref_est)
    assert est != est_r  # the option does change the probes
    S = entropy.dense_entropy(A)
    assert abs(est - S) <= 5 * se + 1e-12


@pytest.mark.parametrize("fp64,tol", [(True, 1e-10), (False, 1e-5)])
def test_hutchpp_gaussian_parity(vctx, fp64, tol):
    g = graphs.barabasi_albert(2500, 3, 6)
    A, _ = density.density_matrix(g)
    mat = vne.matrix_from_graph(vctx, g, fp64=fp64)
    try:
        est, parts = vne.vne_entropy_hutchpp(vctx, mat, 16, 24, 30, seed=4,
                                             opt=vne.options(reorth=1 if fp64 else 0, gaussian_probes=1))
    finally:
        vne.vne_matrix_destroy(mat)
    ref, rp = estimators.hutchpp(A, 16, 24, 30, seed=4, reorth="full" if fp64 else "none",
                                 return_parts=True, dist="gaussian")
    assert int(parts[2]) == rp["Q"].shape[1]
    assert abs(est - ref) <= tol * abs(ref), (est, ref)
    assert abs(parts[0] - rp["low_rank"]) <= tol * abs(ref)
