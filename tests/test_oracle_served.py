"""Pins of the oracle's served estimator (adaptive Hutch++ proxy with the
Krylov stopping rule).  Without the stopping rule it is Hutch++ with a
4-column sketch and the served number of probes; with it, every block's
quadratures are within the requested accuracy of the exact quadratic forms of
the dense f(A), and the blocks stop before m on graphs where Lanczos
converges fast; the statistical stopping rule holds at the end."""
import numpy as np
import pytest

from oracle import density, entropy, estimators, krylov, rng
from paper_2212_09642_gb300 import graphs


@pytest.fixture(scope="module")
def ba():
    g = graphs.barabasi_albert(400, 3, 8)
    A, _ = density.density_matrix(g)
    return A


def test_fixed_steps_is_hutchpp_with_served_probes(ba):
    est, se, nv, steps, _ = estimators.served_hutchpp(ba, 2e-2, 16, 20, 5, max_vectors=256)
    assert nv % 16 == 0 and nv >= 32 and all(s == 20 for s in steps)
    ref = estimators.hutchpp(ba, 4, nv, 20, 5, reorth="none")
    assert abs(est - ref) <= 1e-13 * abs(ref)
    assert 2.576 * se <= 0.5 * 2e-2 * abs(est) or nv >= 256


def test_quad_tol_blocks_within_accuracy_of_exact_forms(ba):
    tol, check, m = 1e-4, 3, 30
    est, se, nv, steps, _ = estimators.served_hutchpp(ba, 2e-2, 16, m, 5, max_vectors=64, quad_tol=tol,
                                                   check_every=check)
    assert all(s % check == 0 and check <= s < m for s in steps), steps  # converged early, at check steps
    # the same estimator with exact quadratic forms (dense f(A)) on the same probes
    F = entropy.dense_matrix_function(ba)
    n = ba.shape[0]
    Omega = rng.probes(5, n, 0, 4)
    Y = np.column_stack([krylov.lanczos_fmatvec(ba, Omega[:, j], m, reorth="none") for j in range(4)])
    Q = estimators.orthonormal_range(Y)
    low = float(np.trace(Q.T @ F @ Q))
    G = rng.probes(5, n, 4, nv)
    Gp = G - Q @ (Q.T @ G)
    exact = []
    for j in range(nv):
        c = krylov.desingularize(Gp[:, j])
        exact.append(float(c @ F @ c))
    ref = low + float(np.mean(exact))
    # per-column relative errors around tol (the stopping estimate is the
    # geometric mean of two bounds, not a bound itself)
    assert abs(est - ref) <= 10 * tol * abs(ref)
    # a tighter tolerance runs more steps and lands closer
    est2, _, nv2, steps2, _ = estimators.served_hutchpp(ba, 2e-2, 16, m, 5, max_vectors=64, quad_tol=1e-8,
                                                     check_every=check)
    assert nv2 == nv and min(steps2) >= max(steps)
    assert abs(est2 - ref) <= 1e-6 * abs(ref)


def test_probe_cap_and_statistical_rule(ba):
    est, se, nv, steps, _ = estimators.served_hutchpp(ba, 1e-6, 16, 12, 3, max_vectors=48)
    assert nv == 48 and len(steps) == 3  # an unreachable accuracy stops at the cap
    est, se, nv, steps, _ = estimators.served_hutchpp(ba, 0.5, 16, 12, 3, max_vectors=4096)
    assert nv == 32 and len(steps) == 2  # at least two blocks
    assert 2.576 * se <= 0.25 * abs(est)
    S = entropy.dense_entropy(ba)
    assert abs(est - S) <= 0.05 * S


def test_sketch_steps_and_sketch_forms(ba):
    """Any sketch keeps Hutch++ unbiased (Q independent of G): a short sketch
    (6 steps) changes the estimate by far less than its statistical error;
    with quad_tol the basis vectors' quadratic forms stop early too."""
    est, se, nv, steps, qs = estimators.served_hutchpp(ba, 2e-2, 16, 30, 5, max_vectors=64)
    est6, se6, nv6, _, _ = estimators.served_hutchpp(ba, 2e-2, 16, 30, 5, max_vectors=64, sketch_steps=6)
    assert nv6 == nv and abs(est6 - est) <= se
    _, _, _, steps_t, qs_t = estimators.served_hutchpp(ba, 2e-2, 16, 30, 5, max_vectors=64, sketch_steps=6,
                                                       quad_tol=1e-4, check_every=3)
    assert qs == 30 and qs_t % 3 == 0 and 3 <= qs_t < 30
