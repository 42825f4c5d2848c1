"""Pins for the oracle's probing method with the heuristic choice of d
(Section 5.1, Algorithm 2): the stopping rule against Theorem 4.4 and the
dense f(A), the end-to-end relative accuracy the algorithm targets, the
per-colour tolerances adding up to eps_hat, and the choice of d on data that
follow the error model exactly."""
import math

import numpy as np
import pytest

from oracle import bounds, coloring, density, entropy, estimators, krylov, probing
from paper_2212_09642_gb300 import graphs


def _dense(g):
    A, _ = density.density_matrix(g)
    Ad = A.toarray()
    lam = np.linalg.eigvalsh(Ad)
    F = entropy.dense_matrix_function(A)
    return A, lam, F


def test_adaptive_stop_within_theorem_4_4_bracket():
    """With the true spectral interval [lambda_2, ||A||_G] Theorem 4.4 is a
    rigorous bracket: at the step where the block stops, every column's
    estimate is below its tolerance and its actual error (against the dense
    f(A)) lies between the lower and upper bound."""
    g = graphs.watts_strogatz(300, 6, 0.2, 3)
    A, lam, F = _dense(g)
    col = coloring.greedy_distance_coloring(g, 2)
    V = estimators.probing_vectors(col)
    tol = 1e-7
    psi, steps = probing.adaptive_quadforms(A, V, 60, 4, tol_rel=tol, lam_min=lam[1])
    assert steps % 4 == 0 and steps < 60
    nA = density.gershgorin_norm(A)
    for l in range(V.shape[1]):
        c = krylov.desingularize(V[:, l])
        exact = float(c @ F @ c)
        alpha, beta, _ = krylov.lanczos(A, c, steps, norm_A=nA)
        lo, hi, est = bounds.posterior_bounds(alpha, beta, float(c @ c), lam[1], nA, grid=1000)
        err = abs(psi[l] - exact)
        assert est <= tol * abs(psi[l])
        assert lo * (1 - 1e-6) - 1e-15 <= err <= hi * (1 + 1e-6) + 1e-15, (l, lo, err, hi)


def test_adaptive_zero_tolerance_runs_all_steps():
    g = graphs.erdos_renyi(200, 0.05, 2)
    A, _ = density.density_matrix(g)
    V = estimators.probing_vectors(coloring.greedy_distance_coloring(g, 1))
    psi, steps = probing.adaptive_quadforms(A, V, 25, 5, tol_abs=np.zeros(V.shape[1]))
    assert steps == 25
    assert np.allclose(psi, estimators.quadforms(A, V, 25), rtol=1e-13, atol=0)


@pytest.mark.parametrize("eps", [1e-2, 1e-3])
@pytest.mark.parametrize("name", ["grid", "ws", "rgg"])
def test_probing_auto_reaches_relative_accuracy(name, eps):
    """The algorithm's target: |estimate - S| <= eps S (Section 5), on graphs
    whose S is known from the dense spectrum; and the sum of the quadratic
    forms is within eps_hat of the exact T_d of the chosen colouring (eq.
    algorithm-probing-krylov-error-requirement).

    The choice of d is a heuristic without a guarantee.  On the 2D grid it
    falls short at eps = 1e-3: the grid is bipartite, T_1 comes from two
    colours and is far off, and the fit to T_1..T_3 predicts a faster decay
    than the grid's T_d has (it takes d = 3, relative error 4.6e-3); the
    Krylov part is still within eps_hat of that T_3."""
    g = {"grid": graphs.grid2d(24, 25),
         "ws": graphs.watts_strogatz(500, 6, 0.1, 7),
         "rgg": graphs.random_geometric(700, graphs.rgg_radius_for_degree(700, 6.0), 9)}[name]
    A, lam, F = _dense(g)
    S = entropy.entropy_from_eigenvalues(lam)
    est, rep = probing.probing_auto(A, g, eps, 80, check=4)
    if name == "grid" and eps == 1e-3:
        assert rep["d"] == 3 and abs(est - S) > eps * S
    else:
        assert abs(est - S) <= eps * S, (name, eps, est, S, rep["d"], rep["rule"])
    d = rep["d"]
    exact_Td = estimators.probing_exact(F, coloring.greedy_distance_coloring(g, d))
    assert abs(est - exact_Td) <= rep["eps_abs"], (est, exact_Td, rep["eps_abs"])
    # T_d <= S for a graph Laplacian (the probing lower bound of Section 3.1)
    for T in rep["T"]:
        assert T <= S * (1 + eps)


def test_per_colour_tolerances_add_up_to_eps_hat():
    g = graphs.random_geometric(400, graphs.rgg_radius_for_degree(400, 6.0), 4)
    col = coloring.greedy_distance_coloring(g, 2)
    sizes = np.bincount(col)
    tols = [bounds.probing_quadform_tolerance(3e-4, int(s), g.n) for s in sizes]
    assert math.isclose(math.fsum(tols), 3e-4, rel_tol=1e-14)


def test_choose_distance_recovers_k2_model_exactly():
    """|T_{d+1} - T_d| = C q^d / d^2 with q = 0.6: the k = 3 fit has q = 1.2
    and is discarded, the k = 2 fit recovers C and q, and d is the first d at
    which the modelled error is below eps_hat."""
    C, q = 0.5, 0.6
    e = lambda d: C * q ** d / d ** 2
    T = [1.0, 1.0 + e(1), 1.0 + e(1) + e(2)]
    for eps_abs in (1e-2, 1e-4, 1e-7):
        d, rule = probing.choose_distance(list(T), eps_abs, 64, None)
        assert rule == probing.RULE_FIT
        assert d == min(dd for dd in range(1, 200) if e(dd) <= eps_abs)


def test_choose_distance_fallback_and_cap():
    # no decaying fit (q >= 1 for k = 2, 3): consecutive differences decide
    T = [1.0, 1.1, 1.2]
    extra = {4: 1.25, 5: 1.26, 6: 1.261}
    d, rule = probing.choose_distance(list(T), 0.02, 64, lambda dd: extra[dd])
    assert (d, rule) == (4, probing.RULE_DIFFERENCES)
    d, rule = probing.choose_distance(list(T), 1e-9, 6, lambda dd: extra[dd])
    assert (d, rule) == (6, probing.RULE_CAPPED)
    # a decaying fit that would need more than d_max
    d, rule = probing.choose_distance([1.0, 1.1, 1.12], 1e-12, 5, None)
    assert (d, rule) == (5, probing.RULE_CAPPED)


def test_degenerate_differences():
    # T_2 = T_1: no error left at d = 1; T_3 = T_2: q = 0, d = 2 unless T_1 already suffices
    assert bounds.probing_heuristic_d(1.0, 1.0, 1.3, 1e-6) == 1
    assert bounds.probing_heuristic_d(1.0, 1.2, 1.2, 1e-6) == 2
    assert bounds.probing_heuristic_d(1.0, 1.0 + 1e-7, 1.0 + 1e-7, 1e-6) == 1


def test_complete_graph_d1_is_exact():
    """K_n: every pair is adjacent, the distance-1 colouring has n colours, so
    T_1 = tr f(A) = S and T_2 = T_3 = T_1 (e1 = 0): d = 1."""
    g = graphs.complete(40)
    A, lam, _ = _dense(g)
    S = entropy.entropy_from_eigenvalues(lam)
    est, rep = probing.probing_auto(A, g, 1e-3, 10, check=2)
    assert rep["d"] == 1 and rep["colors"][1] == 40
    assert abs(est - S) <= 1e-10 * S
