"""Probing with the heuristic choice of d (vne_entropy_probing_auto, Section
5.1 / Algorithm 2) against the oracle: the colour counts at d = 1, 2, 3, the
sums T_1..T_3 at the Lanczos step counts the device stopped at, the stopping
decisions themselves (FP64: the oracle's Theorem 4.4 estimates are below the
tolerances at the device's step and not all below at the check before), the
choice of d from the device's T values, and the final accuracy."""
import numpy as np
import pytest

from oracle import coloring, density, entropy, estimators, krylov, probing
from paper_2212_09642_gb300 import graphs, vne

pytestmark = pytest.mark.gpu


def _block_state(A, V, j, lam_min=0.0, grid=1000):
    nA = density.gershgorin_norm(A)
    out = []
    for l in range(V.shape[1]):
        c = krylov.desingularize(V[:, l])
        alpha, beta, _ = krylov.lanczos(A, c, j, norm_A=nA)
        out.append(probing._column_state(alpha, beta, float(c @ c), j, lam_min, nA, grid))
    return np.array([o[0] for o in out]), np.array([o[1] for o in out])


CASES = [
    ("RGG3000", lambda: graphs.random_geometric(3000, graphs.rgg_radius_for_degree(3000, 6.0), 21)),
    ("WS2000", lambda: graphs.watts_strogatz(2000, 6, 0.1, 22)),
]


@pytest.mark.parametrize("fp64,eps,name,make", [(True, 1e-3) + CASES[0], (False, 1e-3) + CASES[0],
                                                (True, 1e-3) + CASES[1], (False, 1e-3) + CASES[1],
                                                (True, 1e-5) + CASES[0]])
def test_probing_auto_matches_oracle(vctx, name, make, fp64, eps):
    g = make()
    A, _ = density.density_matrix(g)
    S = entropy.dense_entropy(A)
    m, check = 80, 2
    mat = vne.matrix_from_graph(vctx, g, fp64=fp64, reorder="rcm" if name.startswith("RGG") else True)
    try:
        est, rep = vne.vne_entropy_probing_auto(vctx, mat, eps, m, 16, opt=vne.options(check_every=check))
    finally:
        vne.vne_matrix_destroy(mat)
    tol = 1e-10 if fp64 else 1e-5
    for d in (1, 2, 3):
        col = coloring.greedy_distance_coloring(g, d)
        V = estimators.probing_vectors(col)
        assert rep["colors_d"][d - 1] == V.shape[1]
        steps = rep["steps_d"][d - 1]
        assert steps == m or steps % check == 0
        psi, est_now = _block_state(A, V, steps)
        assert abs(rep["T"][d - 1] - psi.sum()) <= tol * abs(psi.sum()), (d, rep["T"][d - 1], psi.sum())
        if fp64 and steps < m:
            # the device stopped where the oracle's estimates meet the tolerances ...
            t = 0.5 * eps * np.abs(psi) if d == 1 else rep["eps_abs"] * V.sum(axis=0) / g.n
            assert np.all(est_now <= t * (1 + 1e-4) + 1e-15), d
            if steps > check:
                # ... and not one check earlier
                psi_b, est_b = _block_state(A, V, steps - check)
                t_b = 0.5 * eps * np.abs(psi_b) if d == 1 else t
                assert np.any(est_b > t_b * (1 - 1e-4)), d
    assert rep["eps_abs"] == pytest.approx(0.5 * eps * rep["T"][0], rel=1e-15)
    # the choice of d from the device's own T values
    d_ref, rule_ref = probing.choose_distance(list(rep["T"]), rep["eps_abs"], 16, lambda dd: None)
    assert (rep["d"], rep["rule"]) == (d_ref, rule_ref)
    if rep["d"] <= 3:
        assert est == rep["T"][rep["d"] - 1]
    else:
        # T_d at the chosen distance, at the device's step count, and within
        # eps_abs of the exact T_d of that colouring
        V = estimators.probing_vectors(coloring.greedy_distance_coloring(g, rep["d"]))
        assert rep["colors"] == V.shape[1]
        psi, _ = _block_state(A, V, rep["steps"])
        assert abs(est - psi.sum()) <= tol * abs(psi.sum())
        F = entropy.dense_matrix_function(A)
        assert abs(est - float(np.sum(V * (F @ V)))) <= rep["eps_abs"]
    if eps >= 1e-3:
        # the target (a heuristic; at eps = 1e-3 these graphs follow its model)
        assert abs(est - S) <= eps * S, (name, est, S, rep)


def test_probing_auto_rejects_bad_arguments(vctx):
    g = graphs.erdos_renyi(300, 0.02, 1)
    mat = vne.matrix_from_graph(vctx, g)
    try:
        for args in [(0.0, 30, 8), (1.5, 30, 8), (1e-3, 0, 8), (1e-3, 30, 0)]:
            with pytest.raises(vne.VneError):
                vne.vne_entropy_probing_auto(vctx, mat, *args)
    finally:
        vne.vne_matrix_destroy(mat)
