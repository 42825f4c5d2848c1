"""The probing method with an a-priori choice of d (Section 5.1, Algorithm 2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Steps, in the paper's order:

1. Choose the distance d.  The heuristic of Section 5.1 fits the model
   |tr f(A) - T_d| ~ C q^d / d^k to the consecutive differences
   |T_{d+1} - T_d| at d = 1, 2 (so T_1, T_2, T_3 are computed first) for k = 2
   and k = 3 and takes the larger of the two smallest d with a modelled error
   at most eps_hat (``bounds.probing_heuristic_d``).
2. Colour the graph at distance d (Algorithm 1, ``coloring``).
3. Evaluate each quadratic form v_l^T f(A) v_l by Lanczos until the
   a-posteriori estimate of Theorem 4.4 (the geometric mean of its lower and
   upper bounds, eq. error-bound-a-posteriori--estimate) is at most
   eps_hat |V_l| / n (eq. algorithm-probing-quadform-error-requirement-abs),
   so that the sum is within eps_hat of T_d (eq.
   algorithm-probing-krylov-error-requirement).
4. Return T_d = sum_l psi_l.

Readings where the paper leaves a choice open:

* eps_hat = eps/2 x S_hat with S_hat a rough value of S (Remark
  rem:algorithm-abs-vs-rel).  Here S_hat = T_1, a lower bound of S for a
  graph Laplacian (the probing lower bound of Section 3.1), and T_1 itself is
  evaluated with the relative rule |psi_l - psi_hat_l| <= (eps/2) psi_hat_l,
  which bounds the error of the sum by (eps/2) T_1 since every psi_l >= 0.
* The quadratic forms of one colouring form one block and stop together: the
  block stops at the first check (every `check` Lanczos steps) at which every
  column meets its tolerance, as the block Lanczos of the library does.  The
  spectral interval of the estimate is [lam_min, ||A||_G], lam_min <= 0
  meaning half the smallest positive Ritz value of each column.
* When neither k gives a decaying fit (q >= 1), d is chosen by the plain
  consecutive-difference estimate of the same section: the smallest d with
  |T_{d+1} - T_d| <= eps_hat, computing T_4, T_5, ... as needed.
* d never exceeds d_max; the report says when it was capped.
* Polynomial Lanczos is the Krylov method (the paper also allows rational
  Krylov; its a-posteriori estimate here is the polynomial case of
  Theorem 4.4).
"""
import math

import numpy as np

from .bounds import posterior_bounds, probing_heuristic_d
from .coloring import greedy_distance_coloring
from .density import gershgorin_norm
from .krylov import desingularize, gauss_quadrature, lanczos, tridiagonal_eig

RULE_FIT, RULE_DIFFERENCES, RULE_CAPPED = 0, 1, 2


def _column_state(alpha, beta, norm2, j, lam_min, lam_max, grid):
    """(psi, estimate) of one column after j steps (fewer on breakdown)."""
    k = len(alpha)
    jj = min(j, k)
    if jj == 0:
        return 0.0, 0.0
    psi = gauss_quadrature(alpha[:jj], beta[:jj - 1], norm2)
    if jj < j or beta[jj - 1] == 0.0:
        return psi, 0.0  # invariant Krylov space: the quadrature is exact
    lo = lam_min
    if not lo > 0.0:
        theta, _ = tridiagonal_eig(alpha[:jj], beta[:jj - 1])
        pos = theta[theta > 0.0]
        lo = 0.5 * float(pos.min()) if pos.size else 0.0
    if not (lo > 0.0 and lam_max > lo):
        return psi, math.inf  # no usable interval: not converged
    return psi, posterior_bounds(alpha[:jj], beta[:jj], norm2, lo, lam_max, grid=grid)[2]


def adaptive_quadforms(A, V, m_max, check, tol_rel=None, tol_abs=None, lam_min=0.0, grid=1000,
                       reorth="full"):
    """Quadratic forms c_l^T f(A) c_l (c_l = desingularised column l of V) of
    one block with the stopping rule above.  Exactly one of tol_rel (scalar)
    and tol_abs (one value per column) is given.  Returns (psi, steps)."""
    nA = gershgorin_norm(A)
    cols = []
    for l in range(V.shape[1]):
        c = desingularize(V[:, l])
        alpha, beta, _ = lanczos(A, c, m_max, reorth=reorth, norm_A=nA)
        cols.append((alpha, beta, float(c @ c)))
    j = 0
    while True:
        j = min(m_max, j + max(1, check))
        states = [_column_state(a, b, nb, j, lam_min, nA, grid) for a, b, nb in cols]
        psi = np.array([s[0] for s in states])
        if j >= m_max:
            return psi, j
        est = np.array([s[1] for s in states])
        tol = tol_rel * np.abs(psi) if tol_abs is None else np.asarray(tol_abs, float)
        if np.all(est <= tol):
            return psi, j


def choose_distance(T, eps_abs, d_max, more):
    """Step 1: the distance from T = [T_1, T_2, T_3] (heuristic fit), else by
    consecutive differences; `more(d)` returns T_d for d > 3 when needed.
    Returns (d, rule)."""
    d = probing_heuristic_d(T[0], T[1], T[2], eps_abs, d_max)
    if d is not None:
        return (d, RULE_FIT) if d <= d_max else (d_max, RULE_CAPPED)
    d = 1
    while True:
        if d >= d_max:
            return d_max, RULE_CAPPED
        if len(T) < d + 1:
            T.append(more(d + 1))
        if abs(T[d] - T[d - 1]) <= eps_abs:
            return d, RULE_DIFFERENCES
        d += 1


def probing_auto(A, graph, eps, m_max, check=5, d_max=64, lam_min=0.0, grid=1000, reorth="full",
                 coloring=None):
    """Algorithm 2 for S(A), A the density matrix of `graph`, relative target
    eps.  `coloring(d)` supplies the distance-d colouring (default: Algorithm
    1).  Returns (estimate, report) with report keys T (T_1, T_2, T_3, ...),
    eps_abs, d, rule, colors (colour count per d), steps (Lanczos steps per d)."""
    n = A.shape[0]
    rep = dict(T=[], colors={}, steps={}, psi={})

    def run(d, eps_abs):
        col = greedy_distance_coloring(graph, d) if coloring is None else np.asarray(coloring(d))
        s = int(col.max()) + 1
        V = np.zeros((n, s))
        V[np.arange(n), col] = 1.0
        if eps_abs is None:
            psi, steps = adaptive_quadforms(A, V, m_max, check, tol_rel=0.5 * eps, lam_min=lam_min, grid=grid,
                                            reorth=reorth)
        else:
            sizes = V.sum(axis=0)
            psi, steps = adaptive_quadforms(A, V, m_max, check, tol_abs=eps_abs * sizes / n, lam_min=lam_min,
                                            grid=grid, reorth=reorth)
        rep["colors"][d] = s
        rep["steps"][d] = steps
        rep["psi"][d] = psi
        return float(np.sum(psi))

    T = [run(1, None)]
    eps_abs = 0.5 * eps * T[0]
    T.append(run(2, eps_abs))
    T.append(run(3, eps_abs))
    d, rule = choose_distance(T, eps_abs, d_max, lambda dd: run(dd, eps_abs))
    est = T[d - 1] if d <= len(T) else run(d, eps_abs)
    rep.update(T=T, eps_abs=eps_abs, d=d, rule=rule)
    return est, rep
