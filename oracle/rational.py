"""Rational Krylov quadrature with negative real poles (Sections 4.2, 5.3).

With poles xi_1..xi_{m-1} the rational Krylov space is
Q_m(A, c) = { r(A) c : r = p_{m-1} / q_{m-1} }
(eq. rational-krylov-subspace-definition).  For distinct finite poles
xi_s = -s_s (s_s > 0) plus ell poles at infinity, partial fractions give

    Q_m(A, c) = span{ c, A c, ..., A^ell c, (A + s_1 I)^{-1} c, ..., (A + s_k I)^{-1} c },

m = 1 + ell + k.  The quadrature is psi_m = ||c||^2 e1^T f(A_m) e1 with
A_m = V_m^T A V_m and V_m an orthonormal basis whose first column is
c / ||c|| (eq. rational-krylov-approximation-quadform).  The paper builds V_m
by rational Arnoldi with full orthogonalisation (Remark rational-lanczos); the
oracle orthonormalises the spanning set above with modified Gram-Schmidt
applied twice, in the order listed.  In exact arithmetic rational Arnoldi
drops nothing (the spanning vectors of distinct poles are independent while
m does not exceed the number of distinct eigenvalues); in floating point a
vector whose remainder after the two passes is at the rounding level of its
norm (below 1e-12 of it) is numerically in the span of the earlier ones and
is dropped, which is the exact-arithmetic space up to rounding.

The shifted solves use dense LU (small n) or, for large n, one conjugate
gradient run per shift with relative residual 1e-10 -- the definition
x_s = (A + s I)^{-1} c, not a multi-shift recurrence.

Readings (the paper gives no formula for its EDS poles):
* default poles s_s = lam_hat * 10^(-4 (s-1) / 7), s = 1..8, log-spaced on
  [1e-4 lam_hat, lam_hat], lam_hat = ||A||_G (Gershgorin bound);
* ell = 2 poles at infinity for the x(1 - x) factor (Section 4.2).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .density import gershgorin_norm
from .entropy import f_entropy
from .krylov import desingularize, projected_quadform


def default_shifts(A, count=8, decades=4.0):
    lam_hat = gershgorin_norm(A)
    return lam_hat * 10.0 ** (-decades * np.arange(count) / (count - 1))


def shifted_solves(A, c, shifts, method="auto", rtol=1e-10):
    n = A.shape[0]
    if method == "auto":
        method = "dense" if n <= 6000 else "cg"
    X = np.zeros((n, len(shifts)))
    if method == "dense":
        Ad = A.toarray() if sp.issparse(A) else np.asarray(A)
        for k, s in enumerate(shifts):
            X[:, k] = np.linalg.solve(Ad + s * np.eye(n), c)
    else:
        I = sp.identity(n, format="csr")
        for k, s in enumerate(shifts):
            x, info = spla.cg(A + s * I, c, rtol=rtol, atol=0.0, maxiter=100000)
            if info != 0:
                raise RuntimeError(f"CG did not converge for shift {s}")
            X[:, k] = x
    return X


def rational_basis(A, c, shifts, n_inf=2, method="auto"):
    """Spanning set [c, A c, .., A^n_inf c, (A+s_1)^-1 c, ...] as columns."""
    cols = [c]
    w = c
    for _ in range(n_inf):
        w = A @ w
        cols.append(w)
    if len(shifts):
        X = shifted_solves(A, c, shifts, method=method)
        cols += [X[:, k] for k in range(X.shape[1])]
    return np.column_stack(cols)


def orthonormalize(W, drop=1e-12):
    """Modified Gram-Schmidt, two passes per vector, in column order; a vector
    whose remainder is at most drop times its norm is dependent (dropped)."""
    basis = []
    for j in range(W.shape[1]):
        w = W[:, j].astype(np.float64).copy()
        nw = np.linalg.norm(w)
        if nw == 0.0:
            continue
        for _ in range(2):
            for q in basis:
                w -= (q @ w) * q
        r = np.linalg.norm(w)
        if r > drop * nw:
            basis.append(w / r)
    return np.column_stack(basis) if basis else np.zeros((W.shape[0], 0))


def rational_quadform(A, b, shifts, n_inf=2, desing=True, f=f_entropy, method="auto"):
    c = desingularize(b) if desing else np.asarray(b, float)
    if np.linalg.norm(c) == 0.0:
        return 0.0
    V = orthonormalize(rational_basis(A, c, shifts, n_inf=n_inf, method=method))
    return projected_quadform(A, V, c, f=f)


# ---- mixed polynomial / rational Krylov (Section 5.3) ----
#
# The method first runs polynomial Krylov iterations (poles at infinity) and
# switches to the finite poles once the polynomial error estimate stalls: after
# iteration k it switches if err_est_k / err_est_{k-ell-1} >= c^ell (ell = 3,
# c = 0.75 in the paper).  Readings: err_est_k is the Theorem 4.4 estimate
# (geometric mean of the bounds, polynomial case) of the k-step Lanczos
# quadrature, whose space is K_k(A, c); the rule applies from k = ell + 2 on
# (the first k with an err_est_{k-ell-1}); an estimate of 0 (invariant Krylov
# space) ends the polynomial phase at that k; without a switch the phase ends
# at k_max.  The polynomial part of the space is K_k(A, c) (k - 1 poles at
# infinity), spanned here by the Lanczos vectors, which span the same space as
# the powers c, A c, .. and stay well conditioned for large k.

def switch_index(est, ell=3, cfac=0.75):
    """The k at which the polynomial phase ends; est[k-1] = err_est_k."""
    est = list(est)
    for k in range(1, len(est) + 1):
        e = est[k - 1]
        if e == 0.0:
            return k
        if k >= ell + 2 and e / est[k - ell - 2] >= cfac ** ell:
            return k
    return len(est)


def polynomial_estimates(A, c, k_max, lam_min=0.0, grid=1000):
    """err_est_k, k = 1..k_max (fewer on breakdown), and the Lanczos vectors
    (columns) of the k_max-step run with full reorthogonalisation."""
    from .bounds import posterior_bounds
    from .krylov import lanczos, tridiagonal_eig
    nA = gershgorin_norm(A)
    alpha, beta, V = lanczos(A, c, k_max, reorth="full", norm_A=nA, keep_basis=True)
    nb2 = float(c @ c)
    est = []
    for k in range(1, len(alpha) + 1):
        if beta[k - 1] == 0.0:
            est.append(0.0)
            break
        lo = lam_min
        if not lo > 0.0:
            theta, _ = tridiagonal_eig(alpha[:k], beta[:k - 1])
            pos = theta[theta > 0.0]
            lo = 0.5 * float(pos.min()) if pos.size else 0.0
        est.append(posterior_bounds(alpha[:k], beta[:k], nb2, lo, nA, grid=grid)[2] if lo > 0.0 else np.inf)
    return np.array(est), V


def mixed_quadform(A, b, shifts, ell=3, cfac=0.75, k_max=12, k_poly=None, desing=True, f=f_entropy,
                   method="auto", lam_min=0.0, grid=1000):
    """psi on K_k(A, c) + span{(A + s I)^{-1} c}, k from the switching rule
    (or k_poly when given).  Returns (psi, k from the rule)."""
    c = desingularize(b) if desing else np.asarray(b, float)
    if np.linalg.norm(c) == 0.0:
        return 0.0, 0
    est, V = polynomial_estimates(A, c, k_max, lam_min=lam_min, grid=grid)
    k_rule = switch_index(est, ell, cfac)
    k = k_rule if k_poly is None else k_poly
    cols = [V[:, j] for j in range(min(k, V.shape[1]))]
    if len(shifts):
        X = shifted_solves(A, c, shifts, method=method)
        cols += [X[:, s] for s in range(X.shape[1])]
    Q = orthonormalize(np.column_stack(cols))
    return projected_quadform(A, Q, c, f=f), k_rule
