"""Error bounds and heuristics of the paper, written out.

* Theorem 2.2 (eq. entropy_polyapprox_integral_explicit):
  E_k(x log x, [a, b]) <= b (1 - sqrt g) (1 + g + 2 k sqrt g) / (4 (k^2 - 1))
                          * ((1 - sqrt g) / (1 + sqrt g))^k,  g = a / b, k >= 2.
* eq. entropy_polyapprox_Chebyshev: E_k(x log x, [0, b]) <= b / (2 k (k + 1)).
* Corollary 3.2 (eq. entropy_probing_bound): probing error with a distance-d
  colouring <= n b (1 - sqrt g)(1 + g + 2 d sqrt g) / (2 (d^2 - 1)) q^d.
* Proposition 4.2 with all poles at infinity (q = 1):
  |psi - psi_m| <= 2 ||b||^2 E_{2m-1}(f, [lam_min, lam_max]).
* Theorem 4.4 (eqs. error-bound--gm-definition, error-bound-a-posteriori):
  ||b||^2 min |g_m| <= |psi - psi_m| <= ||b||^2 max |g_m| on [lam_min, lam_max],
  and the geometric-mean estimate (eq. error-bound-a-posteriori--estimate).
  For the polynomial (Lanczos) case K_m = I and h_{m+1}^T = beta_m e_m^T.
* Section 5.1 heuristic for the probing distance d (eq.
  probing-heuristic-convergence) with k in {2, 3}.
"""
import math

import numpy as np

from .krylov import tridiagonal_eig


def thm22_bound(k, a, b):
    if k < 2:
        raise ValueError("Theorem 2.2 needs k >= 2")
    g = a / b
    sg = math.sqrt(g)
    return b * (1.0 - sg) * (1.0 + g + 2.0 * k * sg) / (4.0 * (k * k - 1.0)) * ((1.0 - sg) / (1.0 + sg)) ** k


def chebyshev_bound(k, b):
    return b / (2.0 * k * (k + 1.0))


def probing_bound(n, d, a, b):
    """Corollary 3.2 (d >= 2): 2 n E_d(f, [a, b]) written out."""
    return 2.0 * n * thm22_bound(d, a, b)


def lanczos_apriori_bound(norm2, m, lam_min, lam_max):
    """Proposition 4.2 with q_{m-1} = 1 and Theorem 2.2 for E_{2m-1} (m >= 2)."""
    return 2.0 * norm2 * thm22_bound(2 * m - 1, lam_min, lam_max)


# ---- a-posteriori bound (Theorem 4.4), polynomial Krylov special case ----

def _f(x):
    return -x * np.log(x)


def _df(x):
    return -np.log(x) - 1.0


def _d2f(x):
    return -1.0 / x


def gm_coefficients(alpha, beta):
    """(theta, a_j, b_j, gamma_j) of eq. error-bound--gm-definition for the
    Lanczos decomposition A V_m = V_m T_m + beta_m v_{m+1} e_m^T.
    alpha: diag of T_m (length m); beta: length-m array, beta[:-1] the
    off-diagonal and beta[-1] = beta_m."""
    m = len(alpha)
    theta, U = tridiagonal_eig(np.asarray(alpha, float), np.asarray(beta[:-1], float))
    a = beta[-1] * U[m - 1, :]          # h_{m+1}^T K_m^{-1} U_m with K_m = I
    bb = U[0, :]                        # U_m^T e1
    gam = np.zeros(m)
    for j in range(m):
        for l in range(m):
            if l != j:
                gam[j] += a[l] * bb[l] / (theta[j] - theta[l])
    return theta, a, bb, gam


def _dd1_dd2(z, t):
    """Divided differences of f(x) = -x log x: f[t, z] and f[t, t, z].

    With z = t (1 + u) they are -log t - h(u) and (1 - h(u)) / (t u), where
    h(u) = (1 + u) log(1 + u) / u; near u = 0 the power series
    1 - h(u) = sum_{k>=1} (-1)^k u^k / (k (k + 1)) replaces the quotient, so
    the values stay accurate however close z is to t (the plain quotients of
    eq. error-bound--gm-definition cancel catastrophically there).  At u = 0
    they are f'(t) and f''(t) / 2, the limits the definition states."""
    z = np.asarray(z, float)
    u = (z - t) / t
    small = np.abs(u) < 0.1
    us = np.where(small, u, 0.0)
    ser = np.zeros_like(u)          # (1 - h(u)) / u, series
    p = np.ones_like(u)
    for k in range(1, 40):
        ser += ((-1.0) ** k) * p / (k * (k + 1))
        p = p * us
    ul = np.where(small, 1.0, u)
    h_large = (1.0 + ul) * np.log1p(ul) / ul
    one_minus_h = np.where(small, ser * us, 1.0 - h_large)
    dd1 = -np.log(t) - (1.0 - one_minus_h)
    dd2 = np.where(small, ser, (1.0 - h_large) / ul) / t
    return dd1, dd2


def gm_eval(z, theta, a, bb, gam):
    """g_m(z) of eq. error-bound--gm-definition: the sum over j of
    a_j^2 b_j^2 f[theta_j, theta_j, z] + 2 a_j b_j gamma_j f[theta_j, z]
    (divided differences of f, evaluated stably by _dd1_dd2)."""
    z = np.atleast_1d(np.asarray(z, float))
    out = np.zeros_like(z)
    for j in range(len(theta)):
        ab = a[j] * bb[j]
        dd1, dd2 = _dd1_dd2(z, theta[j])
        out += ab * ab * dd2 + 2.0 * ab * gam[j] * dd1
    return out


def posterior_bounds(alpha, beta, norm2, lam_min, lam_max, grid=4000):
    """(lower, upper, estimate) of Theorem 4.4 / eq. error-bound-a-posteriori--estimate,
    with min/max of |g_m| taken over a grid of [lam_min, lam_max] plus the Ritz values."""
    theta, a, bb, gam = gm_coefficients(alpha, beta)
    z = np.unique(np.concatenate([np.geomspace(lam_min, lam_max, grid),
                                  np.linspace(lam_min, lam_max, grid),
                                  theta[(theta >= lam_min) & (theta <= lam_max)]]))
    g = np.abs(gm_eval(z, theta, a, bb, gam))
    lo, hi = float(g.min()), float(g.max())
    return norm2 * lo, norm2 * hi, norm2 * math.sqrt(lo * hi)


# ---- probing heuristic (Section 5.1) ----

def probing_heuristic_d(T1, T2, T3, eps_abs, d_max=64):
    """d* = max over k in {2, 3} of min{d : C q^d / d^k <= eps_abs}, with C, q
    fitted from |T_{d+1} - T_d| = C q^d / d^k at d = 1, 2.  A k whose fitted q
    is >= 1 does not describe a decaying error and is skipped; None when
    neither k fits.  Degenerate data: e1 = 0 means C = 0 (d = 1); e2 = 0 means
    q = 0, a modelled error of e1 at d = 1 and 0 from d = 2 on."""
    e1, e2 = abs(T2 - T1), abs(T3 - T2)
    if e1 == 0.0:
        return 1
    if e2 == 0.0:
        return 1 if e1 <= eps_abs else 2
    best = None
    for k in (2, 3):
        q = (2.0 ** k) * e2 / e1
        if q >= 1.0:
            continue
        C = e1 / q
        d = 1
        while d <= d_max and C * q ** d / d ** k > eps_abs:
            d += 1
        best = d if best is None else max(best, d)
    return best


def probing_quadform_tolerance(eps_abs, class_size, n):
    """eq. algorithm-probing-quadform-error-requirement-abs."""
    return eps_abs * class_size / n
