"""Polynomial Krylov (Lanczos) quadrature for b^T f(A) b (Section 4).

The approximation is psi_m = ||b||^2 e1^T f(A_m) e1 with A_m = V_m^T A V_m and
V_m an orthonormal basis of the Krylov space P_m(A, b) whose first column is
b / ||b|| (eq. rational-krylov-approximation-quadform, all poles at infinity).
For symmetric A the basis is built by the Lanczos three-term recurrence, so
A_m is the tridiagonal T_m = tridiag(beta, alpha, beta).  The matrix-vector
counterpart is f(A) b ~ ||b|| V_m f(A_m) e1
(eq. rational-krylov-approximation-matvec).

Implicit desingularisation (Remark graph-laplacian-krylov): when A 1 = 0 the
start vector b is replaced by c = b - (1^T b / n) 1.  Because f(A) 1 =
f(0) 1 = 0, b^T f(A) b = c^T f(A) c and f(A) b = f(A) c exactly.

Readings fixed here (the paper leaves them open):
* breakdown: the recurrence stops at step j when beta_j <= tau * ||A||_G
  (Gershgorin bound; tau = 1e-13), and T_j is used;
* reorthogonalisation: 'full' (classical Gram-Schmidt applied twice against
  all previous basis vectors), 'none' (plain three-term recurrence) or
  'partial' (Simon 1984, partial reorthogonalisation): the loss of
  orthogonality omega_{j+1,k} ~ v_{j+1}^T v_k is estimated by Simon's
  recurrence from the alpha's and beta's alone,
      beta_j omega_{j+1,k} = beta_k omega_{j,k+1} + (alpha_k - alpha_j) omega_{j,k}
                             + beta_{k-1} omega_{j,k-1} - beta_{j-1} omega_{j-1,k}
                             +- 2 eps ||A||,
  with omega_{j,j} = 1 and omega_{j+1,j} = eps; once max_k |omega_{j+1,k}|
  reaches sqrt(eps), w_{j+1} is orthogonalised (classical Gram-Schmidt,
  twice) against the v_k with |omega_{j+1,k}| >= eps^(3/4), those estimates
  are reset to eps, and the next vector is orthogonalised against the same
  set.  eps is the rounding unit of the arithmetic the policy models
  (2^-53 for float64, 2^-24 for float32).
"""
import math

import numpy as np
import scipy.linalg as sla

from .density import gershgorin_norm
from .entropy import f_entropy

BREAKDOWN_TAU = 1e-13


def desingularize(b):
    """c = b - (1^T b / n) 1 (applied per column for 2-D input)."""
    b = np.asarray(b, dtype=np.float64)
    return b - b.mean(axis=0, keepdims=True)


def lanczos(A, c, m, reorth="full", tau=BREAKDOWN_TAU, norm_A=None, keep_basis=False, eps=2.0 ** -53,
            stats=None):
    """m steps of Lanczos on symmetric A started at c / ||c||.

    Returns (alpha, beta, V): alpha[0..k-1] is the diagonal of T_k, beta[0..k-2]
    its off-diagonal, beta[k-1] the residual norm after the last step (0 on
    breakdown), k <= m the number of steps taken.  V (n x k) only if keep_basis
    or when needed for reorthogonalisation.  With reorth='partial', `eps` is
    the modelled rounding unit and `stats` (a dict, optional) receives the
    steps at which vectors were reorthogonalised and the omega estimates."""
    c = np.asarray(c, dtype=np.float64)
    n = c.shape[0]
    nrm = np.linalg.norm(c)
    if nrm == 0.0 or m <= 0:
        return np.zeros(0), np.zeros(0), np.zeros((n, 0))
    if norm_A is None:
        norm_A = gershgorin_norm(A)
    thresh = tau * norm_A
    store = keep_basis or reorth in ("full", "partial")
    V = np.zeros((n, m)) if store else None
    alpha = np.zeros(m)
    beta = np.zeros(m)
    v_prev = np.zeros(n)
    v = c / nrm
    b_prev = 0.0
    k = 0
    # partial reorthogonalisation state: omega rows j-1 and j (omega[j][i] ~ v_j . v_i)
    om_prev = np.zeros(m + 1)
    om = np.zeros(m + 1)
    om[0] = 1.0
    pending = None  # the set the next vector is orthogonalised against
    sq_eps, eta = math.sqrt(eps), eps ** 0.75
    reorth_steps, omegas = [], []
    for j in range(m):
        if store:
            V[:, j] = v
        w = A @ v - b_prev * v_prev
        a = float(v @ w)
        w = w - a * v
        if reorth == "full":
            for _ in range(2):
                w = w - V[:, : j + 1] @ (V[:, : j + 1].T @ w)
        alpha[j] = a
        b = float(np.linalg.norm(w))
        if reorth == "partial" and b > thresh:
            # omega_{j+1, i}, i = 0..j-1, by Simon's recurrence (0-based: beta[i]
            # couples v_i and v_{i+1})
            om_next = np.zeros(m + 1)
            for i in range(j):
                t = beta[i] * om[i + 1] + (alpha[i] - a) * om[i] - b_prev * om_prev[i]
                if i > 0:
                    t += beta[i - 1] * om[i - 1]
                t += math.copysign(2.0 * eps * norm_A, t)
                om_next[i] = t / b
            om_next[j] = eps
            om_next[j + 1] = 1.0
            sel = None
            if pending is not None:
                sel = pending
                pending = None
            elif j > 0 and np.max(np.abs(om_next[:j])) >= sq_eps:
                sel = np.nonzero(np.abs(om_next[: j + 1]) >= eta)[0]
                pending = sel
            if sel is not None and sel.size:
                Vs = V[:, sel]
                for _ in range(2):
                    w = w - Vs @ (Vs.T @ w)
                b = float(np.linalg.norm(w))
                om_next[sel] = eps
                reorth_steps.append(j)
            om_prev, om = om, om_next
            omegas.append(om_next[: j + 1].copy())
        k = j + 1
        if b <= thresh:
            beta[j] = 0.0
            break
        beta[j] = b
        v_prev, v, b_prev = v, w / b, b
    if stats is not None:
        stats["reorth_steps"] = reorth_steps
        stats["omega"] = omegas
    Vout = V[:, :k] if store else np.zeros((n, 0))
    return alpha[:k], beta[:k], Vout


def tridiagonal_eig(alpha, beta_off):
    """Eigenvalues theta and eigenvectors U of T = tridiag(beta_off, alpha, beta_off)."""
    if len(alpha) == 1:
        return np.array([alpha[0]]), np.ones((1, 1))
    return sla.eigh_tridiagonal(alpha, beta_off)


def gauss_quadrature(alpha, beta_off, norm2, f=f_entropy):
    """||c||^2 e1^T f(T) e1 = ||c||^2 sum_j u_{1j}^2 f(theta_j)."""
    if len(alpha) == 0:
        return 0.0
    theta, U = tridiagonal_eig(np.asarray(alpha, float), np.asarray(beta_off, float))
    return float(norm2 * np.sum(U[0, :] ** 2 * f(theta)))


def lanczos_quadform(A, b, m, reorth="full", desing=True, f=f_entropy, tau=BREAKDOWN_TAU, norm_A=None,
                     eps=2.0 ** -53):
    """psi_m ~ b^T f(A) b; returns (psi, alpha, beta) with beta the full length-k array."""
    c = desingularize(b) if desing else np.asarray(b, float)
    alpha, beta, _ = lanczos(A, c, m, reorth=reorth, tau=tau, norm_A=norm_A, eps=eps)
    norm2 = float(c @ c)
    psi = gauss_quadrature(alpha, beta[:-1], norm2, f)
    return psi, alpha, beta


def lanczos_fmatvec(A, b, m, reorth="full", desing=True, f=f_entropy, tau=BREAKDOWN_TAU, norm_A=None):
    """f(A) b ~ ||c|| V_m f(T_m) e1 (eq. rational-krylov-approximation-matvec)."""
    c = desingularize(b) if desing else np.asarray(b, float)
    alpha, beta, V = lanczos(A, c, m, reorth=reorth, tau=tau, norm_A=norm_A, keep_basis=True)
    if len(alpha) == 0:
        return np.zeros_like(c)
    theta, U = tridiagonal_eig(alpha, beta[:-1])
    z = U @ (f(theta) * U[0, :])
    return np.linalg.norm(c) * (V @ z)


def projected_quadform(A, V, c, f=f_entropy):
    """c^T V f(V^T A V) V^T c for V with orthonormal columns spanning a space
    that contains c: the projection definition of psi_m, basis independent."""
    Am = V.T @ (A @ V)
    Am = 0.5 * (Am + Am.T)
    lam, U = np.linalg.eigh(Am)
    y = U.T @ (V.T @ c)
    return float(np.sum(y ** 2 * f(lam)))
