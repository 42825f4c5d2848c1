"""Trace estimators for S(A) = tr f(A) (Section 3).

* Hutchinson (eq. hutchinson-stochastic-trace-estimator):
      tr_N(B) = (1/N) sum_j x_j^T B x_j.
* Hutch++ (eq. Hutch++_formula):
      tr(Q^T B Q) + tr_{N_H}((I - Q Q^T) B (I - Q Q^T)),
  Q an orthonormal basis of range(B Omega), Omega with N_r columns; the cost is
  N_r products B x and N_r + N_H quadratic forms.
* Probing (eqs. probing_vectors, trace_probing):
      T_d = sum_l v_l^T f(A) v_l,  v_l = sum_{i in V_l} e_i.

B = f(A) is applied through Lanczos (module krylov).  Probes are Rademacher
(module rng).  Hutch++ takes its sketch from probe columns 0..N_r-1 and its
Hutchinson vectors from columns N_r..N_r+N_H-1.

orth() in eq. Hutch++_formula is any orthonormal basis of range(B Omega).
With exact quadratic forms the estimate does not depend on the choice, but
tr(Q^T B Q) is evaluated here as a sum of Lanczos quadratures psi_m(q_i),
which is not invariant under rotations of Q.  The oracle therefore fixes
orth() as the column-pivoted QR factorisation Y P = Q R (Businger and Golub
1965: at every step the column with the largest norm after projecting out
the chosen ones is taken), R with a positive diagonal, truncated at the
numerical rank; this is a unique Q, and it is the factorisation a pivoted
Cholesky of Y^T Y computes.
"""
import numpy as np

from .density import gershgorin_norm
from .entropy import f_entropy
from .krylov import lanczos_quadform, lanczos_fmatvec
from .rng import probes, rademacher


def quadforms(A, X, m, reorth="full", desing=True, f=f_entropy):
    """psi_m for every column of X (each column its own Krylov space)."""
    nA = gershgorin_norm(A)
    return np.array([lanczos_quadform(A, X[:, j], m, reorth=reorth, desing=desing, f=f, norm_A=nA)[0]
                     for j in range(X.shape[1])])


def hutchinson(A, num_vectors, m, seed, reorth="full", col_begin=0, rows=None, dist="rademacher"):
    """Returns (estimate, psi) for Rademacher (or Gaussian) probes of columns col_begin.."""
    X = probes(seed, A.shape[0], col_begin, num_vectors, rows=rows, dist=dist)
    psi = quadforms(A, X, m, reorth=reorth)
    return float(np.mean(psi)) if num_vectors else 0.0, psi


def orthonormal_range(Y, rtol=None, return_pivots=False):
    """Q of the column-pivoted QR factorisation Y P = Q R (Householder, via
    LAPACK geqp3), columns in pivot order, signs chosen so that diag(R) > 0,
    truncated at the numerical rank: the pivots with |R_jj| > rtol |R_11|
    (default rtol = max(n, k) * eps)."""
    import scipy.linalg as sla
    k = Y.shape[1]
    if k == 0:
        return (Y, np.zeros(0, dtype=np.int64)) if return_pivots else Y
    Q, R, piv = sla.qr(np.asarray(Y, dtype=np.float64), mode="economic", pivoting=True)
    if rtol is None:
        rtol = max(Y.shape) * np.finfo(np.float64).eps
    d = np.abs(np.diag(R))
    r = 0 if d.size == 0 or d[0] == 0.0 else int(np.sum(d > rtol * d[0]))
    sgn = np.where(np.diag(R)[:r] < 0.0, -1.0, 1.0)
    Q = Q[:, :r] * sgn
    return (Q, piv[:r].astype(np.int64)) if return_pivots else Q


def hutchpp(A, n_sketch, n_hutch, m, seed, reorth="full", rows=None, return_parts=False, dist="rademacher"):
    """Hutch++ estimate of tr f(A) (eq. Hutch++_formula)."""
    n = A.shape[0]
    nA = gershgorin_norm(A)
    Omega = probes(seed, n, 0, n_sketch, rows=rows, dist=dist)
    Y = np.column_stack([lanczos_fmatvec(A, Omega[:, j], m, reorth=reorth, norm_A=nA)
                         for j in range(n_sketch)]) if n_sketch else np.zeros((n, 0))
    Q, piv = orthonormal_range(Y, return_pivots=True)
    psi_q = np.array([lanczos_quadform(A, Q[:, i], m, reorth=reorth, norm_A=nA)[0]
                      for i in range(Q.shape[1])])
    G = probes(seed, n, n_sketch, n_hutch, rows=rows, dist=dist)
    Gp = G - Q @ (Q.T @ G)
    psi_g = np.array([lanczos_quadform(A, Gp[:, j], m, reorth=reorth, norm_A=nA)[0]
                      for j in range(n_hutch)])
    low_rank = float(np.sum(psi_q))
    resid = float(np.mean(psi_g)) if n_hutch else 0.0
    est = low_rank + resid
    if return_parts:
        return est, dict(Y=Y, Q=Q, pivots=piv, psi_q=psi_q, psi_g=psi_g, low_rank=low_rank, resid=resid)
    return est


def served_hutchpp(A, eps, block, m, seed, n_sketch=4, max_vectors=8192, quad_tol=None, check_every=5,
                   grid=256, reorth="none", sketch_steps=None):
    """The adaptive Hutch++ proxy of a served query (readings R31, R33): the
    Hutch++ estimate of eq. Hutch++_formula with a sketch of `n_sketch`
    columns (probe columns 0..n_sketch-1, Y = f(A) Omega by Lanczos with
    `sketch_steps` steps (default m), Q = orth(Y) and the quadratic forms
    psi(q_i)), then blocks of `block` deflated probes g' = (I - Q Q^T) g
    (probe columns n_sketch + b * block ...) until, after at least two blocks,
    2.576 stderr(psi(g')) <= (eps / 2) |sum psi(q_i) + mean psi(g')|, or
    max_vectors probes.

    quad_tol (R33): the Lanczos runs of a block of quadratic forms (the
    psi(q_i) as one block, then each block of deflated probes) stop together
    at the first multiple j of check_every below m at which every column's
    a-posteriori estimate of Theorem 4.4 (eq.
    error-bound-a-posteriori--estimate: the geometric mean of the bounds, with
    lam_min half the column's smallest positive Ritz value and lam_max the
    Gershgorin bound of A; the min and max of |g_m| over `grid` geometric and
    `grid` linear points of that interval and the Ritz values in it) is at
    most quad_tol |psi_j|; else after m steps.  None: always m steps.

    Returns (estimate, std_error, vectors, block_steps, sketch_form_steps)."""
    from .bounds import posterior_bounds
    from .krylov import desingularize, gauss_quadrature, lanczos, tridiagonal_eig
    n = A.shape[0]
    nA = gershgorin_norm(A)
    ms = m if sketch_steps is None else sketch_steps
    Omega = probes(seed, n, 0, n_sketch)
    Y = np.column_stack([lanczos_fmatvec(A, Omega[:, j], ms, reorth=reorth, norm_A=nA) for j in range(n_sketch)])
    Q = orthonormal_range(Y)

    def block_psi(Gp):
        runs = []
        for j in range(Gp.shape[1]):
            c = desingularize(Gp[:, j])
            alpha, beta, _ = lanczos(A, c, m, reorth=reorth, norm_A=nA)
            runs.append((alpha, beta, float(c @ c)))

        def psi_at(run, k):
            alpha, beta, nb = run
            k = min(k, len(alpha))
            return gauss_quadrature(alpha[:k], beta[:k - 1], nb) if k else 0.0

        def estimate_at(run, k):
            alpha, beta, nb = run
            if len(alpha) < k or beta[k - 1] == 0.0:
                return 0.0  # the Krylov space is invariant: exact
            theta, _ = tridiagonal_eig(alpha[:k], beta[:k - 1])
            pos = theta[theta > 0.0]
            if pos.size == 0:
                return np.inf
            return posterior_bounds(alpha[:k], beta[:k], nb, 0.5 * float(pos.min()), nA, grid=grid)[2]

        steps = m
        if quad_tol is not None:
            for k in range(check_every, m, check_every):
                if all(estimate_at(r, k) <= quad_tol * abs(psi_at(r, k)) for r in runs):
                    steps = k
                    break
        return np.array([psi_at(r, steps) for r in runs]), steps

    # the quadratic forms of the basis vectors, as one block
    psi_q, q_steps = block_psi(Q) if Q.shape[1] else (np.zeros(0), 0)
    low = float(np.sum(psi_q))
    psi_all, steps_all = [], []
    b = 0
    while True:
        G = probes(seed, n, n_sketch + b * block, block)
        psi, steps = block_psi(G - Q @ (Q.T @ G))
        psi_all.extend(psi.tolist())
        steps_all.append(steps)
        b += 1
        x = np.array(psi_all)
        est = low + float(np.mean(x))
        se = float(np.std(x, ddof=1) / np.sqrt(len(x))) if len(x) > 1 else 0.0
        if (b >= 2 and 2.576 * se <= 0.5 * eps * abs(est)) or len(x) >= max_vectors:
            return est, se, len(x), steps_all, q_steps


def probing_vectors(colors, n_colors=None):
    """n x s 0/1 matrix with column l the indicator of colour class l (eq. probing_vectors)."""
    colors = np.asarray(colors, dtype=np.int64)
    s = int(colors.max()) + 1 if n_colors is None else int(n_colors)
    V = np.zeros((colors.size, s))
    V[np.arange(colors.size), colors] = 1.0
    return V


def probing(A, colors, m, reorth="full"):
    """T_d = sum_l psi(v_l) (eq. trace_probing); returns (T_d, psi per colour)."""
    V = probing_vectors(colors)
    psi = quadforms(A, V, m, reorth=reorth)
    return float(np.sum(psi)), psi


def probing_exact(Fdense, colors):
    """sum_l v_l^T F v_l for an explicit dense F = f(A) (no Krylov error)."""
    V = probing_vectors(colors)
    return float(np.sum(V * (Fdense @ V)))
