"""Von Neumann entropy by its definition (Section 2).

S(rho) = -sum_{lambda in sigma(rho)} lambda log lambda with 0 log 0 = 0 and
the natural logarithm (eq. entropy_definition_eigenvalues).  The spectrum is
taken from a dense symmetric eigendecomposition (numpy.linalg.eigh), the sum
with math.fsum.  Eigenvalues that rounding pushes slightly below zero carry
f = 0, the same convention as 0 log 0 = 0.

Closed-form Laplacian spectra of classic graph families pin the whole chain
(graph -> Laplacian -> density -> eigenvalues -> entropy).
"""
import math

import numpy as np
import scipy.sparse as sp


def f_entropy(x):
    """f(x) = -x log x, with f(x) = 0 for x <= 0 (0 log 0 = 0)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    pos = x > 0
    out[pos] = -x[pos] * np.log(x[pos])
    return out


def entropy_from_eigenvalues(lams) -> float:
    return math.fsum(f_entropy(np.asarray(lams, dtype=np.float64)).tolist())


def dense(A) -> np.ndarray:
    return A.toarray() if sp.issparse(A) else np.asarray(A, dtype=np.float64)


def dense_entropy(A) -> float:
    """S(A) from numpy.linalg.eigvalsh of the dense matrix."""
    return entropy_from_eigenvalues(np.linalg.eigvalsh(dense(A)))


def dense_matrix_function(A, f=f_entropy) -> np.ndarray:
    """f(A) = U f(Lambda) U^T (Section 3 opening paragraph)."""
    lam, U = np.linalg.eigh(dense(A))
    return (U * f(lam)[None, :]) @ U.T


def scaled_entropy(S_A: float, gamma: float, trace_A: float) -> float:
    """S(gamma A) = gamma S(A) - gamma log(gamma) tr(A)  (eq. entropy_normalization)."""
    return gamma * S_A - gamma * math.log(gamma) * trace_A


# --------------------------------------------------------------------------
# closed-form Laplacian spectra (unnormalised L = D - W)

def spectrum_complete(n):
    return np.array([0.0] + [float(n)] * (n - 1))


def spectrum_path(n):
    k = np.arange(n)
    return 2.0 - 2.0 * np.cos(np.pi * k / n)


def spectrum_cycle(n):
    k = np.arange(n)
    return 2.0 - 2.0 * np.cos(2.0 * np.pi * k / n)


def spectrum_star(n):
    return np.array([0.0] + [1.0] * (n - 2) + [float(n)])


def spectrum_complete_bipartite(a, b):
    return np.array([0.0] + [float(a)] * (b - 1) + [float(b)] * (a - 1) + [float(a + b)])


def spectrum_hypercube(d):
    out = []
    for i in range(d + 1):
        out += [2.0 * i] * math.comb(d, i)
    return np.array(out)


def spectrum_cartesian(s1, s2):
    """Laplacian spectrum of a Cartesian product graph: all sums mu_i + nu_j."""
    return (np.asarray(s1)[:, None] + np.asarray(s2)[None, :]).ravel()


def spectrum_grid(rows, cols, periodic=False):
    f = spectrum_cycle if periodic else spectrum_path
    return spectrum_cartesian(f(rows), f(cols))


def entropy_from_laplacian_spectrum(lams) -> float:
    """Entropy of rho = L / tr(L) given the spectrum of L (tr L = sum of eigenvalues)."""
    lams = np.asarray(lams, dtype=np.float64)
    tr = math.fsum(lams.tolist())
    return entropy_from_eigenvalues(lams / tr)
