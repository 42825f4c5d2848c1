"""Density matrix of a graph (Section 2, eq. graph_laplacian).

L = D - W with W the (binary) adjacency matrix and D = diag(W 1); the graph's
density matrix is rho = L / tr(L).  Written with scipy.sparse only.
"""
import numpy as np
import scipy.sparse as sp


def adjacency(graph) -> sp.csr_matrix:
    data = np.ones(graph.nnz, dtype=np.float64)
    return sp.csr_matrix((data, graph.col.astype(np.int64), graph.rowptr), shape=(graph.n, graph.n))


def laplacian(graph) -> sp.csr_matrix:
    """L = D - W, D = diag(W 1)."""
    W = adjacency(graph)
    deg = np.asarray(W.sum(axis=1)).ravel()
    return (sp.diags(deg) - W).tocsr()


def density_matrix(graph):
    """Return (rho, tr L) with rho = L / tr(L)."""
    L = laplacian(graph)
    tr = float(L.diagonal().sum())
    if tr <= 0:
        raise ValueError("graph has no edges: tr(L) = 0")
    return (L / tr).tocsr(), tr


def gershgorin_norm(A) -> float:
    """max_i sum_j |a_ij|, an upper bound on ||A||_2 for symmetric A."""
    A = sp.csr_matrix(A)
    return float(np.max(np.asarray(abs(A).sum(axis=1)).ravel())) if A.shape[0] else 0.0
