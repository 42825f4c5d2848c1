"""GB300-native von Neumann entropy of large sparse density matrices.

Benzi, Rinelli, Simunec, "Computation of the von Neumann entropy of large
matrices via trace estimators and rational Krylov methods": S(A) = tr f(A),
f(x) = -x log x, estimated from many quadratic forms v^T f(A) v evaluated at
once by Lanczos Gauss quadrature (Section 4) inside Hutchinson, Hutch++ or
probing trace estimators (Section 3).

Submodules are imported lazily: ``graphs`` (seeded input graphs, no CUDA) and
``vne`` (the ctypes binding of the C-ABI library ``libvne.so``).
"""
__all__ = ["graphs", "vne"]
