"""Optimal distance-d colouring of the 2D grid graph with ceil((d+1)^2 / 2)
colours, the colouring the paper's scaling study uses for the grid (Section
6, after the cited construction for banded/lattice matrices).

Two grid nodes get the same colour only when they differ by a vector of a
lattice whose nonzero vectors all have L1 length >= d + 1, so nodes within
graph distance d always differ:

* d = 2r: the lattice of the perfect tiling of Z^2 by L1 balls of radius r,
  spanned by (r, r+1) and (r+1, -r), of index N = 2r^2 + 2r + 1; the colour
  of (i, j) is (i + k j) mod N with k = (r+1) r^{-1} mod N, a functional
  whose kernel is that lattice.
* d = 2r + 1: the lattice spanned by (r+1, r+1) and (r+1, -(r+1)), of index
  2(r+1)^2; with u = i + j and v = i - j the colour is (u mod M, v mod M),
  M = 2(r+1), two residues of equal parity, numbered (u mod M) M/2 +
  (v mod M) // 2.

This is an input a caller hands to the probing method (a colouring
callback); it is not part of the estimator's arithmetic.
"""
from __future__ import annotations

import math

import numpy as np


def colors_needed(d: int) -> int:
    return math.ceil((d + 1) ** 2 / 2)


def lattice_coloring(rows: int, cols: int, d: int) -> np.ndarray:
    """int32 colours of the rows x cols grid (node id = i * cols + j)."""
    if d < 1:
        raise ValueError("d must be >= 1")
    i, j = np.meshgrid(np.arange(rows, dtype=np.int64), np.arange(cols, dtype=np.int64), indexing="ij")
    if d % 2 == 0:
        r = d // 2
        N = 2 * r * r + 2 * r + 1
        k = ((r + 1) * pow(r, -1, N)) % N
        c = (i + k * j) % N
    else:
        M = d + 1  # 2(r + 1)
        u, v = (i + j) % M, (i - j) % M
        c = u * (M // 2) + v // 2
    return c.ravel().astype(np.int32)
