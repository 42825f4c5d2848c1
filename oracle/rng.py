"""Counter-based Rademacher probes (oracle side; independent of the CUDA side).

The paper draws Gaussian probes for Hutchinson / Hutch++ (Section 3.2); this
build uses Rademacher (+-1) entries, which satisfy the same requirement
E[x x^T] = I.  Both sides must produce identical vectors without sharing code,
so the generator is fixed by its published definition:

  mix64(z)      -- the SplitMix64 output mixer (Steele, Lea, Flood, "Fast
                   splittable pseudorandom number generators", OOPSLA 2014):
                   z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
                   z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31
  gamma         -- 0x9E3779B97F4A7C15 (the SplitMix64 increment)
  s             -- mix64(seed + gamma)
  h(j, i)       -- mix64((((j << 32) | i) XOR s) + gamma)       (mod 2^64)
  x_i^{(j)}     -- +1 if the top bit of h(j, i) is 0, else -1

j is the global probe index (column), i the node index in the caller's
numbering.  Hutch++ uses columns 0..N_r-1 for the sketch Omega and
N_r..N_r+N_H-1 for the Hutchinson vectors G.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix64_stream(seed: int, count: int) -> np.ndarray:
    """The SplitMix64 sequence: k-th output = mix64(seed + k * gamma), k = 1..count."""
    k = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(np.uint64(seed) + k * GAMMA)


def hash_entries(seed: int, cols, rows) -> np.ndarray:
    """h(j, i) for broadcast arrays of column indices j and row indices i."""
    with np.errstate(over="ignore"):
        s = mix64(np.uint64(seed & (2**64 - 1)) + GAMMA)
        key = (np.asarray(cols, dtype=np.uint64) << np.uint64(32)) | np.asarray(rows, dtype=np.uint64)
        return mix64((key ^ s) + GAMMA)


def rademacher(seed: int, n: int, col_begin: int, col_count: int, rows=None) -> np.ndarray:
    """n x col_count matrix of +-1 (float64), columns col_begin..col_begin+col_count-1.

    ``rows`` optionally gives the node index used for each of the n rows
    (defaults to 0..n-1)."""
    r = np.arange(n, dtype=np.uint64) if rows is None else np.asarray(rows, dtype=np.uint64)
    c = np.arange(col_begin, col_begin + col_count, dtype=np.uint64)
    h = hash_entries(seed, c[None, :], r[:, None])
    return np.where((h >> np.uint64(63)) == 0, 1.0, -1.0)


# ---- Gaussian probes (the paper's distribution, Section 3.2) ----
#
# Box-Muller on the same counters (Box & Muller, "A note on the generation of
# random normal deviates", Ann. Math. Statist. 1958):
#   h1 = h(j, i),  h2 = mix64(h1 + gamma)
#   u1 = ((h1 >> 11) + 1/2) 2^-53  in (0, 1),   u2 = (h2 >> 11) 2^-53  in [0, 1)
#   x_i^{(j)} = sqrt(-2 log u1) cos(2 pi u2)
# in FP64 on both sides (the two sides' log and cos may differ in the last
# bits, so the vectors agree to rounding, not bit for bit).

def gaussian(seed: int, n: int, col_begin: int, col_count: int, rows=None) -> np.ndarray:
    """n x col_count standard normal entries, columns col_begin.. (see above)."""
    r = np.arange(n, dtype=np.uint64) if rows is None else np.asarray(rows, dtype=np.uint64)
    c = np.arange(col_begin, col_begin + col_count, dtype=np.uint64)
    h1 = hash_entries(seed, c[None, :], r[:, None])
    with np.errstate(over="ignore"):
        h2 = mix64(h1 + GAMMA)
    u1 = ((h1 >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    u2 = (h2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def probes(seed: int, n: int, col_begin: int, col_count: int, rows=None, dist: str = "rademacher") -> np.ndarray:
    if dist == "gaussian":
        return gaussian(seed, n, col_begin, col_count, rows)
    return rademacher(seed, n, col_begin, col_count, rows)
