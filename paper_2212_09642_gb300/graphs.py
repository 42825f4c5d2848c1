"""Seeded synthetic graph inputs (shared by the oracle and the GPU path).

This module only draws graphs.  It contains none of the entropy method's
arithmetic: no Laplacian, no trace, no probe vectors.  Every generator returns
a :class:`Graph`, an undirected simple graph stored as a symmetric CSR
*pattern* (int64 ``rowptr`` of length n+1, int32 ``col`` with sorted columns,
no self-loops, no duplicates).  The density matrix rho = L / tr(L) of
Section 2 (eq. graph_laplacian) is built from this pattern separately by each
side.

The paper's experiments (Section 6, Table 1) use SuiteSparse networks, which
are not available; these seeded families stand in for them:

* large-world road networks  -> random geometric graphs (RGG),
* small-world social/collaboration networks -> Barabasi-Albert (BA),
  Erdos-Renyi (ER) and Watts-Strogatz (WS),
* closed-form families (complete, path, cycle, star, complete bipartite,
  hypercube, 2D grid, torus) whose Laplacian spectra are known exactly.

The heavy generators live in ``gen/graphgen.c`` (compiled on first use with
the host C compiler; plain C, no architecture flags).
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_GEN_SRC = os.path.join(_HERE, "gen", "graphgen.c")
_GEN_LIB = os.path.join(_HERE, "gen", "libgraphgen.so")
_GEN_STAMP = os.path.join(_HERE, "gen", "libgraphgen.stamp")
_lock = threading.Lock()
_lib = None


@dataclasses.dataclass
class Graph:
    """Undirected simple graph as a symmetric CSR pattern."""

    n: int
    rowptr: np.ndarray  # int64 [n+1]
    col: np.ndarray  # int32 [nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @property
    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr)

    def edges(self):
        """Return (u, v) arrays with u > v, one entry per undirected edge."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), self.degrees)
        c = self.col.astype(np.int64)
        keep = rows > c
        return rows[keep], c[keep]


def build_generator_library(force: bool = False) -> str:
    """Compile ``gen/graphgen.c`` into a shared library (idempotent)."""
    import hashlib
    import platform
    with open(_GEN_SRC, "rb") as fh:
        tag = f"{platform.machine()}:{hashlib.sha256(fh.read()).hexdigest()}"
    with _lock:
        stale = (not os.path.exists(_GEN_LIB)) or (not os.path.exists(_GEN_STAMP)) or (
            open(_GEN_STAMP).read() != tag)
        if force or stale:
            tmp = _GEN_LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11",
                   _GEN_SRC, "-o", tmp, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _GEN_LIB)
            with open(_GEN_STAMP, "w") as fh:
                fh.write(tag)
    return _GEN_LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build_generator_library()
    lib = ctypes.CDLL(_GEN_LIB)
    p64 = ctypes.POINTER(ctypes.POINTER(ctypes.c_int64))
    pi64 = ctypes.POINTER(ctypes.c_int64)
    lib.gg_erdos_renyi.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, p64, p64, pi64]
    lib.gg_barabasi_albert.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, p64, p64, pi64]
    lib.gg_watts_strogatz.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64,
                                      p64, p64, pi64]
    lib.gg_random_geometric.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, p64, p64, pi64]
    lib.gg_edges_to_csr.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                    p64, ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))]
    lib.gg_free.argtypes = [ctypes.c_void_p]
    for f in (lib.gg_erdos_renyi, lib.gg_barabasi_albert, lib.gg_watts_strogatz,
              lib.gg_random_geometric, lib.gg_edges_to_csr):
        f.restype = ctypes.c_int
    _lib = lib
    return lib


def _take(ptr, count, dtype):
    if count == 0:
        return np.zeros(0, dtype=dtype)
    ctype = ctypes.c_int64 if dtype == np.int64 else ctypes.c_int32
    buf = ctypes.cast(ptr, ctypes.POINTER(ctype * count)).contents
    out = np.frombuffer(buf, dtype=dtype).copy()
    return out


def _edges_call(fn, *args):
    lib = _load()
    eu = ctypes.POINTER(ctypes.c_int64)()
    ev = ctypes.POINTER(ctypes.c_int64)()
    ne = ctypes.c_int64(0)
    rc = fn(*args, ctypes.byref(eu), ctypes.byref(ev), ctypes.byref(ne))
    if rc != 0:
        raise RuntimeError(f"graph generator failed with code {rc}")
    u = _take(eu, ne.value, np.int64)
    v = _take(ev, ne.value, np.int64)
    if ne.value:
        lib.gg_free(ctypes.cast(eu, ctypes.c_void_p))
        lib.gg_free(ctypes.cast(ev, ctypes.c_void_p))
    return u, v


def from_edges(n: int, u: np.ndarray, v: np.ndarray, name: str = "") -> Graph:
    """Symmetric CSR pattern from an undirected edge list (self-loops dropped,
    duplicates merged, columns sorted)."""
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.int64)
    v = np.ascontiguousarray(v, dtype=np.int64)
    rp = ctypes.POINTER(ctypes.c_int64)()
    cp = ctypes.POINTER(ctypes.c_int32)()
    rc = lib.gg_edges_to_csr(int(n), u.ctypes.data, v.ctypes.data, int(u.size),
                             ctypes.byref(rp), ctypes.byref(cp))
    if rc != 0:
        raise RuntimeError(f"CSR assembly failed with code {rc}")
    rowptr = _take(rp, n + 1, np.int64)
    col = _take(cp, int(rowptr[-1]), np.int32)
    lib.gg_free(ctypes.cast(rp, ctypes.c_void_p))
    lib.gg_free(ctypes.cast(cp, ctypes.c_void_p))
    return Graph(int(n), rowptr, col, name)


# ----------------------------------------------------------------------------
# random families

def erdos_renyi(n: int, p: float, seed: int) -> Graph:
    u, v = _edges_call(_load().gg_erdos_renyi, int(n), float(p), int(seed) & (2**64 - 1))
    return from_edges(n, u, v, f"ER(n={n},p={p},seed={seed})")


def barabasi_albert(n: int, m: int, seed: int) -> Graph:
    u, v = _edges_call(_load().gg_barabasi_albert, int(n), int(m), int(seed) & (2**64 - 1))
    return from_edges(n, u, v, f"BA(n={n},m={m},seed={seed})")


def watts_strogatz(n: int, k: int, beta: float, seed: int) -> Graph:
    u, v = _edges_call(_load().gg_watts_strogatz, int(n), int(k), float(beta), int(seed) & (2**64 - 1))
    return from_edges(n, u, v, f"WS(n={n},k={k},beta={beta},seed={seed})")


def random_geometric(n: int, radius: float, seed: int) -> Graph:
    u, v = _edges_call(_load().gg_random_geometric, int(n), float(radius), int(seed) & (2**64 - 1))
    return from_edges(n, u, v, f"RGG(n={n},r={radius:.3e},seed={seed})")


def rgg_radius_for_degree(n: int, avg_degree: float) -> float:
    """Radius giving expected degree ``avg_degree`` for n uniform points in the unit square."""
    return math.sqrt(avg_degree / (math.pi * n))


# ----------------------------------------------------------------------------
# closed-form families

def complete(n: int) -> Graph:
    a, b = np.tril_indices(n, -1)
    return from_edges(n, a, b, f"K{n}")


def path(n: int) -> Graph:
    a = np.arange(1, n)
    return from_edges(n, a, a - 1, f"P{n}")


def cycle(n: int) -> Graph:
    a = np.arange(n)
    return from_edges(n, a, (a + 1) % n, f"C{n}")


def star(n: int) -> Graph:
    a = np.arange(1, n)
    return from_edges(n, a, np.zeros_like(a), f"S{n}")


def complete_bipartite(a: int, b: int) -> Graph:
    x, y = np.meshgrid(np.arange(a), np.arange(a, a + b), indexing="ij")
    return from_edges(a + b, x.ravel(), y.ravel(), f"K{a},{b}")


def hypercube(d: int) -> Graph:
    n = 1 << d
    nodes = np.arange(n)
    us, vs = [], []
    for bit in range(d):
        nb = nodes ^ (1 << bit)
        keep = nb > nodes
        us.append(nodes[keep]); vs.append(nb[keep])
    return from_edges(n, np.concatenate(us), np.concatenate(vs), f"Q{d}")


def grid2d(rows: int, cols: int, periodic: bool = False) -> Graph:
    """rows x cols grid (node id = r * cols + c); periodic=True gives the torus."""
    r, c = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    idx = r * cols + c
    us, vs = [], []
    if periodic:
        us += [idx.ravel(), idx.ravel()]
        vs += [(r * cols + (c + 1) % cols).ravel(), (((r + 1) % rows) * cols + c).ravel()]
    else:
        us += [idx[:, :-1].ravel(), idx[:-1, :].ravel()]
        vs += [idx[:, 1:].ravel(), idx[1:, :].ravel()]
    name = ("T" if periodic else "G") + f"{rows}x{cols}"
    return from_edges(rows * cols, np.concatenate(us), np.concatenate(vs), name)


def disjoint_union(graphs) -> Graph:
    """Block-diagonal union of several graphs (node ids shifted)."""
    off = 0
    us, vs = [], []
    for g in graphs:
        a, b = g.edges()
        us.append(a + off); vs.append(b + off)
        off += g.n
    if not us:
        return Graph(0, np.zeros(1, np.int64), np.zeros(0, np.int32), "empty")
    return from_edges(off, np.concatenate(us), np.concatenate(vs), "union")


# ----------------------------------------------------------------------------
# workloads used by the tests and the benchmark (sizes follow the configs)

def batched_uneven_family(count: int = 512, n_min: int = 1000, n_max: int = 200000,
                          seed: int = 1000):
    """Uneven batch: n_i = round(exp(U(ln n_min, ln n_max))), type i mod 3 in
    {ER avg degree 8, BA m=3, WS k=6 beta=0.1}, graph seed = seed + i."""
    out = []
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.rint(np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=count))).astype(np.int64)
    for i, n in enumerate(sizes):
        n = int(n)
        kind = i % 3
        if kind == 0:
            g = erdos_renyi(n, 8.0 / (n - 1), seed + i)
        elif kind == 1:
            g = barabasi_albert(n, 3, seed + i)
        else:
            g = watts_strogatz(n, 6, 0.1, seed + i)
        out.append(g)
    return out
