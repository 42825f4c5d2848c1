"""Greedy distance-d colouring (Algorithm 1, Section 3.1).

Nodes are visited in order of descending degree, ties broken by ascending
node id (the paper recommends the degree ordering; the tie-break is this
build's reading).  Each node receives the smallest colour (0-based here) not
used by an already coloured node within geodesic distance d, found by a
breadth-first search of depth d.
"""
from collections import deque

import numpy as np


def greedy_order(graph):
    deg = np.diff(graph.rowptr)
    return np.lexsort((np.arange(graph.n), -deg))


def ball(graph, src, d):
    """Nodes at geodesic distance 1..d from src (BFS)."""
    seen = {src: 0}
    q = deque([src])
    out = []
    while q:
        u = q.popleft()
        du = seen[u]
        if du == d:
            continue
        for k in range(graph.rowptr[u], graph.rowptr[u + 1]):
            w = int(graph.col[k])
            if w not in seen:
                seen[w] = du + 1
                out.append(w)
                q.append(w)
    return out


def greedy_distance_coloring(graph, d):
    col = np.full(graph.n, -1, dtype=np.int64)
    for i in greedy_order(graph):
        used = {int(col[w]) for w in ball(graph, int(i), d) if col[w] >= 0}
        c = 0
        while c in used:
            c += 1
        col[i] = c
    return col


def is_distance_coloring(graph, colors, d):
    """Brute-force check: col(i) != col(j) whenever 1 <= dist(i, j) <= d."""
    for i in range(graph.n):
        for w in ball(graph, i, d):
            if colors[w] == colors[i]:
                return False
    return True
