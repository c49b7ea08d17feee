"""Small graph builders and independent reference computations for tests.

Nothing here calls the oracle or the CUDA library; these are the textbook
constructions the oracle is pinned against.
"""
from __future__ import annotations

from collections import deque
from fractions import Fraction

import numpy as np

import graphgen as gg


def csr(n, arcs, weights=None):
    """CSR from an arc list (sorted, duplicates rejected)."""
    arcs = list(arcs)
    order = sorted(range(len(arcs)), key=lambda i: arcs[i])
    a = [arcs[i] for i in order]
    assert len(set(a)) == len(a), "duplicate arc"
    assert all(u != v for u, v in a), "self-loop"
    off = np.zeros(n + 1, dtype=np.int64)
    for u, _ in a:
        off[u + 1] += 1
    off = np.cumsum(off)
    cols = np.array([v for _, v in a], dtype=np.int32)
    w = None
    if weights is not None:
        w = np.array([weights[i] for i in order], dtype=np.uint32)
    return gg.CSR(n, off, cols, w)


def arcs_of(g):
    t, h = g.arcs()
    return list(zip(t.tolist(), h.tolist()))


def brute_force_bc(g):
    """BC(v) for all v by enumerating every simple path (Eq. 1), exact
    fractions, ordered pairs s != t, pairs with no path contribute 0."""
    n = g.n
    adj = [[] for _ in range(n)]
    t, h = g.arcs()
    w = g.weights if g.weights is not None else np.ones(g.m, dtype=np.uint32)
    for i in range(g.m):
        adj[int(t[i])].append((int(h[i]), int(w[i])))
    bc = [Fraction(0)] * n
    for s in range(n):
        best = {}  # t -> (length, [paths])
        stack = [(s, 0, (s,))]
        while stack:
            x, L, path = stack.pop()
            if x != s:
                cur = best.get(x)
                if cur is None or L < cur[0]:
                    best[x] = (L, [path])
                elif L == cur[0]:
                    cur[1].append(path)
            for y, wt in adj[x]:
                if y not in path:
                    stack.append((y, L + wt, path + (y,)))
        for tt, (_, paths) in best.items():
            sig = len(paths)
            through = [0] * n
            for p in paths:
                for v in p[1:-1]:
                    through[v] += 1
            for v in range(n):
                if through[v]:
                    bc[v] += Fraction(through[v], sig)
    return bc


def bfs_dist_sigma(g, s):
    """Unweighted BFS from s: hop distances (-1 unreached) and exact sigma."""
    n = g.n
    dist = [-1] * n
    sig = [0] * n
    dist[s] = 0
    sig[s] = 1
    q = deque([s])
    while q:
        x = q.popleft()
        for e in range(g.offsets[x], g.offsets[x + 1]):
            y = int(g.cols[e])
            if dist[y] < 0:
                dist[y] = dist[x] + 1
                q.append(y)
            if dist[y] == dist[x] + 1:
                sig[y] += sig[x]
    return dist, sig


def dijkstra_dist_sigma(g, s):
    """Weighted shortest paths from s: distances (-1 unreached) by Dijkstra
    with a binary heap, then exact sigma by visiting vertices in increasing
    distance (weights are positive, so a tight arc climbs in distance)."""
    import heapq
    n = g.n
    w = g.weights
    dist = [-1] * n
    best = {s: 0}
    pq = [(0, s)]
    while pq:
        d, x = heapq.heappop(pq)
        if dist[x] >= 0:
            continue
        dist[x] = d
        for e in range(g.offsets[x], g.offsets[x + 1]):
            y = int(g.cols[e])
            nd = d + int(w[e])
            if dist[y] < 0 and nd < best.get(y, nd + 1):
                best[y] = nd
                heapq.heappush(pq, (nd, y))
    sig = [0] * n
    sig[s] = 1
    for x in sorted((v for v in range(n) if dist[v] >= 0), key=lambda v: dist[v]):
        for e in range(g.offsets[x], g.offsets[x + 1]):
            y = int(g.cols[e])
            if dist[y] == dist[x] + int(w[e]):
                sig[y] += sig[x]
    return dist, sig


def random_digraph(n, p, seed, weighted=False, wmax=4):
    r = np.random.default_rng(seed)
    arcs = [(u, v) for u in range(n) for v in range(n) if u != v and r.random() < p]
    weights = [int(x) for x in r.integers(1, wmax + 1, size=len(arcs))] if weighted else None
    return csr(n, arcs, weights)


REL = 1e-9


def close(a, b, rel=REL):
    """The parity bar for fp64 scores and dependencies: |a - b| <= rel * |b|,
    a purely relative bound (every delta and BC is a sum of non-negative
    terms, so its rounding error is relative too); a reference value of
    exactly 0 (no source reaches past r) must be matched exactly."""
    a = float(a)
    b = float(b)
    if b == 0.0:
        return a == 0.0
    return abs(a - b) <= rel * abs(b)
