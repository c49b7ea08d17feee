"""Seeded synthetic inputs: directed graphs, arc weights and query vertices.

This module holds no arithmetic of the betweenness method itself. It only
draws graphs and query vertices, so that the CPU oracle and the CUDA library
can be fed identical inputs. Every generator is a pure function of its seed.

Graphs follow the paper's model (Section 2): directed, without self-loops and
without multi-arcs; weights, when present, are positive integers. Rows of the
returned CSR are strictly increasing (sorted, no duplicates), which is the
layout the library's graph-creation call requires.

All random draws use numpy's Philox bit generator keyed by the seed, so a
recipe is fully described by (generator, sizes, seed).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng",
    "CSR",
    "csr_from_arcs",
    "erdos_renyi",
    "rmat",
    "add_reciprocal",
    "uniform_weights",
    "random_vertices",
    "top_inout_vertices",
    "zipf_vertices",
]


def rng(seed: int) -> np.random.Generator:
    """numpy Generator on a Philox stream keyed by ``seed``."""
    return np.random.Generator(np.random.Philox(key=int(seed)))


class CSR:
    """Directed graph in CSR form: int64 row offsets, int32 column ids.

    ``weights`` is None (unweighted) or a uint32 array parallel to ``cols``.
    """

    def __init__(self, n, offsets, cols, weights=None):
        self.n = int(n)
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.cols = np.ascontiguousarray(cols, dtype=np.int32)
        self.weights = None if weights is None else np.ascontiguousarray(weights, dtype=np.uint32)
        assert self.offsets.shape == (self.n + 1,)
        assert self.offsets[-1] == self.cols.shape[0]

    @property
    def m(self) -> int:
        return int(self.cols.shape[0])

    def out_degree(self) -> np.ndarray:
        return np.diff(self.offsets)

    def in_degree(self) -> np.ndarray:
        return np.bincount(self.cols, minlength=self.n).astype(np.int64)

    def arcs(self):
        """(tails, heads) arrays in CSR order."""
        tails = np.repeat(np.arange(self.n, dtype=np.int32), self.out_degree())
        return tails, self.cols.copy()

    def with_weights(self, weights) -> "CSR":
        return CSR(self.n, self.offsets, self.cols, weights)


def _sorted_unique(keys: np.ndarray) -> np.ndarray:
    s = np.sort(keys)
    if s.shape[0] == 0:
        return s
    keep = np.empty(s.shape[0], dtype=bool)
    keep[0] = True
    np.not_equal(s[1:], s[:-1], out=keep[1:])
    return s[keep]


def csr_from_arcs(n: int, tails, heads) -> CSR:
    """Sorted, de-duplicated CSR of an arc list; self-loops are dropped."""
    tails = np.asarray(tails, dtype=np.int64)
    heads = np.asarray(heads, dtype=np.int64)
    keep = tails != heads
    key = _sorted_unique(tails[keep] * np.int64(n) + heads[keep])
    t = (key // n).astype(np.int64)
    h = (key % n).astype(np.int32)
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(t, minlength=n), out=offsets[1:])
    return CSR(n, offsets, h)


def erdos_renyi(n: int, m: int, seed: int) -> CSR:
    """Directed G(n, m): ordered pairs drawn uniformly, self-loops and repeats
    rejected, until exactly ``m`` distinct arcs (first occurrences kept)."""
    if m > n * (n - 1):
        raise ValueError("m exceeds the number of possible arcs")
    g = rng(seed)
    keys = np.empty(0, dtype=np.int64)
    while True:
        need = m - keys.shape[0]
        draw = g.integers(0, n, size=(2, max(2 * need, 1024)), dtype=np.int64)
        cand = draw[0] * n + draw[1]
        cand = cand[draw[0] != draw[1]]
        allk = np.concatenate([keys, cand])
        order = np.argsort(allk, kind="stable")
        srt = allk[order]
        first = np.ones(srt.shape[0], dtype=bool)
        first[1:] = srt[1:] != srt[:-1]
        keys = allk[np.sort(order[first])]
        if keys.shape[0] >= m:
            keys = keys[:m]
            break
    return csr_from_arcs(n, keys // n, keys % n)


def rmat(scale: int, edge_factor: int, a=0.57, b=0.19, c=0.19, seed: int = 0) -> CSR:
    """R-MAT (Chakrabarti et al. 2004): ``edge_factor * 2**scale`` arcs, each
    choosing, bit by bit from the top, the quadrant (0,0)/(0,1)/(1,0)/(1,1)
    with probabilities a/b/c/d (one uniform 32-bit draw per arc and bit,
    compared with the cumulative thresholds). No noise, no vertex
    permutation. Self-loops and duplicate arcs are removed afterwards."""
    n = 1 << scale
    m_draw = edge_factor * n
    g = rng(seed)
    tails = np.zeros(m_draw, dtype=np.int32)
    heads = np.zeros(m_draw, dtype=np.int32)
    # quadrant thresholds on a uniform 32-bit draw per (arc, bit)
    ta, tab, tabc = (np.uint32(min(round(x * 2.0**32), 2**32 - 1)) for x in (a, a + b, a + b + c))
    for level in range(scale):
        u = g.integers(0, 2**32, size=m_draw, dtype=np.uint32)
        shift = np.int32(scale - 1 - level)
        src_bit = u >= tab                                   # quadrants c, d
        dst_bit = ((u >= ta) & (u < tab)) | (u >= tabc)      # quadrants b, d
        tails |= src_bit.astype(np.int32) << shift
        heads |= dst_bit.astype(np.int32) << shift
        del u, src_bit, dst_bit
    return csr_from_arcs(n, tails, heads)


def add_reciprocal(gr: CSR, frac: float, seed: int) -> CSR:
    """Adds the reversed arc (v, u) for a Bernoulli(frac) subset of arcs (u, v),
    mimicking reciprocal links; duplicates are removed again."""
    t, h = gr.arcs()
    pick = rng(seed).random(gr.m) < frac
    tails = np.concatenate([t, h[pick]])
    heads = np.concatenate([h, t[pick]])
    return csr_from_arcs(gr.n, tails, heads)


def uniform_weights(m: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """uint32 weights uniform in [lo, hi], one per arc in CSR order."""
    return rng(seed).integers(lo, hi + 1, size=m, dtype=np.int64).astype(np.uint32)


def random_vertices(n: int, k: int, seed: int) -> np.ndarray:
    """``k`` vertex ids drawn uniformly (with replacement) over [0, n)."""
    return rng(seed).integers(0, n, size=k, dtype=np.int64).astype(np.int32)


def top_inout_vertices(gr: CSR, k: int) -> np.ndarray:
    """The ``k`` vertices with the largest in-degree x out-degree, ties by id."""
    prod = gr.in_degree() * gr.out_degree()
    order = np.lexsort((np.arange(gr.n), -prod))
    return order[:k].astype(np.int32)


def zipf_vertices(n: int, k: int, s: float, seed: int) -> np.ndarray:
    """``k`` ids whose popularity follows Zipf(s) over ranks 1..n; rank k maps
    to a vertex through a seeded permutation (popularity independent of id)."""
    g = rng(seed)
    perm = g.permutation(n)
    ranks = np.arange(1, n + 1, dtype=np.float64)
    cdf = np.cumsum(ranks ** (-s))
    cdf /= cdf[-1]
    idx = np.searchsorted(cdf, g.random(k), side="right")
    idx = np.minimum(idx, n - 1)
    return perm[idx].astype(np.int32)
