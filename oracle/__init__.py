"""CPU oracle for single-vertex betweenness (test infrastructure only).

A ctypes front end to ``bc_oracle.c``: a plain, sequential-per-source CPU
statement of the method of Chehreghani, Bifet and Abdessalem (Sections 2 and
4). Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package. It shares no code with the CUDA library.

Functions and the passage each follows:
  reverse        Section 4.1, Def. 2 (reverse graph R(G))
  rv             Section 4.1 procedure (BFS on R(G) from r, r excluded), Prop. 2
  source_state   Section 2 (SPD, sigma) and Eq. 4 (dependencies) for one source
  dependencies   delta_s.(r_q) for many sources and query vertices (Eq. 4)
  bc_exact       Algorithm 1 (E-BCD), Prop. 1 and Eq. 5
  bc_approx      Algorithm 2 (A-BCD), draws by the Philox stream below
  bc_all         Brandes over all sources, Eq. 3 (for small graphs)
  samples_for    T from Eq. "samplesnumber" under the relative-epsilon reading
  philox4x64_10  Philox4x64-10 (Salmon et al., SC'11); sample_index maps a
                 draw to an RV index
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

_lib = None

I32P = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
I64P = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
U32P = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
U64P = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
F64P = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
VP = C.c_void_p

FLAG_SIGMA_GT_2_53 = 1


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_reverse.argtypes = [C.c_int32, I64P, I32P, VP, I64P, I32P, VP]
        L.orc_reverse.restype = C.c_int
        L.orc_rv.argtypes = [C.c_int32, I64P, I32P, C.c_int32, VP]
        L.orc_rv.restype = C.c_int64
        L.orc_source_state.argtypes = [C.c_int32, I64P, I32P, VP, I64P, I32P, VP, C.c_int32,
                                       VP, VP, VP, VP, VP, VP]
        L.orc_source_state.restype = C.c_int
        L.orc_dependencies.argtypes = [C.c_int32, I64P, I32P, VP, I64P, I32P, VP,
                                       I32P, C.c_int64, I32P, C.c_int32, F64P, U32P, VP, C.c_int]
        L.orc_dependencies.restype = C.c_int
        L.orc_bc_exact.argtypes = [C.c_int32, I64P, I32P, VP, I64P, I32P, VP, C.c_int32, C.c_int,
                                   C.POINTER(C.c_int64), C.POINTER(C.c_uint)]
        L.orc_bc_exact.restype = C.c_double
        L.orc_bc_approx.argtypes = [C.c_int32, I64P, I32P, VP, I64P, I32P, VP, C.c_int32,
                                    C.c_int64, C.c_uint64, C.c_int, VP,
                                    C.POINTER(C.c_int64), C.POINTER(C.c_uint)]
        L.orc_bc_approx.restype = C.c_double
        L.orc_bc_all.argtypes = [C.c_int32, I64P, I32P, VP, I64P, I32P, VP, F64P]
        L.orc_bc_all.restype = C.c_int
        L.orc_philox4x64_10.argtypes = [U64P, U64P, U64P]
        L.orc_philox4x64_10.restype = None
        L.orc_sample_index.argtypes = [C.c_uint64, C.c_int64, C.c_int64]
        L.orc_sample_index.restype = C.c_int64
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Graph:
    """Forward CSR plus the oracle's own R(G), built by ``reverse``."""

    def __init__(self, n, offsets, cols, weights=None):
        self.n = int(n)
        self.off = np.ascontiguousarray(offsets, dtype=np.int64)
        self.col = np.ascontiguousarray(cols, dtype=np.int32)
        self.w = None if weights is None else np.ascontiguousarray(weights, dtype=np.uint32)
        self.roff, self.rcol, self.rw = reverse(self.n, self.off, self.col, self.w)

    @classmethod
    def from_csr(cls, g):
        return cls(g.n, g.offsets, g.cols, g.weights)

    def _args(self):
        return (self.n, self.off, self.col, _ptr(self.w), self.roff, self.rcol, _ptr(self.rw))


def reverse(n, off, col, w=None):
    """R(G) as CSR (Def. 2); rows list tails in ascending order."""
    m = int(off[-1])
    roff = np.zeros(n + 1, dtype=np.int64)
    rcol = np.zeros(max(m, 1), dtype=np.int32)
    rw = None if w is None else np.zeros(max(m, 1), dtype=np.uint32)
    if lib().orc_reverse(n, off, col, _ptr(w), roff, rcol, _ptr(rw)) != 0:
        raise MemoryError("orc_reverse")
    return roff, rcol[:m], (None if rw is None else rw[:m])


def rv(g: Graph, r: int) -> np.ndarray:
    """RV(r) in ascending order (r excluded)."""
    out = np.zeros(g.n, dtype=np.int32)
    k = lib().orc_rv(g.n, g.roff, g.rcol, int(r), _ptr(out))
    if k < 0:
        raise MemoryError("orc_rv")
    return out[:k].copy()


def source_state(g: Graph, s: int) -> dict:
    """dist (uint64, 2**64-1 unreached), sigma (fp64), sigma_exact (python
    ints), delta (fp64), reached count and the sigma flag for source s."""
    n = g.n
    dist = np.zeros(n, dtype=np.uint64)
    sigma = np.zeros(n, dtype=np.float64)
    lo = np.zeros(n, dtype=np.uint64)
    hi = np.zeros(n, dtype=np.uint64)
    delta = np.zeros(n, dtype=np.float64)
    reached = C.c_int64(0)
    f = lib().orc_source_state(*g._args(), int(s), _ptr(dist), _ptr(sigma), _ptr(lo), _ptr(hi),
                               _ptr(delta), C.cast(C.pointer(reached), C.c_void_p))
    if f < 0:
        raise MemoryError("orc_source_state")
    return {"dist": dist, "sigma": sigma, "sigma_lo": lo, "sigma_hi": hi, "delta": delta,
            "reached": reached.value, "flags": f}


def sigma_exact(state: dict, v: int) -> int:
    return int(state["sigma_lo"][v]) | (int(state["sigma_hi"][v]) << 64)


def dependencies(g: Graph, sources, queries, nthreads: int = 0):
    """delta_s.(r_q) as an array [len(sources), len(queries)], the per-source
    sigma flags and the number of vertices each source reaches."""
    src = np.ascontiguousarray(sources, dtype=np.int32)
    qs = np.ascontiguousarray(queries, dtype=np.int32)
    dep = np.zeros((max(src.shape[0], 1), max(qs.shape[0], 1)), dtype=np.float64)
    flags = np.zeros(max(src.shape[0], 1), dtype=np.uint32)
    reached = np.zeros(max(src.shape[0], 1), dtype=np.int64)
    rc = lib().orc_dependencies(*g._args(), src, src.shape[0], qs, qs.shape[0],
                                dep.reshape(-1), flags, _ptr(reached), int(nthreads))
    if rc != 0:
        raise MemoryError("orc_dependencies")
    k = src.shape[0]
    return dep[:k, :qs.shape[0]], flags[:k], reached[:k]


def bc_exact(g: Graph, r: int, nthreads: int = 0):
    """E-BCD: (BC(r), |RV(r)|, flags)."""
    k = C.c_int64(0)
    f = C.c_uint(0)
    bc = lib().orc_bc_exact(*g._args(), int(r), int(nthreads), C.byref(k), C.byref(f))
    return bc, k.value, f.value


def bc_approx(g: Graph, r: int, T: int, seed: int, nthreads: int = 0):
    """A-BCD with T draws: (bc, draws v_t, |RV(r)|, flags)."""
    samples = np.full(max(int(T), 1), -1, dtype=np.int32)
    k = C.c_int64(0)
    f = C.c_uint(0)
    bc = lib().orc_bc_approx(*g._args(), int(r), int(T), int(seed) & (2**64 - 1), int(nthreads),
                             _ptr(samples), C.byref(k), C.byref(f))
    drawn = samples[: int(T)] if k.value > 0 and g.off[r + 1] > g.off[r] else samples[:0]
    return bc, drawn.copy(), k.value, f.value


def bc_all(g: Graph) -> np.ndarray:
    """BC(v) for every vertex by Brandes over all sources (Eq. 3)."""
    bc = np.zeros(g.n, dtype=np.float64)
    if lib().orc_bc_all(*g._args(), bc) < 0:
        raise MemoryError("orc_bc_all")
    return bc


def samples_for(eps: float, delta: float) -> int:
    """Eq. "samplesnumber" with epsilon taken relative to the range K*|RV(r)|
    of one estimate bc_t (Hoeffding with a = 0, b = K*|RV(r)|):
    T = ceil(ln(2/delta) / (2 eps^2))."""
    if not (eps > 0.0) or not (0.0 < delta < 1.0):
        raise ValueError("need eps > 0 and 0 < delta < 1")
    return int(math.ceil(math.log(2.0 / delta) / (2.0 * eps * eps)))


def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(c, k, out)
    return out


def sample_index(seed: int, t: int, k: int) -> int:
    return lib().orc_sample_index(int(seed) & (2**64 - 1), int(t), int(k))
