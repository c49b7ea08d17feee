"""Python binding of libbcd (include/bcd.h): single-vertex betweenness
centrality in directed graphs on a GB300 GPU.

Argument marshalling only: every step runs in the CUDA library. The names
follow the C ABI (bc_graph_create, bc_rv_compute, bc_exact, bc_approx,
bc_approx_T, bc_batch, ...). Host arrays are numpy arrays; device arrays may
be passed as CUDA torch tensors to bc_graph_create (mem_kind DEVICE).

If libbcd.so has not been built the import fails; there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbcd.so")

BC_OK = 0
BC_E_INVALID_ARG = 1
BC_E_INVALID_GRAPH = 2
BC_E_OOM = 3
BC_E_CUDA = 4
BC_E_BUFFER_TOO_SMALL = 5
BC_E_TIMEOUT = 6
BC_E_INTERNAL = 7
BC_E_BUSY = 8
BC_E_PENDING = 9
BC_E_CANCELLED = 10

BC_MEM_HOST = 0
BC_MEM_DEVICE = 1

BC_FLAG_SIGMA_2_53 = 0x1
BC_FLAG_TRIVIAL_ZERO = 0x2

BC_QUERY_EXACT = 0
BC_QUERY_APPROX = 1
BC_QUERY_APPROX_T = 2
BC_QUERY_HYBRID = 3


class bc_graph_desc(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int64), ("row_offsets", C.c_void_p), ("cols", C.c_void_p),
                ("weights", C.c_void_p), ("mem_kind", C.c_int32), ("stream", C.c_void_p)]


class bc_info(C.Structure):
    _fields_ = [("rv_size", C.c_int64), ("samples", C.c_int64), ("sources_run", C.c_int64),
                ("edges_traversed", C.c_int64), ("max_level", C.c_int32), ("flags", C.c_uint32),
                ("ms_rv", C.c_double), ("ms_sample", C.c_double), ("ms_spd", C.c_double),
                ("ms_total", C.c_double)]


class bc_query(C.Structure):
    _fields_ = [("r", C.c_int32), ("kind", C.c_int32), ("eps", C.c_double), ("delta", C.c_double),
                ("T", C.c_int64), ("seed", C.c_uint64)]


class bc_result(C.Structure):
    _fields_ = [("bc", C.c_double), ("status", C.c_int32), ("flags", C.c_uint32), ("rv_size", C.c_int64),
                ("samples", C.c_int64)]


class bc_batch_info(C.Structure):
    _fields_ = [("queries", C.c_int64), ("sources_run", C.c_int64), ("edges_traversed", C.c_int64),
                ("launches", C.c_int64), ("ms_rv", C.c_double), ("ms_sample", C.c_double),
                ("ms_spd", C.c_double), ("ms_total", C.c_double), ("ms_forward", C.c_double),
                ("ms_backward", C.c_double), ("tiles", C.c_int64), ("max_level", C.c_int32),
                ("grid_blocks", C.c_int32), ("ms_traversal", C.c_double), ("reached_pairs", C.c_int64),
                ("tight_pairs", C.c_int64), ("arc_visits", C.c_int64), ("union_vertices", C.c_int64),
                ("union_arcs", C.c_int64), ("scan_pairs", C.c_int64), ("ms_root", C.c_double),
                ("pull_levels", C.c_int64), ("scan_tiles", C.c_int64), ("eq4_reached_pairs", C.c_int64),
                ("eq4_tight_pairs", C.c_int64)]


class bc_config(C.Structure):
    _fields_ = [("tile_words", C.c_int32), ("chunk_arcs", C.c_int32), ("block_threads", C.c_int32),
                ("source_order", C.c_int32), ("blocks_per_sm", C.c_int32), ("weighted_words", C.c_int32),
                ("accumulation", C.c_int32), ("timeout_us", C.c_int32), ("pull_permille", C.c_int32),
                ("weighted_short_row", C.c_int32), ("weighted_kernel", C.c_int32)]


class bc_tune_report(C.Structure):
    _fields_ = [("candidates", C.c_int64), ("probe_queries", C.c_int64), ("ms_default", C.c_double),
                ("ms_best", C.c_double)]


class bc_server_config(C.Structure):
    _fields_ = [("max_active", C.c_int32), ("tiles_per_slice", C.c_int32), ("max_device_bytes", C.c_int64),
                ("max_queue", C.c_int64)]


class bc_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("slices", C.c_int64), ("sources_run", C.c_int64), ("edges_traversed", C.c_int64),
                ("active", C.c_int64), ("queued", C.c_int64), ("busy_ms", C.c_double)]


# every symbol declared in include/bcd.h, with its ctypes signature
_SIGNATURES = {
    "bc_graph_create": (C.c_int, [C.POINTER(bc_graph_desc), C.POINTER(C.c_void_p)]),
    "bc_graph_destroy": (None, [C.c_void_p]),
    "bc_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "bc_graph_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "bc_graph_reverse": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "bc_rv_compute": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "bc_exact": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_double), C.POINTER(bc_info)]),
    "bc_approx": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_double, C.c_uint64, C.POINTER(C.c_double),
                            C.POINTER(bc_info)]),
    "bc_approx_T": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.POINTER(C.c_double),
                              C.POINTER(bc_info)]),
    "bc_samples_for": (C.c_int, [C.c_double, C.c_double, C.POINTER(C.c_int64)]),
    "bc_draw_samples": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_void_p,
                                  C.POINTER(C.c_int64)]),
    "bc_batch": (C.c_int, [C.c_void_p, C.POINTER(bc_query), C.c_int64, C.POINTER(bc_result),
                           C.POINTER(bc_batch_info)]),
    "bc_batch_shard": (C.c_int, [C.c_void_p, C.POINTER(bc_query), C.c_int64, C.c_int32, C.c_int32,
                                 C.POINTER(bc_result), C.POINTER(bc_batch_info)]),
    "bc_spd_probe": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p,
                               C.c_void_p, C.c_void_p, C.c_void_p]),
    "bc_set_config": (C.c_int, [C.c_void_p, C.POINTER(bc_config)]),
    "bc_get_config": (C.c_int, [C.c_void_p, C.POINTER(bc_config)]),
    "bc_rv_compute_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int64,
                                        C.POINTER(C.c_int64), C.c_void_p]),
    "bc_server_create": (C.c_int, [C.c_void_p, C.POINTER(bc_server_config), C.POINTER(C.c_void_p)]),
    "bc_submit": (C.c_int, [C.c_void_p, C.POINTER(bc_query), C.POINTER(C.c_uint64)]),
    "bc_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(bc_result), C.POINTER(C.c_double), C.c_int64]),
    "bc_server_stats_get": (C.c_int, [C.c_void_p, C.POINTER(bc_server_stats)]),
    "bc_server_destroy": (None, [C.c_void_p]),
    "bc_tune": (C.c_int, [C.c_void_p, C.POINTER(bc_query), C.c_int64, C.c_int64, C.POINTER(bc_config),
                          C.POINTER(bc_tune_report)]),
    "bc_cancel": (C.c_int, [C.c_void_p]),
    "bc_debug_fail_alloc": (C.c_int, [C.c_int64]),
    "bc_last_error": (C.c_char_p, []),
    "bc_version": (C.c_char_p, []),
}

_lib = None


def lib():
    """The loaded libbcd.so. Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libbcd.so is not built (run __graft_entry__.build() or "
                              "python paper_1708_08739_gb300/build.py)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class BCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("bcd status %d: %s" % (status, msg))
        self.status = status


def _check(st):
    if st != BC_OK:
        raise BCError(st, lib().bc_last_error().decode())


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _default_stream():
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


class Graph:
    """Owning handle of a device-resident graph (bc_graph)."""

    def __init__(self, handle, n, m, weighted):
        self.handle = handle
        self.n = n
        self.m = m
        self.weighted = weighted

    def __del__(self):
        self.close()

    def close(self):
        h = getattr(self, "handle", None)
        if h:
            lib().bc_graph_destroy(h)
            self.handle = None


def bc_graph_create(n, offsets, cols, weights=None, stream=None) -> Graph:
    """Creates the device graph from CSR arrays: numpy (host) or CUDA torch
    tensors (device). Rows must be strictly increasing."""
    keep = []

    def as_arg(a, dtype):
        if a is None:
            return None, None
        if hasattr(a, "is_cuda") and a.is_cuda:
            return C.c_void_p(a.data_ptr()), BC_MEM_DEVICE
        arr = np.ascontiguousarray(a, dtype=dtype)
        keep.append(arr)
        return C.c_void_p(arr.ctypes.data), BC_MEM_HOST

    po, ko = as_arg(offsets, np.int64)
    pc, kc = as_arg(cols, np.int32)
    pw, kw = as_arg(weights, np.uint32)
    kinds = {k for k in (ko, kc, kw) if k is not None}
    if len(kinds) != 1:
        raise ValueError("offsets, cols and weights must all be host arrays or all be device tensors")
    m = int(cols.shape[0])
    d = bc_graph_desc(int(n), m, po, pc, pw, kinds.pop(),
                      C.c_void_p(stream if stream is not None else _default_stream() or 0))
    h = C.c_void_p()
    _check(lib().bc_graph_create(C.byref(d), C.byref(h)))
    return Graph(h, int(n), m, weights is not None)


def bc_graph_destroy(g: Graph):
    g.close()


def bc_set_stream(g: Graph, stream):
    _check(lib().bc_set_stream(g.handle, C.c_void_p(stream or 0)))


def bc_set_config(g: Graph, tile_words=0, chunk_arcs=0, block_threads=0, source_order=0, blocks_per_sm=0,
                  weighted_words=0, accumulation=0, timeout_us=0, pull_permille=0, weighted_short_row=0,
                  weighted_kernel=0):
    c = bc_config(int(tile_words), int(chunk_arcs), int(block_threads), int(source_order), int(blocks_per_sm),
                  int(weighted_words), int(accumulation), int(timeout_us), int(pull_permille),
                  int(weighted_short_row), int(weighted_kernel))
    _check(lib().bc_set_config(g.handle, C.byref(c)))


def bc_get_config(g: Graph) -> dict:
    c = bc_config()
    _check(lib().bc_get_config(g.handle, C.byref(c)))
    return {k: getattr(c, k) for k, _ in bc_config._fields_}


def bc_tune(g: Graph, specs, probe_T=256):
    """Times candidate launch parameters on a probe of the batch `specs`
    (every query as A-BCD with at most probe_T draws), applies the fastest to
    g and returns (config dict, report dict)."""
    q, nq = make_queries(specs)
    c = bc_config()
    rep = bc_tune_report()
    _check(lib().bc_tune(g.handle, q, nq, int(probe_T), C.byref(c), C.byref(rep)))
    return {k: getattr(c, k) for k, _ in bc_config._fields_}, {k: getattr(rep, k) for k, _ in bc_tune_report._fields_}


def bc_cancel(g: Graph):
    """Asks the call running on g (in another thread) to stop at its next
    tile; that call then raises BCError with BC_E_CANCELLED."""
    _check(lib().bc_cancel(g.handle))


def bc_debug_fail_alloc(k: int):
    """Makes the k-th device allocation of the library from now on fail
    (BC_E_OOM); 0 switches the injection off."""
    _check(lib().bc_debug_fail_alloc(int(k)))


def bc_graph_info(g: Graph):
    n, m, w = C.c_int32(), C.c_int64(), C.c_int32()
    _check(lib().bc_graph_info(g.handle, C.byref(n), C.byref(m), C.byref(w)))
    return n.value, m.value, bool(w.value)


def bc_graph_reverse(g: Graph):
    roff = np.zeros(g.n + 1, dtype=np.int64)
    rcol = np.zeros(max(g.m, 1), dtype=np.int32)
    rw = np.zeros(max(g.m, 1), dtype=np.uint32) if g.weighted else None
    _check(lib().bc_graph_reverse(g.handle, _ptr(roff), _ptr(rcol), _ptr(rw)))
    return roff, rcol[: g.m], (None if rw is None else rw[: g.m])


def bc_rv_compute(g: Graph, r: int) -> np.ndarray:
    """RV(r): ascending ids of the vertices with a path to r (r excluded)."""
    cnt = C.c_int64()
    st = lib().bc_rv_compute(g.handle, int(r), None, 0, C.byref(cnt))
    if st not in (BC_OK, BC_E_BUFFER_TOO_SMALL):
        _check(st)
    out = np.zeros(max(cnt.value, 1), dtype=np.int32)
    _check(lib().bc_rv_compute(g.handle, int(r), _ptr(out), out.shape[0], C.byref(cnt)))
    return out[: cnt.value]


def _info_dict(info: bc_info) -> dict:
    return {k: getattr(info, k) for k, _ in bc_info._fields_}


def bc_exact(g: Graph, r: int):
    """E-BCD: (BC(r), info dict)."""
    bc = C.c_double()
    info = bc_info()
    _check(lib().bc_exact(g.handle, int(r), C.byref(bc), C.byref(info)))
    return bc.value, _info_dict(info)


def bc_approx(g: Graph, r: int, eps: float, delta: float, seed: int):
    """A-BCD with T from (eps, delta): (bc, info dict)."""
    bc = C.c_double()
    info = bc_info()
    _check(lib().bc_approx(g.handle, int(r), float(eps), float(delta), int(seed) & (2**64 - 1), C.byref(bc),
                           C.byref(info)))
    return bc.value, _info_dict(info)


def bc_approx_T(g: Graph, r: int, T: int, seed: int):
    """A-BCD with T samples: (bc, info dict)."""
    bc = C.c_double()
    info = bc_info()
    _check(lib().bc_approx_T(g.handle, int(r), int(T), int(seed) & (2**64 - 1), C.byref(bc), C.byref(info)))
    return bc.value, _info_dict(info)


def bc_samples_for(eps: float, delta: float) -> int:
    t = C.c_int64()
    _check(lib().bc_samples_for(float(eps), float(delta), C.byref(t)))
    return t.value


def bc_draw_samples(g: Graph, r: int, T: int, seed: int):
    """The T draws of A-BCD in draw order and |RV(r)|."""
    out = np.full(int(T), -1, dtype=np.int32)
    k = C.c_int64()
    _check(lib().bc_draw_samples(g.handle, int(r), int(T), int(seed) & (2**64 - 1), _ptr(out), C.byref(k)))
    return (out if k.value > 0 else out[:0]), k.value


def make_queries(specs) -> "C.Array":
    """specs: iterable of dicts with r, kind and eps/delta/T/seed as needed."""
    specs = list(specs)
    arr = (bc_query * max(len(specs), 1))()
    for i, s in enumerate(specs):
        arr[i] = bc_query(int(s["r"]), int(s.get("kind", BC_QUERY_EXACT)), float(s.get("eps", 0.0)),
                          float(s.get("delta", 0.0)), int(s.get("T", 0)), int(s.get("seed", 0)) & (2**64 - 1))
    return arr, len(specs)


def bc_batch(g: Graph, specs):
    """Many queries at once: (list of result dicts, batch info dict)."""
    q, nq = make_queries(specs)
    res = (bc_result * max(nq, 1))()
    info = bc_batch_info()
    _check(lib().bc_batch(g.handle, q, nq, res, C.byref(info)))
    out = [{"bc": res[i].bc, "status": res[i].status, "flags": res[i].flags, "rv_size": res[i].rv_size,
            "samples": res[i].samples} for i in range(nq)]
    return out, {k: getattr(info, k) for k, _ in bc_batch_info._fields_}


def bc_batch_shard(g: Graph, specs, shard: int, nshards: int):
    """Shard `shard` of `nshards` of bc_batch: (list of result dicts whose
    "bc" is this shard's part of each score, batch info dict)."""
    q, nq = make_queries(specs)
    res = (bc_result * max(nq, 1))()
    info = bc_batch_info()
    _check(lib().bc_batch_shard(g.handle, q, nq, int(shard), int(nshards), res, C.byref(info)))
    out = [{"bc": res[i].bc, "status": res[i].status, "flags": res[i].flags, "rv_size": res[i].rv_size,
            "samples": res[i].samples} for i in range(nq)]
    return out, {k: getattr(info, k) for k, _ in bc_batch_info._fields_}


def bc_spd_probe(g: Graph, sources, targets, want_dist=True, want_sigma=True, want_dep=True):
    """Per-source dist [nsrc, n] (uint64, 2**64-1 unreached), sigma [nsrc, n],
    dep [nsrc, nt] = delta_s.(t) and flags [nsrc] from one tile of the
    batched kernel."""
    src = np.ascontiguousarray(sources, dtype=np.int32)
    tg = np.ascontiguousarray(targets, dtype=np.int32)
    ns, nt = src.shape[0], tg.shape[0]
    dist = np.zeros((ns, g.n), dtype=np.uint64) if want_dist else None
    sig = np.zeros((ns, g.n), dtype=np.float64) if want_sigma else None
    dep = np.zeros((ns, max(nt, 1)), dtype=np.float64) if want_dep else None
    flags = np.zeros(ns, dtype=np.uint32)
    _check(lib().bc_spd_probe(g.handle, _ptr(src), ns, _ptr(tg), nt, _ptr(dist), _ptr(sig), _ptr(dep),
                              _ptr(flags)))
    return dist, sig, (None if dep is None else dep[:, :nt]), flags


class Server:
    """Owning handle of a serving loop (bc_server) on a graph."""

    def __init__(self, g: Graph, max_active=0, tiles_per_slice=0, max_device_bytes=0, max_queue=0):
        cfg = bc_server_config(int(max_active), int(tiles_per_slice), int(max_device_bytes), int(max_queue))
        h = C.c_void_p()
        _check(lib().bc_server_create(g.handle, C.byref(cfg), C.byref(h)))
        self.handle = h
        self.graph = g

    def submit(self, spec) -> int:
        q, _ = make_queries([spec])
        t = C.c_uint64()
        _check(lib().bc_submit(self.handle, q, C.byref(t)))
        return t.value

    def poll(self, ticket, timeout_us=0):
        """(result dict, latency ms) or None while pending."""
        r = bc_result()
        lat = C.c_double()
        st = lib().bc_poll(self.handle, C.c_uint64(ticket), C.byref(r), C.byref(lat), int(timeout_us))
        if st == BC_E_PENDING:
            return None
        _check(st)
        return ({"bc": r.bc, "status": r.status, "flags": r.flags, "rv_size": r.rv_size, "samples": r.samples},
                lat.value)

    def stats(self) -> dict:
        s = bc_server_stats()
        _check(lib().bc_server_stats_get(self.handle, C.byref(s)))
        return {k: getattr(s, k) for k, _ in bc_server_stats._fields_}

    def close(self):
        h = getattr(self, "handle", None)
        if h:
            lib().bc_server_destroy(h)
            self.handle = None

    def __del__(self):
        self.close()


BC_NOALLOC_MAX_VERTICES = 4194304


def bc_rv_compute_noalloc(d_roffsets, d_rcols, n, r, d_out, cap, stream=None):
    """RV(r) with no allocation by the library: all arguments are device
    pointers (ints) the caller owns; returns |RV(r)| (raises BCError with
    BC_E_BUFFER_TOO_SMALL, count unknown to the caller, if cap is short)."""
    cnt = C.c_int64()
    st = lib().bc_rv_compute_noalloc(C.c_void_p(d_roffsets), C.c_void_p(d_rcols), int(n), int(r),
                                     C.c_void_p(d_out), int(cap), C.byref(cnt), C.c_void_p(stream or 0))
    if st == BC_E_BUFFER_TOO_SMALL:
        raise BCError(st, "%s (|RV(r)| = %d)" % (lib().bc_last_error().decode(), cnt.value))
    _check(st)
    return cnt.value


def bc_version() -> str:
    return lib().bc_version().decode()


def bc_last_error() -> str:
    return lib().bc_last_error().decode()
