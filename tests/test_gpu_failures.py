"""Failure detection without a GPU fault (every failure is made on the host
or by a bounded device wait that runs out):
  - a grid-barrier wait limit of 1 us makes the traversal kernel give up:
    the call returns BC_E_TIMEOUT, and with the default limit restored the
    same handle answers as the oracle does;
  - bc_cancel from another thread stops a long batch between two tiles
    (BC_E_CANCELLED), or, on a weighted graph, between two sources of a
    block, and the handle answers correctly afterwards;
  - an injected allocation failure (the k-th cudaMalloc) returns BC_E_OOM
    from graph creation or from the first query, and the next call, with the
    injection off, matches the oracle.
"""
import threading
import time

import numpy as np
import pytest

import graphgen as gg
import oracle as O
from helpers import close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bcd():
    import paper_1708_08739_gb300 as m
    m.lib()
    yield m
    m.bc_debug_fail_alloc(0)


@pytest.fixture(scope="module")
def er():
    g = gg.erdos_renyi(2000, 16000, 1)
    return g, O.Graph.from_csr(g)


def test_barrier_timeout_then_recovery(bcd, er):
    g, og = er
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols)
    bcd.bc_set_config(dg, accumulation=1)
    qs = gg.random_vertices(g.n, 8, 102).tolist()
    want = {r: O.bc_exact(og, r, 0)[0] for r in qs}
    default = bcd.bc_get_config(dg)["timeout_us"]
    assert default == 10_000_000
    bcd.bc_set_config(dg, timeout_us=1)
    with pytest.raises(bcd.BCError) as e:
        bcd.bc_batch(dg, [{"r": r} for r in qs])
    assert e.value.status == bcd.BC_E_TIMEOUT
    bcd.bc_set_config(dg, timeout_us=default)
    out, _ = bcd.bc_batch(dg, [{"r": r} for r in qs])
    for r, o in zip(qs, out):
        assert o["status"] == 0 and close(o["bc"], want[r]), (r, o, want[r])
    # a single query and a sampled one on the same handle
    assert close(bcd.bc_exact(dg, qs[0])[0], want[qs[0]])
    w, _, _, _ = O.bc_approx(og, qs[1], 300, 7, 0)
    assert close(bcd.bc_approx_T(dg, qs[1], 300, 7)[0], w)


@pytest.mark.parametrize("kernel", [1, 2])
def test_weighted_barrier_timeout_then_recovery(bcd, kernel):
    """Tile kernel: a grid-barrier wait runs out; source kernel: a block's
    source runs past the limit (checked after each distance level)."""
    g = gg.erdos_renyi(600, 4000, 21)
    g = g.with_weights(gg.uniform_weights(g.m, 1, 255, 3))
    og = O.Graph.from_csr(g)
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols, g.weights)
    qs = gg.random_vertices(g.n, 4, 104).tolist()
    bcd.bc_set_config(dg, timeout_us=1, weighted_kernel=kernel)
    with pytest.raises(bcd.BCError) as e:
        bcd.bc_batch(dg, [{"r": r} for r in qs])
    assert e.value.status == bcd.BC_E_TIMEOUT
    bcd.bc_set_config(dg, timeout_us=10_000_000)
    out, _ = bcd.bc_batch(dg, [{"r": r} for r in qs])
    for r, o in zip(qs, out):
        assert close(o["bc"], O.bc_exact(og, r, 0)[0]), r


def test_cancel_between_tiles(bcd):
    """A batch of exact queries in the giant component of R-MAT 18 (about
    a second of tiles) is cancelled 0.3 s after it starts."""
    g = gg.rmat(18, 16, 0.57, 0.19, 0.19, seed=18)
    og = O.Graph.from_csr(g)
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols)
    top = [int(x) for x in gg.top_inout_vertices(g, 8)]
    box = {}

    def run():
        t = time.time()
        try:
            box["out"] = bcd.bc_batch(dg, [{"r": r} for r in top])
        except bcd.BCError as ex:
            box["err"] = ex
        box["s"] = time.time() - t

    th = threading.Thread(target=run)
    th.start()
    time.sleep(0.3)
    bcd.bc_cancel(dg)
    th.join(timeout=120)
    assert not th.is_alive()
    assert "err" in box, "the batch finished before the cancel request (%.2f s)" % box.get("s", -1)
    assert box["err"].status == bcd.BC_E_CANCELLED
    # a cancel request made while no call runs is dropped by the next call
    bcd.bc_cancel(dg)
    r = top[0]
    want, draws, k, _ = O.bc_approx(og, r, 64, 7, 0)
    got, info = bcd.bc_approx_T(dg, r, 64, 7)
    assert info["rv_size"] == k and close(got, want), (got, want)


def test_weighted_cancel_between_sources(bcd):
    """The weighted source kernel checks the cancel request each time a
    block takes a source: exact queries on the top vertices of weighted
    R-MAT 18 (seconds of sources), cancelled 0.3 s in; the handle then
    answers a sampled query as the oracle does."""
    g = gg.rmat(18, 16, 0.57, 0.19, 0.19, seed=18)
    g = g.with_weights(gg.uniform_weights(g.m, 1, 255, 3))
    og = O.Graph.from_csr(g)
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols, g.weights)
    assert bcd.bc_get_config(dg)["weighted_kernel"] == 2
    top = [int(x) for x in gg.top_inout_vertices(g, 8)]
    box = {}

    def run():
        t = time.time()
        try:
            box["out"] = bcd.bc_batch(dg, [{"r": r} for r in top])
        except bcd.BCError as ex:
            box["err"] = ex
        box["s"] = time.time() - t

    th = threading.Thread(target=run)
    th.start()
    time.sleep(0.3)
    bcd.bc_cancel(dg)
    th.join(timeout=300)
    assert not th.is_alive()
    assert "err" in box, "the batch finished before the cancel request (%.2f s)" % box.get("s", -1)
    assert box["err"].status == bcd.BC_E_CANCELLED
    r = top[0]
    want, draws, k, _ = O.bc_approx(og, r, 64, 7, 0)
    got, info = bcd.bc_approx_T(dg, r, 64, 7)
    assert info["rv_size"] == k and close(got, want), (got, want)


@pytest.mark.parametrize("k", [1, 2, 5, 12, 25, 33])
def test_allocation_failure_leaves_graph_usable(bcd, er, k):
    g, og = er
    r = 11
    want = O.bc_exact(og, r, 0)[0]
    # graph creation (the first few allocations)
    bcd.bc_debug_fail_alloc(k)
    try:
        dg = bcd.bc_graph_create(g.n, g.offsets, g.cols)
    except bcd.BCError as ex:
        assert ex.status == bcd.BC_E_OOM
        bcd.bc_debug_fail_alloc(0)
        dg = bcd.bc_graph_create(g.n, g.offsets, g.cols)
    bcd.bc_debug_fail_alloc(0)
    # the first query builds the workspace (dozens of allocations)
    bcd.bc_debug_fail_alloc(k)
    failed = False
    try:
        bcd.bc_exact(dg, r)
    except bcd.BCError as ex:
        assert ex.status == bcd.BC_E_OOM
        failed = True
    bcd.bc_debug_fail_alloc(0)
    assert failed, "the workspace build made fewer than %d allocations" % k
    got, _ = bcd.bc_exact(dg, r)
    assert close(got, want), (k, got, want)
    out, _ = bcd.bc_batch(dg, [{"r": q} for q in (3, 5, r)])
    for q, o in zip((3, 5, r), out):
        assert close(o["bc"], O.bc_exact(og, q, 0)[0]), q
