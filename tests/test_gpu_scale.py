"""Parity at full size, in the launch configuration bench.py times (tiles of
256 sources at two blocks per SM, 128-arc chunks, default tile order).

R-MAT scale 20 (the exact batch): RV lists of all 64 queries bit-exact;
dist and sigma of sampled union sources bit-exact and their dependencies on
every query within 1e-9; full BC(r) for the queries the oracle can finish;
the vertex-scan accumulation on single queries.
A whole 256-source tile probed element by element.
R-MAT scale 22 with 30 % reciprocal arcs (the sampled batch): the draws of
eps = 0.01, delta = 0.1, seed 7 bit-exact, the dependencies of drawn
sources within 1e-9, and four of its sampled queries end to end (T = 128)
against the oracle's A-BCD on the same draws.
The R-MAT scale 20 graph with weights uniform in [1, 255] (seed 3; the
weighted batch of 32 uniform queries, seed 104), in the default weighted tile
width: RV lists bit-exact, uint64 distances and sigma of sampled sources
bit-exact and their dependencies on all 32 queries within 1e-9, the
queries with empty RV answered 0, and the vertex scan on a sampled query.
"""
import concurrent.futures as cf
import os

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
    return m


@pytest.fixture(scope="module")
def rmat20(bcd):
    g = gg.rmat(20, 16, 0.57, 0.19, 0.19, seed=20)
    qs = [int(x) for x in gg.random_vertices(g.n, 32, 103)] + [int(x) for x in gg.top_inout_vertices(g, 32)]
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols)
    bcd.bc_set_config(dg, tile_words=4, chunk_arcs=128, blocks_per_sm=2, accumulation=1)
    return g, O.Graph.from_csr(g), dg, qs


def test_rmat20_rv_lists(bcd, rmat20):
    g, og, dg, qs = rmat20
    seen = {}
    for r in qs:
        if r in seen:
            continue
        got = bcd.bc_rv_compute(dg, r)
        seen[r] = got
        assert np.array_equal(got, O.rv(og, r)), r


def test_rmat20_sampled_sources(bcd, rmat20):
    g, og, dg, qs = rmat20
    top = qs[32]
    union = O.rv(og, top)
    rng = np.random.default_rng(5)
    srcs = np.sort(rng.choice(union, size=12, replace=False)).astype(np.int32)
    qv = np.array(list(dict.fromkeys(qs)), dtype=np.int32)[:64]
    dist, sig, dep, flags = bcd.bc_spd_probe(dg, srcs, qv)
    odep, ofl, _ = O.dependencies(og, srcs, qv, 0)
    for i, s in enumerate(srcs.tolist()):
        st = O.source_state(og, s)
        assert np.array_equal(dist[i], st["dist"]), s
        if not st["flags"]:
            assert np.array_equal(sig[i], st["sigma"]), s
        for j in range(qv.shape[0]):
            if qv[j] != s:
                assert close(dep[i, j], odep[i, j]), (s, int(qv[j]), dep[i, j], odep[i, j])


def test_rmat20_small_queries_full(bcd, rmat20):
    g, og, dg, qs = rmat20
    small = []
    for r in dict.fromkeys(qs):
        k = bcd.bc_rv_compute(dg, r).shape[0]
        if 0 < k <= 200:
            small.append(r)
    out, _ = bcd.bc_batch(dg, [{"r": r} for r in small])
    for r, o in zip(small, out):
        want, k, _ = O.bc_exact(og, r, 0)
        assert o["rv_size"] == k and close(o["bc"], want), (r, o["bc"], want)


def test_rmat20_vertex_scan(bcd, rmat20):
    """accumulation = 2 at full size, one query per call: 96 and 512 draws on
    the top in*out vertex (seed 7) against the oracle on the same draws, both
    accumulations; the small exact queries against the oracle."""
    g, og, dg, qs = rmat20
    top = qs[32]
    threads = os.cpu_count() or 1
    want96, _, k, _ = O.bc_approx(og, top, 96, 7, threads)
    want512, _, k512, _ = O.bc_approx(og, top, 512, 7, threads)
    assert k512 == k
    bcd.bc_set_config(dg, accumulation=2)
    try:
        out, info = bcd.bc_batch(dg, [{"r": top, "kind": bcd.BC_QUERY_APPROX_T, "T": 96, "seed": 7}])
        assert info["scan_pairs"] > 0 and out[0]["rv_size"] == k
        assert close(out[0]["bc"], want96), (out[0]["bc"], want96)
        scan, info = bcd.bc_batch(dg, [{"r": top, "kind": bcd.BC_QUERY_APPROX_T, "T": 512, "seed": 7}])
        assert info["scan_pairs"] > 0
        assert close(scan[0]["bc"], want512), (scan[0]["bc"], want512)
        small = []
        for r in dict.fromkeys(qs):
            kk = bcd.bc_rv_compute(dg, r).shape[0]
            if 0 < kk <= 200:
                small.append(r)
        for r in small:
            got, _ = bcd.bc_exact(dg, r)
            assert close(got, O.bc_exact(og, r, 0)[0]), r
    finally:
        bcd.bc_set_config(dg, accumulation=1)
    push, info = bcd.bc_batch(dg, [{"r": top, "kind": bcd.BC_QUERY_APPROX_T, "T": 512, "seed": 7}])
    assert info["scan_pairs"] == 0
    assert close(push[0]["bc"], want512), (push[0]["bc"], want512)


def test_rmat20_full_tile_probe(bcd, rmat20):
    """One whole 256-source tile of the bench's kernel (slots 0..255), element
    by element: every source's distances and sigma bit-exact, and its
    dependencies on the 64 query vertices within the relative bar."""
    g, og, dg, qs = rmat20
    S = 64 * bcd.bc_get_config(dg)["tile_words"]
    assert S == 256
    union = O.rv(og, qs[32])
    rng = np.random.default_rng(9)
    srcs = np.sort(rng.choice(union, size=S, replace=False)).astype(np.int32)
    qv = np.array(list(dict.fromkeys(qs)), dtype=np.int32)[:64]
    dist, sig, dep, flags = bcd.bc_spd_probe(dg, srcs, qv)
    threads = os.cpu_count() or 1
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        # the oracle's C code releases the GIL: sources run in parallel
        states = ex.map(lambda s: (s, O.source_state(og, int(s))), srcs.tolist())
        for i, (s, st) in enumerate(states):
            assert np.array_equal(dist[i], st["dist"]), (i, s)
            assert (flags[i] != 0) == (st["flags"] != 0), (i, s)
            if not st["flags"]:
                assert np.array_equal(sig[i], st["sigma"]), (i, s)
            for j, t in enumerate(qv.tolist()):
                if t != s:
                    assert close(dep[i, j], st["delta"][t]), (i, s, t, dep[i, j], st["delta"][t])


def test_rmat20_multi_vertex_scan(bcd, rmat20):
    """accumulation = 3 at full size: 8 of the bench's queries (4 uniform,
    4 of largest in*out degree) in one group, A-BCD with 32 draws each
    (seed 7), against the oracle's A-BCD on the same draws."""
    g, og, dg, qs = rmat20
    pick = [q for q in qs[:32] if g.out_degree()[q] > 0][:4] + qs[32:36]
    specs = [{"r": r, "kind": bcd.BC_QUERY_APPROX_T, "T": 32, "seed": 7} for r in pick]
    bcd.bc_set_config(dg, accumulation=3)
    try:
        out, info = bcd.bc_batch(dg, specs)
    finally:
        bcd.bc_set_config(dg, accumulation=1)
    assert info["scan_pairs"] > 0
    threads = os.cpu_count() or 1
    for r, o in zip(pick, out):
        want = O.bc_approx(og, r, 32, 7, threads)[0]
        assert o["status"] == 0 and close(o["bc"], want), (r, o["bc"], want)


@pytest.fixture(scope="module")
def rmat22(bcd):
    g = gg.add_reciprocal(gg.rmat(22, 8, seed=22), 0.3, seed=22)
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols)
    bcd.bc_set_config(dg, tile_words=4, chunk_arcs=128, blocks_per_sm=2, accumulation=1)
    return g, O.Graph.from_csr(g), dg


def test_rmat22_sampled_draws_and_dependencies(bcd, rmat22):
    g, og, dg = rmat22
    T = O.samples_for(0.01, 0.1)
    assert T == 14979
    qs = [int(x) for x in gg.random_vertices(g.n, 64, 105)]
    checked = 0
    for r in qs:
        if g.out_degree()[r] == 0:
            continue
        draws, k = bcd.bc_draw_samples(dg, r, T, 7)
        rvl = O.rv(og, r)
        assert k == rvl.shape[0]
        if k == 0:
            continue
        want = np.array([rvl[O.sample_index(7, t, k)] for t in range(T)], dtype=np.int32)
        assert np.array_equal(draws, want), r
        if checked == 0 and k > 1000:
            srcs = np.array(sorted(set(want[:8].tolist())), dtype=np.int32)
            dist, sig, dep, flags = bcd.bc_spd_probe(dg, srcs, [r], want_sigma=False)
            odep, _, _ = O.dependencies(og, srcs, [r], 0)
            for i in range(srcs.shape[0]):
                st = O.source_state(og, int(srcs[i]))
                assert np.array_equal(dist[i], st["dist"])
                assert close(dep[i, 0], odep[i, 0]), (int(srcs[i]), dep[i, 0], odep[i, 0])
            checked += 1
    assert checked == 1


def test_rmat22_sampled_batch_end_to_end(bcd, rmat22):
    """The bench's sampled R-MAT 22 batch shape end to end: the first four of
    the 64 uniform queries (seed 105) whose RV holds more than 1000 sources,
    A-BCD with T = 128 draws (Philox seed 7) in one bc_batch, each bc(r)
    against the oracle's A-BCD on the same draws (128 draws keep the oracle's
    four runs of Brandes from 128 sources on 42.7 M arcs to about a minute)."""
    g, og, dg = rmat22
    qs = [int(x) for x in gg.random_vertices(g.n, 64, 105)]
    big = []
    for r in qs:
        if g.out_degree()[r] > 0 and r not in big and bcd.bc_rv_compute(dg, r).shape[0] > 1000:
            big.append(r)
        if len(big) == 4:
            break
    assert len(big) == 4
    T = 128
    specs = [{"r": r, "kind": bcd.BC_QUERY_APPROX_T, "T": T, "seed": 7} for r in big]
    out, info = bcd.bc_batch(dg, specs)
    threads = os.cpu_count() or 1
    for r, o in zip(big, out):
        want, draws, k, f = O.bc_approx(og, r, T, 7, threads)
        assert o["status"] == 0 and o["rv_size"] == k and o["samples"] == T
        assert close(o["bc"], want), (r, o["bc"], want)


@pytest.fixture(scope="module")
def rmat20w(bcd):
    g = gg.rmat(20, 16, 0.57, 0.19, 0.19, seed=20)
    g = g.with_weights(gg.uniform_weights(g.m, 1, 255, 3))
    qs = [int(x) for x in gg.random_vertices(g.n, 32, 104)]
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols, g.weights)
    bcd.bc_set_config(dg, accumulation=1)
    return g, O.Graph.from_csr(g), dg, qs


def test_rmat20_weighted_rv_lists(bcd, rmat20w):
    g, og, dg, qs = rmat20w
    for r in dict.fromkeys(qs):
        assert np.array_equal(bcd.bc_rv_compute(dg, r), O.rv(og, r)), r


def test_rmat20_weighted_sampled_sources(bcd, rmat20w):
    g, og, dg, qs = rmat20w
    assert bcd.bc_get_config(dg)["weighted_words"] == 4
    sizes = {r: bcd.bc_rv_compute(dg, r).shape[0] for r in dict.fromkeys(qs)}
    big = max(sizes, key=sizes.get)
    union = O.rv(og, big)
    rng = np.random.default_rng(6)
    srcs = np.sort(rng.choice(union, size=12, replace=False)).astype(np.int32)
    qv = np.array(list(dict.fromkeys(qs)), dtype=np.int32)
    dist, sig, dep, flags = bcd.bc_spd_probe(dg, srcs, qv)
    odep, ofl, _ = O.dependencies(og, srcs, qv, 0)
    for i, s in enumerate(srcs.tolist()):
        st = O.source_state(og, s)
        assert np.array_equal(dist[i], st["dist"]), s
        if not st["flags"]:
            assert np.array_equal(sig[i], st["sigma"]), s
        for j in range(qv.shape[0]):
            if qv[j] != s:
                assert close(dep[i, j], odep[i, j]), (s, int(qv[j]), dep[i, j], odep[i, j])


def test_rmat20_weighted_vertex_scan(bcd, rmat20w):
    """accumulation = 2 on the weighted graph at full size: 48 draws (seed 7)
    on the vertex of largest in*out degree, against the oracle on the same
    draws and against the Eq. 4 path."""
    g, og, dg, qs = rmat20w
    # the vertex of largest in*out degree: RV is the giant component and the
    # score is far from 0 (the giant-component queries of the batch have one
    # out-arc or none, and 48 draws give them 0)
    top = int(gg.top_inout_vertices(g, 1)[0])
    spec = {"r": top, "kind": bcd.BC_QUERY_APPROX_T, "T": 48, "seed": 7}
    want = O.bc_approx(og, top, 48, 7, 0)[0]
    assert want > 0.0
    push, info = bcd.bc_batch(dg, [spec])
    assert info["scan_pairs"] == 0
    bcd.bc_set_config(dg, accumulation=2)
    try:
        scan, info = bcd.bc_batch(dg, [spec])
    finally:
        bcd.bc_set_config(dg, accumulation=1)
    assert info["scan_pairs"] > 0
    assert close(scan[0]["bc"], want) and close(push[0]["bc"], want), (scan[0]["bc"], push[0]["bc"], want)


def test_rmat20_weighted_kernels_agree(bcd, rmat20w):
    """Both weighted kernels at full size, each under the Eq. 4 pull and the
    vertex scan: 96 draws (seed 5) on the vertex of largest in*out degree,
    all four against the oracle on the same draws."""
    g, og, dg, qs = rmat20w
    top = int(gg.top_inout_vertices(g, 1)[0])
    spec = {"r": top, "kind": bcd.BC_QUERY_APPROX_T, "T": 96, "seed": 5}
    want = O.bc_approx(og, top, 96, 5, os.cpu_count() or 1)[0]
    assert want > 0.0
    try:
        for kernel in (1, 2):
            for acc in (1, 2):
                bcd.bc_set_config(dg, weighted_kernel=kernel, accumulation=acc)
                out, info = bcd.bc_batch(dg, [spec])
                assert (info["scan_pairs"] > 0) == (acc == 2)
                assert out[0]["status"] == 0 and close(out[0]["bc"], want), (kernel, acc, out[0]["bc"], want)
    finally:
        bcd.bc_set_config(dg, weighted_kernel=2, accumulation=1)


def test_rmat20_weighted_multi_vertex_scan(bcd, rmat20w):
    """The weighted batch's query vertices in the giant component (seed 104)
    as one group under the default per-group choice (the vertex scan over
    several vertices on the first tile, then the cheaper backward), A-BCD
    with 32 draws each and its own seed, against the oracle's A-BCD on the
    same draws."""
    g, og, dg, qs = rmat20w
    big = [r for r in dict.fromkeys(qs) if g.out_degree()[r] > 0 and bcd.bc_rv_compute(dg, r).shape[0] > 1000][:6]
    assert len(big) >= 4
    specs = [{"r": r, "kind": bcd.BC_QUERY_APPROX_T, "T": 32, "seed": 11 + i} for i, r in enumerate(big)]
    bcd.bc_set_config(dg, accumulation=4)
    try:
        out, info = bcd.bc_batch(dg, specs)
    finally:
        bcd.bc_set_config(dg, accumulation=1)
    assert info["scan_tiles"] >= 1
    threads = os.cpu_count() or 1
    for s, o in zip(specs, out):
        want = O.bc_approx(og, s["r"], 32, s["seed"], threads)[0]
        assert o["status"] == 0 and close(o["bc"], want), (s, o["bc"], want)


def test_rmat20_weighted_empty_rv_queries(bcd, rmat20w):
    """The queries outside the giant component have no in-arcs here: RV is
    empty and BC(r) = 0 (Prop. 1); the oracle agrees on each."""
    g, og, dg, qs = rmat20w
    empty = [r for r in dict.fromkeys(qs) if bcd.bc_rv_compute(dg, r).shape[0] == 0]
    assert len(empty) >= 10
    out, _ = bcd.bc_batch(dg, [{"r": r} for r in empty])
    for r, o in zip(empty, out):
        want, k, _ = O.bc_exact(og, r, 0)
        assert o["status"] == 0 and o["rv_size"] == k == 0 and o["bc"] == want == 0.0, (r, o)
