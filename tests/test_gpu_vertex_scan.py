"""The vertex-scan accumulation (bc_config.accumulation = 2) against the CPU
oracle: delta_s.(r) = sigma_sr * sum of sigma_rt / sigma_st over the t with
d(s, r) + d(r, t) = d(s, t), one pass over a tile's reached (vertex, source)
pairs after a traversal from r, instead of the backward pass of Eq. 4.

The oracle computes BC(r) with Eq. 4 (Brandes' stack order); the scan sums
the same pair dependencies (Eq. 2) in another grouping, so the bar is a
relative 1e-9, and equality where every term is an integer. Sizes span
several tiles with ragged tails; the edge cases are the ones of the Eq. 4
path (trivial zero, empty RV, long level chains, split rows, sigma past
2^53). Unweighted graphs scan the per-level (vertex, source mask) entries,
weighted graphs the settled (vertex, source) pairs. Calls whose queries sit
at more than one vertex keep the Eq. 4 path.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle as O
from helpers import csr, close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bcd():
    import paper_1708_08739_gb300 as m
    m.lib()
    return m


def make(bcd, g, **cfg):
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols, g.weights)
    bcd.bc_set_config(dg, accumulation=2, **cfg)
    return dg


def scan_one(bcd, dg, q):
    """One query through bc_batch, so that the batch report shows the path."""
    out, info = bcd.bc_batch(dg, [q])
    assert out[0]["status"] == 0
    return out[0], info


@pytest.fixture(scope="module")
def er1():
    g = gg.erdos_renyi(2000, 16000, 1)
    return g, O.Graph.from_csr(g)


@pytest.fixture(scope="module")
def sparse_er():
    g = gg.erdos_renyi(3000, 3600, 2)
    return g, O.Graph.from_csr(g)


def test_config_roundtrip(bcd, er1):
    g, _ = er1
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols)
    assert bcd.bc_get_config(dg)["accumulation"] == 4
    bcd.bc_set_config(dg, accumulation=1)
    assert bcd.bc_get_config(dg)["accumulation"] == 1
    bcd.bc_set_config(dg, accumulation=2)
    assert bcd.bc_get_config(dg)["accumulation"] == 2
    bcd.bc_set_config(dg, accumulation=3)
    assert bcd.bc_get_config(dg)["accumulation"] == 3
    bcd.bc_set_config(dg, accumulation=4)
    assert bcd.bc_get_config(dg)["accumulation"] == 4
    bcd.bc_set_config(dg, accumulation=2)
    with pytest.raises(bcd.BCError) as e:
        bcd.bc_set_config(dg, accumulation=5)
    assert e.value.status == bcd.BC_E_INVALID_ARG
    # a tile's sources are seeded one per thread
    bcd.bc_set_config(dg, tile_words=2, block_threads=128)
    with pytest.raises(bcd.BCError) as e:
        bcd.bc_set_config(dg, tile_words=4)
    assert e.value.status == bcd.BC_E_INVALID_ARG
    with pytest.raises(bcd.BCError) as e:
        bcd.bc_set_config(dg, tile_words=4, block_threads=192)
    assert e.value.status == bcd.BC_E_INVALID_ARG
    assert bcd.bc_get_config(dg)["tile_words"] == 2
    assert bcd.bc_get_config(dg)["weighted_kernel"] == 2
    bcd.bc_set_config(dg, weighted_kernel=1)
    assert bcd.bc_get_config(dg)["weighted_kernel"] == 1
    with pytest.raises(bcd.BCError) as e:
        bcd.bc_set_config(dg, weighted_kernel=3)
    assert e.value.status == bcd.BC_E_INVALID_ARG


@pytest.mark.parametrize("cfg", [{"tile_words": 1}, {"tile_words": 2}, {"tile_words": 4, "blocks_per_sm": 1},
                                 {"tile_words": 4, "blocks_per_sm": 2}, {"chunk_arcs": 32},
                                 {"block_threads": 256, "chunk_arcs": 64}])
def test_scan_exact_matches_oracle(bcd, er1, cfg):
    """16 queries of the 2,000-vertex ER graph: |RV| near 2,000, so up to
    32 tiles of 64 sources with a ragged last tile."""
    g, og = er1
    dg = make(bcd, g, **cfg)
    for r in gg.random_vertices(g.n, 16, 102).tolist():
        o, info = scan_one(bcd, dg, {"r": r})
        want, k, f = O.bc_exact(og, r, 0)
        assert o["rv_size"] == k and o["flags"] == f
        assert close(o["bc"], want), (r, o["bc"], want)
        if k > 0 and g.out_degree()[r] > 0:
            assert info["ms_root"] > 0.0, info
        if want > 0.0:
            assert info["scan_pairs"] > 0, info


def test_scan_sparse_graph(bcd, sparse_er):
    """Sparse ER: many small RV sets and deep BFS levels."""
    g, og = sparse_er
    dg = make(bcd, g)
    for r in gg.random_vertices(g.n, 40, 5).tolist():
        got, info = bcd.bc_exact(dg, r)
        want, k, _ = O.bc_exact(og, r, 0)
        assert info["rv_size"] == k and close(got, want), (r, got, want)


def test_scan_all_sources_brandes(bcd):
    """Every vertex of a 400-vertex ER graph, one call each, against
    all-sources Brandes."""
    g = gg.erdos_renyi(400, 2400, 77)
    og = O.Graph.from_csr(g)
    allbc = O.bc_all(og)
    dg = make(bcd, g, tile_words=1)
    for r in range(g.n):
        got, _ = bcd.bc_exact(dg, r)
        assert close(got, allbc[r]), (r, got, allbc[r])


def test_scan_sampled_matches_oracle(bcd, er1):
    g, og = er1
    dg = make(bcd, g)
    for r, T, seed in [(5, 1000, 7), (1234, 333, 99), (77, 14979, 7)]:
        want, _, k, _ = O.bc_approx(og, r, T, seed, 0)
        o, info = scan_one(bcd, dg, {"r": r, "kind": bcd.BC_QUERY_APPROX_T, "T": T, "seed": seed})
        assert o["samples"] == T and o["rv_size"] == k
        assert close(o["bc"], want), (r, o["bc"], want)
        assert info["scan_pairs"] > 0 or want == 0.0


def test_scan_same_vertex_group(bcd, er1):
    """Exact, sampled and hybrid queries of one vertex in one group share the
    traversal from r and one scan per tile."""
    g, og = er1
    dg = make(bcd, g)
    r = 1234
    specs = [{"r": r}, {"r": r, "kind": bcd.BC_QUERY_APPROX_T, "T": 500, "seed": 3},
             {"r": r, "kind": bcd.BC_QUERY_APPROX_T, "T": 900, "seed": 4},
             {"r": r, "kind": bcd.BC_QUERY_HYBRID, "T": 100, "seed": 5},
             {"r": r, "kind": bcd.BC_QUERY_HYBRID, "T": 100000, "seed": 5}]
    out, info = bcd.bc_batch(dg, specs)
    assert info["scan_pairs"] > 0
    exact = O.bc_exact(og, r, 0)[0]
    wants = [exact, O.bc_approx(og, r, 500, 3, 0)[0], O.bc_approx(og, r, 900, 4, 0)[0],
             O.bc_approx(og, r, 100, 5, 0)[0], exact]
    for s, o, w in zip(specs, out, wants):
        assert o["status"] == 0 and close(o["bc"], w), (s, o["bc"], w)


def test_scan_mixed_vertices_keep_eq4(bcd, er1):
    """Two query vertices in one group: the call runs the Eq. 4 backward."""
    g, og = er1
    dg = make(bcd, g)
    out, info = bcd.bc_batch(dg, [{"r": 5}, {"r": 9}])
    assert info["scan_pairs"] == 0 and info["ms_root"] == 0.0
    for r, o in zip((5, 9), out):
        assert close(o["bc"], O.bc_exact(og, r, 0)[0])


@pytest.fixture(scope="module")
def wer():
    """ER 600 / 4,000 with weights uniform in [1, 255] (seed 3) and in [1, 3]
    (seed 4: many equal-length paths, sigma > 1)."""
    g = gg.erdos_renyi(600, 4000, 21)
    g255 = g.with_weights(gg.uniform_weights(g.m, 1, 255, 3))
    g3 = g.with_weights(gg.uniform_weights(g.m, 1, 3, 4))
    return [(x, O.Graph.from_csr(x)) for x in (g255, g3)]


@pytest.mark.parametrize("cfg", [{}, {"weighted_words": 1}, {"weighted_words": 16, "chunk_arcs": 32}])
@pytest.mark.parametrize("which", [0, 1])
def test_scan_weighted_matches_oracle(bcd, wer, which, cfg):
    """Weighted graphs: the scan over settled (vertex, source) pairs, exact
    and sampled, in 64-, 256- and 1024-source tiles."""
    g, og = wer[which]
    dg = make(bcd, g, **cfg)
    for r in gg.random_vertices(g.n, 10, 104).tolist():
        o, info = scan_one(bcd, dg, {"r": r})
        want, k, _ = O.bc_exact(og, r, 0)
        assert o["rv_size"] == k and close(o["bc"], want), (r, o["bc"], want)
        if want > 0.0:
            assert info["scan_pairs"] > 0 and info["ms_root"] > 0.0, info
    for r, T, seed in [(4, 600, 7), (77, 300, 9)]:
        want = O.bc_approx(og, r, T, seed, 0)[0]
        o, _ = scan_one(bcd, dg, {"r": r, "kind": bcd.BC_QUERY_APPROX_T, "T": T, "seed": seed})
        assert close(o["bc"], want), (r, o["bc"], want)


def test_scan_weighted_closed_forms(bcd):
    # a->b (2), a->c (1), c->b (1): two shortest a-b paths, one through c
    dg = make(bcd, csr(3, [(0, 1), (0, 2), (2, 1)], [2, 1, 1]))
    assert bcd.bc_exact(dg, 2)[0] == 0.5
    # weighted path: only the hop structure matters
    dg = make(bcd, csr(5, [(i, i + 1) for i in range(4)], [7, 1, 255, 3]))
    assert [bcd.bc_exact(dg, r)[0] for r in range(5)] == [0.0, 3.0, 4.0, 3.0, 0.0]


def test_scan_weighted_repeated_multitile(bcd, wer):
    """Ten 64-source tiles per launch (weights 1..3), repeated with several
    block sizes."""
    g, og = wer[1]
    qs = gg.random_vertices(g.n, 4, 104).tolist()
    want = {r: O.bc_exact(og, r, 0)[0] for r in qs}
    for it in range(4):
        dg = make(bcd, g, weighted_words=1, block_threads=(512, 256, 128, 384)[it])
        for r in qs:
            got = bcd.bc_exact(dg, r)[0]
            assert close(got, want[r]), (it, r, got, want[r])
        dg.close()


def test_scan_weighted_rmat_small(bcd):
    """Weighted R-MAT scale 12 (weights 1..255): hub rows split into chunks;
    scan and Eq. 4 against the oracle."""
    g = gg.rmat(12, 8, seed=12)
    g = g.with_weights(gg.uniform_weights(g.m, 1, 255, 3))
    og = O.Graph.from_csr(g)
    scan = make(bcd, g)
    push = bcd.bc_graph_create(g.n, g.offsets, g.cols, g.weights)
    bcd.bc_set_config(push, accumulation=1)
    for r in gg.top_inout_vertices(g, 2).tolist() + gg.random_vertices(g.n, 4, 104).tolist():
        want = O.bc_exact(og, r, 0)[0]
        a = bcd.bc_exact(scan, r)[0]
        b = bcd.bc_exact(push, r)[0]
        assert close(a, want) and close(b, want), (r, a, b, want)


def test_scan_weighted_mixed_vertices_keep_eq4(bcd, wer):
    g, og = wer[0]
    dg = make(bcd, g)
    out, info = bcd.bc_batch(dg, [{"r": 5}, {"r": 9}])
    assert info["scan_pairs"] == 0 and info["ms_root"] == 0.0
    for r, o in zip((5, 9), out):
        assert close(o["bc"], O.bc_exact(og, r, 0)[0])


def test_scan_closed_forms(bcd):
    # directed path: BC(v_i) = (i - 1)(n - i) for 1-based i; every term is 1
    n = 3000  # 2,999 levels in one tile
    dg = make(bcd, csr(n, [(i, i + 1) for i in range(n - 1)]))
    for r in [1, 1500, n - 2]:
        assert bcd.bc_exact(dg, r)[0] == r * (n - 1 - r)
    # directed cycle C_n: (n - 1)(n - 2) / 2 for every vertex
    n = 300
    dg = make(bcd, csr(n, [(i, (i + 1) % n) for i in range(n)]))
    for r in [0, 7, 299]:
        assert bcd.bc_exact(dg, r)[0] == (n - 1) * (n - 2) / 2
    # bidirected star: centre (n - 1)(n - 2), leaves 0
    n = 200
    arcs = [(0, i) for i in range(1, n)] + [(i, 0) for i in range(1, n)]
    dg = make(bcd, csr(n, arcs))
    assert bcd.bc_exact(dg, 0)[0] == (n - 1) * (n - 2)
    assert bcd.bc_exact(dg, 5)[0] == 0.0
    # diamond s->a, s->b, a->t, b->t: BC(a) = BC(b) = 1/2
    dg = make(bcd, csr(4, [(0, 1), (0, 2), (1, 3), (2, 3)]))
    assert bcd.bc_exact(dg, 1)[0] == 0.5 and bcd.bc_exact(dg, 2)[0] == 0.5


def test_scan_trivial_and_empty(bcd):
    g = csr(5, [(0, 1), (1, 2), (3, 2), (2, 4)])
    dg = make(bcd, g)
    bc, info = bcd.bc_exact(dg, 4)  # out-degree 0
    assert bc == 0.0 and info["flags"] & bcd.BC_FLAG_TRIVIAL_ZERO
    bc, info = bcd.bc_exact(dg, 0)  # RV empty
    assert bc == 0.0 and info["rv_size"] == 0
    bc, info = bcd.bc_exact(dg, 2)
    assert bc == 3.0 and info["rv_size"] == 3


def test_scan_heavy_rows(bcd):
    """A hub with 20,000 out- and in-arcs: rows split into many chunks."""
    n = 20001
    arcs = [(0, i) for i in range(1, n)] + [(i, 0) for i in range(1, n)] + [(i, i + 1) for i in range(1, n - 1)]
    g = csr(n, arcs)
    og = O.Graph.from_csr(g)
    for cfg in [{}, {"chunk_arcs": 32}]:
        dg = make(bcd, g, **cfg)
        for r in [0, 5, 19999]:
            got = bcd.bc_exact(dg, r)[0]
            want = O.bc_exact(og, r, 0)[0]
            assert close(got, want), (cfg, r, got, want)


@pytest.mark.parametrize("k", [52, 53, 54])
def test_scan_sigma_flag(bcd, k):
    """Chain of k diamonds: sigma reaches 2^k; the flag matches the oracle's."""
    arcs = []
    for i in range(k):
        a, b, c, d = 3 * i, 3 * i + 1, 3 * i + 2, 3 * i + 3
        arcs += [(a, b), (a, c), (b, d), (c, d)]
    arcs.append((3 * k, 3 * k + 1))
    g = csr(3 * k + 2, arcs)
    og = O.Graph.from_csr(g)
    dg = make(bcd, g)
    for r in (3 * k, 3 * (k // 2)):
        bc, info = bcd.bc_exact(dg, r)
        want, _, wf = O.bc_exact(og, r, 0)
        assert bool(info["flags"] & bcd.BC_FLAG_SIGMA_2_53) == bool(wf & O.FLAG_SIGMA_GT_2_53)
        if k <= 52:
            assert close(bc, want), (r, bc, want)


def test_scan_rmat_small_multitile(bcd):
    """R-MAT scale 13: hub rows, many tiles, the top in*out vertices (largest
    RV) and uniform ones; both accumulations agree with the oracle."""
    g = gg.rmat(13, 8, seed=13)
    og = O.Graph.from_csr(g)
    qs = gg.top_inout_vertices(g, 3).tolist() + gg.random_vertices(g.n, 5, 103).tolist()
    scan = make(bcd, g)
    push = bcd.bc_graph_create(g.n, g.offsets, g.cols)
    for r in qs:
        want = O.bc_exact(og, r, 0)[0]
        a = bcd.bc_exact(scan, r)[0]
        b = bcd.bc_exact(push, r)[0]
        assert close(a, want) and close(b, want), (r, a, b, want)


def test_scan_repeated_launches(bcd, er1):
    """The same queries over many launches with different block sizes."""
    g, og = er1
    qs = gg.random_vertices(g.n, 4, 17).tolist()
    want = {r: O.bc_exact(og, r, 0)[0] for r in qs}
    for it in range(6):
        dg = make(bcd, g, block_threads=(512, 128, 256)[it % 3], tile_words=(1, 2, 4)[it % 3])
        for r in qs:
            got = bcd.bc_exact(dg, r)[0]
            assert close(got, want[r]), (it, r, got, want[r])
        dg.close()


# ------------------------------------------------ several query vertices (accumulation = 3)

@pytest.mark.parametrize("cfg", [{}, {"tile_words": 1}, {"tile_words": 2, "chunk_arcs": 32},
                                 {"tile_words": 4, "blocks_per_sm": 1}, {"tile_words": 8}])
def test_multi_vertex_scan_exact(bcd, er1, cfg):
    """A batch of exact queries at 20 distinct vertices (three passes of 8
    columns) with repeated vertices, against the oracle's E-BCD."""
    g, og = er1
    dg = make(bcd, g, **cfg)
    bcd.bc_set_config(dg, accumulation=3)
    rs = gg.random_vertices(g.n, 20, 61).tolist()
    rs = rs + rs[:3]
    out, info = bcd.bc_batch(dg, [{"r": r} for r in rs])
    assert info["scan_pairs"] > 0
    for r, o in zip(rs, out):
        assert o["status"] == 0
        assert close(o["bc"], O.bc_exact(og, r, 0)[0]), (cfg, r, o["bc"])


def test_multi_vertex_scan_mixed_kinds(bcd, er1):
    """64 queries at up to 64 distinct vertices in one group: exact, sampled
    (shared and own seeds), hybrid; several kinds at one vertex."""
    g, og = er1
    dg = make(bcd, g)
    bcd.bc_set_config(dg, accumulation=3)
    rs = gg.random_vertices(g.n, 56, 62).tolist()
    specs = []
    for i, r in enumerate(rs):
        k = i % 4
        if k == 0:
            specs.append({"r": r, "kind": bcd.BC_QUERY_EXACT})
        elif k == 1:
            specs.append({"r": r, "kind": bcd.BC_QUERY_APPROX_T, "T": 600, "seed": 7})
        elif k == 2:
            specs.append({"r": r, "kind": bcd.BC_QUERY_APPROX_T, "T": 300, "seed": 1000 + i})
        else:
            specs.append({"r": r, "kind": bcd.BC_QUERY_HYBRID, "T": 1000, "seed": 3})
    for r in rs[:8]:
        specs.append({"r": r, "kind": bcd.BC_QUERY_APPROX_T, "T": 200, "seed": 9})
    assert len(specs) == 64
    out, info = bcd.bc_batch(dg, specs)
    for s, o in zip(specs, out):
        r = s["r"]
        rvk = O.rv(og, r).shape[0]
        if s["kind"] == bcd.BC_QUERY_EXACT or (s["kind"] == bcd.BC_QUERY_HYBRID and rvk <= s["T"]):
            want = O.bc_exact(og, r, 0)[0]
        else:
            want = O.bc_approx(og, r, s["T"], s["seed"], 0)[0]
        assert o["status"] == 0 and close(o["bc"], want), (s, o["bc"], want)


def test_multi_vertex_scan_edge_cases(bcd, sparse_er):
    """Sparse ER (many small reach sets, long levels): queries with empty
    RV and out-degree 0 beside ordinary ones; 2^k path counts on a diamond
    chain with the sink and a middle vertex as two query vertices."""
    g, og = sparse_er
    dg = make(bcd, g)
    bcd.bc_set_config(dg, accumulation=3)
    rs = gg.random_vertices(g.n, 40, 63).tolist()
    out, _ = bcd.bc_batch(dg, [{"r": r} for r in rs])
    for r, o in zip(rs, out):
        assert close(o["bc"], O.bc_exact(og, r, 0)[0]), r
    k = 40
    arcs = []
    for i in range(k):
        a, b, c, d = 3 * i, 3 * i + 1, 3 * i + 2, 3 * i + 3
        arcs += [(a, b), (a, c), (b, d), (c, d)]
    arcs.append((3 * k, 3 * k + 1))
    gd = csr(3 * k + 2, arcs)
    ogd = O.Graph.from_csr(gd)
    dgd = make(bcd, gd)
    bcd.bc_set_config(dgd, accumulation=3)
    qs = [3 * k, 3 * (k // 2), 3 * (k // 2) + 1, 0]
    out, _ = bcd.bc_batch(dgd, [{"r": r} for r in qs])
    for r, o in zip(qs, out):
        assert close(o["bc"], O.bc_exact(ogd, r, 0)[0]), r


@pytest.mark.parametrize("cfg", [{}, {"weighted_words": 1}, {"weighted_words": 2, "chunk_arcs": 32}])
@pytest.mark.parametrize("wmax", [255, 3])
def test_multi_vertex_scan_weighted(bcd, cfg, wmax):
    """Weighted graphs (weights 1..255, and 1..3 with many equal-length
    paths): a group at 10 distinct vertices (repeats and a sampled query
    among them) takes the vertex scan over settled (vertex, source) pairs
    with accumulation 3 and matches the oracle."""
    g = gg.erdos_renyi(600, 4000, 21)
    g = g.with_weights(gg.uniform_weights(g.m, 1, wmax, 4))
    og = O.Graph.from_csr(g)
    dg = make(bcd, g, **cfg)
    bcd.bc_set_config(dg, accumulation=3)
    rs = gg.random_vertices(g.n, 10, 64).tolist()
    specs = [{"r": r} for r in rs] + [{"r": rs[0]}, {"r": rs[1], "kind": bcd.BC_QUERY_APPROX_T, "T": 200, "seed": 7}]
    out, info = bcd.bc_batch(dg, specs)
    assert info["scan_pairs"] > 0
    for sp, o in zip(specs, out):
        if sp.get("kind", 0) == 0:
            want = O.bc_exact(og, sp["r"], 0)[0]
        else:
            want = O.bc_approx(og, sp["r"], 200, 7, 0)[0]
        assert o["status"] == 0 and close(o["bc"], want), (cfg, sp, o["bc"], want)


def test_auto_choice_per_group(bcd, er1):
    """accumulation = 4 (the default): on ER (no hubs) a group of 12 vertices
    keeps the scan after its first tile; with a hub among the query
    vertices (20,000 in- and out-arcs: nearly every shortest path runs
    through it) the first tile's terms outnumber the push's and the other
    tiles take Eq. 4. Results match the oracle either way."""
    g, og = er1
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols)
    bcd.bc_set_config(dg, tile_words=1)
    rs = gg.random_vertices(g.n, 12, 65).tolist()
    out, info = bcd.bc_batch(dg, [{"r": r} for r in rs])
    assert info["tiles"] > 1 and info["scan_tiles"] == info["tiles"], info
    for r, o in zip(rs, out):
        assert close(o["bc"], O.bc_exact(og, r, 0)[0]), r
    n = 20001
    arcs = [(0, i) for i in range(1, n)] + [(i, 0) for i in range(1, n)]
    arcs += [(i, i + 1) for i in range(1, n - 1)]
    gh = csr(n, arcs)
    ogh = O.Graph.from_csr(gh)
    dgh = bcd.bc_graph_create(gh.n, gh.offsets, gh.cols)
    qs = [0, 17, 5000]
    out, info = bcd.bc_batch(dgh, [{"r": r} for r in qs])
    assert info["tiles"] > 1 and info["scan_tiles"] == 1, info
    for r, o in zip(qs, out):
        assert close(o["bc"], O.bc_exact(ogh, r, 0)[0]), r
