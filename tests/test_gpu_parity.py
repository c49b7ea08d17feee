"""CUDA library against the CPU oracle, element by element, on seeded inputs.

Bars: RV lists, distances, sigma and sampled source lists bit-exact; delta
and BC within a relative 1e-9 (fp64 sums in a different order). Sizes span
several tiles and ragged tails; edge cases cover empty and trivial inputs,
long level chains, heavy rows split into many chunks and sigma past 2^53.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle as O
from helpers import csr, close

pytestmark = pytest.mark.gpu

UNREACHED = np.iinfo(np.uint64).max


@pytest.fixture(scope="module")
def bcd():
    import paper_1708_08739_gb300 as m
    m.lib()
    return m


def make(bcd, g, **cfg):
    """A graph handle on the Eq. 4 backward (the vertex scan, the default for
    one-vertex calls, has its own tests)."""
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols, g.weights)
    bcd.bc_set_config(dg, **{"accumulation": 1, **cfg})
    return dg


@pytest.fixture(scope="module")
def er1():
    """Directed ER, 2,000 vertices, 16,000 arcs, seed 1."""
    g = gg.erdos_renyi(2000, 16000, 1)
    return g, O.Graph.from_csr(g)


@pytest.fixture(scope="module")
def sparse_er():
    """Sparser ER with many small reach sets and long BFS depth."""
    g = gg.erdos_renyi(3000, 3600, 2)
    return g, O.Graph.from_csr(g)


def test_reverse_graph(bcd, er1):
    g, og = er1
    dg = make(bcd, g)
    roff, rcol, _ = bcd.bc_graph_reverse(dg)
    assert np.array_equal(roff, og.roff)
    for v in range(g.n):  # row order is unspecified: compare sets
        assert np.array_equal(np.sort(rcol[roff[v]:roff[v + 1]]), og.rcol[og.roff[v]:og.roff[v + 1]])


@pytest.mark.parametrize("which", ["er1", "sparse_er"])
def test_rv_lists_bit_exact(bcd, which, request):
    g, og = request.getfixturevalue(which)
    dg = make(bcd, g)
    for r in list(gg.random_vertices(g.n, 24, 102)) + [0, g.n - 1]:
        assert np.array_equal(bcd.bc_rv_compute(dg, int(r)), O.rv(og, int(r))), r


@pytest.mark.parametrize("tile_words", [1, 2, 4, 8])
def test_probe_dist_sigma_delta(bcd, er1, tile_words):
    g, og = er1
    dg = make(bcd, g, tile_words=tile_words)
    srcs = np.array(sorted(set(gg.random_vertices(g.n, 40, 7).tolist())), dtype=np.int32)[:37]
    tgts = gg.random_vertices(g.n, 20, 8)
    tgts = np.array([t for t in dict.fromkeys(tgts.tolist())], dtype=np.int32)
    dist, sig, dep, flags = bcd.bc_spd_probe(dg, srcs, tgts)
    for i, s in enumerate(srcs.tolist()):
        st = O.source_state(og, s)
        assert np.array_equal(dist[i], st["dist"]), s
        assert np.array_equal(sig[i], st["sigma"]), s
        assert flags[i] == 0
        for j, t in enumerate(tgts.tolist()):
            if t == s:
                continue
            assert close(dep[i, j], st["delta"][t]), (s, t, dep[i, j], st["delta"][t])


@pytest.mark.parametrize("cfg", [{}, {"tile_words": 1}, {"tile_words": 2}, {"tile_words": 4, "blocks_per_sm": 1},
                                 {"tile_words": 4, "blocks_per_sm": 2}, {"tile_words": 8}, {"chunk_arcs": 32},
                                 {"block_threads": 256, "chunk_arcs": 64}])
def test_exact_matches_oracle(bcd, er1, cfg):
    g, og = er1
    dg = make(bcd, g, **cfg)
    qs = gg.random_vertices(g.n, 16, 102)
    for r in qs.tolist():
        got, info = bcd.bc_exact(dg, r)
        want, k, f = O.bc_exact(og, r, 0)
        assert info["rv_size"] == k
        assert close(got, want), (r, got, want)
        assert info["flags"] == f


def test_exact_matches_all_sources_brandes(bcd):
    g = gg.erdos_renyi(400, 2400, 77)
    og = O.Graph.from_csr(g)
    allbc = O.bc_all(og)
    dg = make(bcd, g)
    out, _ = bcd.bc_batch(dg, [{"r": r} for r in range(g.n)])
    for r in range(g.n):
        assert out[r]["status"] == 0
        assert close(out[r]["bc"], allbc[r]), (r, out[r]["bc"], allbc[r])


def test_batch_equals_single(bcd, sparse_er):
    g, og = sparse_er
    dg = make(bcd, g)
    qs = gg.random_vertices(g.n, 100, 5).tolist()  # > 64: two groups, repeated roots possible
    out, info = bcd.bc_batch(dg, [{"r": r} for r in qs])
    for r, o in zip(qs, out):
        single, _ = bcd.bc_exact(dg, r)
        want, k, _ = O.bc_exact(og, r, 0)
        assert o["status"] == 0 and o["rv_size"] == k
        assert close(o["bc"], want) and close(single, want)
    assert info["queries"] == 100


def test_sampled_draws_and_estimate(bcd, er1):
    g, og = er1
    dg = make(bcd, g)
    for r, T, seed in [(5, 1000, 7), (1234, 333, 99), (77, 14979, 7)]:
        draws, k = bcd.bc_draw_samples(dg, r, T, seed)
        want, wdraws, wk, _ = O.bc_approx(og, r, T, seed, 0)
        assert k == wk
        assert np.array_equal(draws, wdraws)
        got, info = bcd.bc_approx_T(dg, r, T, seed)
        assert info["samples"] == T and info["rv_size"] == k
        assert close(got, want), (r, got, want)


def test_approx_eps_delta(bcd, er1):
    g, og = er1
    dg = make(bcd, g)
    T = O.samples_for(0.05, 0.1)
    got, info = bcd.bc_approx(dg, 9, 0.05, 0.1, 7)
    want, _, _, _ = O.bc_approx(og, 9, T, 7, 0)
    assert info["samples"] == T
    assert close(got, want)


def test_mixed_batch(bcd, er1):
    """Exact, sampled and hybrid queries in one group, repeated roots."""
    g, og = er1
    dg = make(bcd, g)
    specs = []
    rs = gg.random_vertices(g.n, 30, 31).tolist()
    for i, r in enumerate(rs):
        kind = i % 4
        if kind == 0:
            specs.append({"r": r, "kind": bcd.BC_QUERY_EXACT})
        elif kind == 1:
            specs.append({"r": r, "kind": bcd.BC_QUERY_APPROX_T, "T": 700, "seed": 7})
        elif kind == 2:
            specs.append({"r": rs[0], "kind": bcd.BC_QUERY_APPROX_T, "T": 500, "seed": i})
        else:
            specs.append({"r": r, "kind": bcd.BC_QUERY_HYBRID, "T": 1000, "seed": 3})
    out, _ = bcd.bc_batch(dg, specs)
    for s, o in zip(specs, out):
        assert o["status"] == 0
        r = s["r"]
        rvk = O.rv(og, r).shape[0]
        if s["kind"] == bcd.BC_QUERY_EXACT or (s["kind"] == bcd.BC_QUERY_HYBRID and rvk <= s["T"]):
            want = O.bc_exact(og, r, 0)[0]
            assert o["samples"] == 0
        else:
            want = O.bc_approx(og, r, s["T"], s["seed"], 0)[0]
            assert o["samples"] == (s["T"] if rvk > 0 and g.out_degree()[r] > 0 else 0)
        assert close(o["bc"], want), (s, o["bc"], want)


# ---------------------------------------------------------------- edge cases

def test_trivial_zero_and_empty_rv(bcd):
    g = csr(5, [(0, 1), (1, 2), (3, 2), (2, 4)])
    dg = make(bcd, g)
    bc, info = bcd.bc_exact(dg, 4)  # out-degree 0
    assert bc == 0.0 and info["flags"] & bcd.BC_FLAG_TRIVIAL_ZERO and info["rv_size"] == 0
    bc, info = bcd.bc_exact(dg, 0)  # in-degree 0: RV empty
    assert bc == 0.0 and info["rv_size"] == 0 and info["sources_run"] == 0
    bc, info = bcd.bc_exact(dg, 2)
    assert bc == 3.0 and info["rv_size"] == 3  # pairs (0,4),(1,4),(3,4)
    bc, info = bcd.bc_approx_T(dg, 0, 10, 1)
    assert bc == 0.0 and info["samples"] == 0
    assert bcd.bc_rv_compute(dg, 0).shape[0] == 0
    draws, k = bcd.bc_draw_samples(dg, 4, 10, 1)
    assert k == 0 and draws.shape[0] == 0


def test_graph_without_arcs_and_single_vertex(bcd):
    g = gg.CSR(1, np.zeros(2, dtype=np.int64), np.zeros(0, dtype=np.int32))
    dg = make(bcd, g)
    assert bcd.bc_exact(dg, 0)[0] == 0.0
    g = gg.CSR(7, np.zeros(8, dtype=np.int64), np.zeros(0, dtype=np.int32))
    dg = make(bcd, g)
    assert bcd.bc_exact(dg, 3)[0] == 0.0
    assert bcd.bc_rv_compute(dg, 3).shape[0] == 0


def test_long_path_levels(bcd):
    n = 3000  # 2999 BFS levels in one tile
    g = csr(n, [(i, i + 1) for i in range(n - 1)])
    dg = make(bcd, g)
    for r in [1, 1500, n - 2]:
        assert bcd.bc_exact(dg, r)[0] == r * (n - 1 - r)


def test_heavy_rows_chunked(bcd):
    """A hub with 20,000 out-arcs and 20,000 in-arcs: rows split into many
    chunks whose partial sums are combined in order."""
    n = 20001
    arcs = [(0, i) for i in range(1, n)] + [(i, 0) for i in range(1, n)]
    arcs += [(i, i + 1) for i in range(1, n - 1)]
    g = csr(n, arcs)
    og = O.Graph.from_csr(g)
    want = {r: O.bc_exact(og, r, 0)[0] for r in [0, 5, 19999]}
    for cfg in [{}, {"chunk_arcs": 32}]:
        dg = make(bcd, g, **cfg)
        for r in want:
            got = bcd.bc_exact(dg, r)[0]
            assert close(got, want[r]), (cfg, r, got, want[r])


@pytest.mark.parametrize("k", [52, 53, 54, 60])
def test_sigma_flag(bcd, k):
    arcs = []
    for i in range(k):
        a, b, c, d = 3 * i, 3 * i + 1, 3 * i + 2, 3 * i + 3
        arcs += [(a, b), (a, c), (b, d), (c, d)]
    arcs.append((3 * k, 3 * k + 1))
    g = csr(3 * k + 2, arcs)
    og = O.Graph.from_csr(g)
    dg = make(bcd, g)
    dist, sig, _, flags = bcd.bc_spd_probe(dg, [0], [3 * k])
    st = O.source_state(og, 0)
    assert int(dist[0, 3 * k]) == 2 * k
    if k <= 52:
        assert np.array_equal(sig[0], st["sigma"])
    assert bool(flags[0] & bcd.BC_FLAG_SIGMA_2_53) == bool(st["flags"] & O.FLAG_SIGMA_GT_2_53)
    bc, info = bcd.bc_exact(dg, 3 * k)  # r = sink of the chain: 2^k paths from 0 reach it
    want, _, wf = O.bc_exact(og, 3 * k, 0)
    assert bool(info["flags"] & bcd.BC_FLAG_SIGMA_2_53) == bool(wf & O.FLAG_SIGMA_GT_2_53)
    if k <= 52:
        assert close(bc, want)


def test_invalid_graphs_rejected(bcd):
    def create(n, off, cols, w=None):
        return bcd.bc_graph_create(n, np.array(off, dtype=np.int64), np.array(cols, dtype=np.int32),
                                   None if w is None else np.array(w, dtype=np.uint32))
    with pytest.raises(bcd.BCError) as e:
        create(3, [0, 1, 1, 1], [0])  # self-loop
    assert e.value.status == bcd.BC_E_INVALID_GRAPH
    with pytest.raises(bcd.BCError) as e:
        create(3, [0, 2, 2, 2], [2, 1])  # unsorted row
    assert e.value.status == bcd.BC_E_INVALID_GRAPH
    with pytest.raises(bcd.BCError) as e:
        create(3, [0, 2, 2, 2], [1, 1])  # repeated arc
    assert e.value.status == bcd.BC_E_INVALID_GRAPH
    with pytest.raises(bcd.BCError) as e:
        create(3, [0, 1, 1, 1], [5])  # head out of range
    assert e.value.status == bcd.BC_E_INVALID_ARG
    with pytest.raises(bcd.BCError) as e:
        create(3, [0, 2, 1, 1], [1, 2])  # offsets decrease
    assert e.value.status == bcd.BC_E_INVALID_ARG
    dg = create(3, [0, 1, 2, 2], [1, 2])
    with pytest.raises(bcd.BCError) as e:
        bcd.bc_exact(dg, 3)
    assert e.value.status == bcd.BC_E_INVALID_ARG
    with pytest.raises(bcd.BCError):
        bcd.bc_approx(dg, 1, 0.0, 0.1, 1)
    out, _ = bcd.bc_batch(dg, [{"r": 1}, {"r": -1}, {"r": 1, "kind": bcd.BC_QUERY_APPROX, "eps": 0.1,
                                                     "delta": 2.0}])
    assert out[0]["status"] == 0 and out[0]["bc"] == 1.0
    assert out[1]["status"] == bcd.BC_E_INVALID_ARG and out[2]["status"] == bcd.BC_E_INVALID_ARG


# ---------------------------------------------------------------- weighted

@pytest.fixture(scope="module")
def wer():
    """ER 600 / 4,000 with weights uniform in [1, 255] (seed 3) and a copy
    with weights in [1, 3], whose many equal-length paths make sigma > 1."""
    g = gg.erdos_renyi(600, 4000, 21)
    g255 = g.with_weights(gg.uniform_weights(g.m, 1, 255, 3))
    g3 = g.with_weights(gg.uniform_weights(g.m, 1, 3, 4))
    return [(x, O.Graph.from_csr(x)) for x in (g255, g3)]


WCFGS = [{}, {"weighted_words": 1}, {"weighted_words": 4, "chunk_arcs": 32},
         {"weighted_kernel": 1}, {"weighted_kernel": 1, "weighted_words": 1},
         {"weighted_kernel": 1, "weighted_words": 4, "chunk_arcs": 32},
         {"weighted_short_row": 2, "chunk_arcs": 32, "block_threads": 128},
         {"weighted_words": 16}, {"weighted_kernel": 1, "weighted_words": 16}]


@pytest.mark.parametrize("cfg", WCFGS)
@pytest.mark.parametrize("which", [0, 1])
def test_weighted_probe_dist_sigma_delta(bcd, wer, which, cfg):
    g, og = wer[which]
    dg = make(bcd, g, **cfg)
    srcs = np.array(sorted(set(gg.random_vertices(g.n, 30, 5).tolist())), dtype=np.int32)
    tgts = np.array(list(dict.fromkeys(gg.random_vertices(g.n, 12, 6).tolist())), dtype=np.int32)
    dist, sig, dep, flags = bcd.bc_spd_probe(dg, srcs, tgts)
    for i, s in enumerate(srcs.tolist()):
        st = O.source_state(og, s)
        assert np.array_equal(dist[i], st["dist"]), s
        assert np.array_equal(sig[i], st["sigma"]), s
        for j, t in enumerate(tgts.tolist()):
            if t != s:
                assert close(dep[i, j], st["delta"][t]), (s, t, dep[i, j], st["delta"][t])


@pytest.mark.parametrize("cfg", WCFGS)
@pytest.mark.parametrize("which", [0, 1])
def test_weighted_exact_and_batch(bcd, wer, which, cfg):
    """Batches over several tiles (64-source tiles) with a ragged last tile,
    and one wide tile; long rows split into 32-arc chunks."""
    g, og = wer[which]
    dg = make(bcd, g, **cfg)
    qs = gg.random_vertices(g.n, 12, 104).tolist()
    out, _ = bcd.bc_batch(dg, [{"r": r} for r in qs])
    for r, o in zip(qs, out):
        want, k, _ = O.bc_exact(og, r, 0)
        single, info = bcd.bc_exact(dg, r)
        assert o["status"] == 0 and o["rv_size"] == k == info["rv_size"]
        assert close(o["bc"], want) and close(single, want), (r, o["bc"], single, want)


def test_weighted_repeated_multitile(bcd, wer):
    """Many launches of ten 64-source tiles (weights 1..3: many ties and
    distance levels): every result must match, run after run. Guards the
    ordering between the last forward level and the backward pass."""
    g, og = wer[1]
    qs = gg.random_vertices(g.n, 6, 104).tolist()
    want = {r: O.bc_exact(og, r, 0)[0] for r in qs}
    for it in range(6):
        dg = make(bcd, g, weighted_words=1, block_threads=(512, 256, 128)[it % 3])
        for r in qs:
            got, _ = bcd.bc_exact(dg, r)
            assert close(got, want[r]), (it, r, got, want[r])
        dg.close()


def test_weighted_closed_forms_and_sampling(bcd, wer):
    wt = csr(3, [(0, 1), (0, 2), (2, 1)], [2, 1, 1])
    dg = make(bcd, wt)
    assert bcd.bc_exact(dg, 2)[0] == 0.5
    path = csr(5, [(i, i + 1) for i in range(4)], [7, 1, 255, 3])
    dg = make(bcd, path)
    assert [bcd.bc_exact(dg, r)[0] for r in range(5)] == [0.0, 3.0, 4.0, 3.0, 0.0]
    g, og = wer[1]
    dg = make(bcd, g)
    for r in (4, 77):
        want, draws, k, _ = O.bc_approx(og, r, 600, 7, 0)
        got, info = bcd.bc_approx_T(dg, r, 600, 7)
        assert info["rv_size"] == k and close(got, want)


@pytest.mark.parametrize("cfg", [{}, {"weighted_words": 2, "chunk_arcs": 64}, {"weighted_kernel": 1},
                                 {"weighted_short_row": 8, "block_threads": 256}])
def test_weighted_rmat_small(bcd, cfg):
    """A small weighted R-MAT (the weighted configuration at scale 12): hub
    rows of hundreds of arcs go through the chunked path."""
    g = gg.rmat(12, 8, seed=12)
    g = g.with_weights(gg.uniform_weights(g.m, 1, 255, 3))
    og = O.Graph.from_csr(g)
    dg = make(bcd, g, **cfg)
    qs = gg.random_vertices(g.n, 8, 104).tolist() + gg.top_inout_vertices(g, 2).tolist()
    out, _ = bcd.bc_batch(dg, [{"r": r} for r in qs])
    for r, o in zip(qs, out):
        want = O.bc_exact(og, r, 0)[0]
        assert close(o["bc"], want), (r, o["bc"], want)


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("lo", [1, 4000])
def test_weighted_largest_weights(bcd, kernel, lo):
    """Weights up to 4095, the largest the library takes (a ring of 4,096
    distance slots): uniform in [1, 4095], or in [4000, 4095] where a
    distance value rarely repeats; exact scores of a batch against the
    oracle."""
    g = gg.erdos_renyi(600, 4000, 21)
    g = g.with_weights(gg.uniform_weights(g.m, lo, 4095, 8))
    og = O.Graph.from_csr(g)
    dg = make(bcd, g, weighted_kernel=kernel)
    qs = gg.random_vertices(g.n, 10, 104).tolist()
    out, _ = bcd.bc_batch(dg, [{"r": r} for r in qs])
    for r, o in zip(qs, out):
        want = O.bc_exact(og, r, 0)[0]
        assert o["status"] == 0 and close(o["bc"], want), (r, o["bc"], want)
    with pytest.raises(bcd.BCError) as e:
        w = g.weights.copy()
        w[0] = 4096
        bcd.bc_graph_create(g.n, g.offsets, g.cols, w)
    assert e.value.status == bcd.BC_E_INVALID_GRAPH


@pytest.mark.parametrize("kernel", [1, 2])
def test_weighted_large_counts(bcd, kernel):
    """Layers of 4 vertices, each joined to all 4 of the next by arcs of
    weight 1, 24 layers: path counts between the first and the
    last layers reach 4^22 = 2^44, past what the source kernel's 8-byte
    words hold (2^40), so its vertex-scan launch reruns with 16-byte pairs.
    Exact scores of the vertex scan (the default for one query vertex) and
    of the Eq. 4 pull against the oracle; no count reaches 2^53."""
    L, k = 24, 4
    arcs = [(l * k + i, (l + 1) * k + j) for l in range(L - 1) for i in range(k) for j in range(k)]
    g = csr(L * k, arcs, [1] * len(arcs))
    og = O.Graph.from_csr(g)
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols, g.weights)
    bcd.bc_set_config(dg, weighted_kernel=kernel)
    for acc in (4, 1):
        bcd.bc_set_config(dg, accumulation=acc)
        for r in (k * 12 + 1, k * 3, k * 20 + 3):
            got, info = bcd.bc_exact(dg, r)
            want, _, flags = O.bc_exact(og, r, 0)
            assert flags == 0 and info["flags"] == 0
            assert close(got, want), (acc, r, got, want)
    dg.close()


@pytest.mark.parametrize("kernel", [1, 2])
def test_weighted_growth_paths_closed_forms(bcd, kernel):
    """Capacities that start too small and grow on the rerun.
    - A directed path of 10,000 vertices with weights 1..2 has about 15,000
      distinct distances from its first vertex (more than the initial level
      arrays hold); BC(r) = r (n - 1 - r) whatever the weights.
    - An out-star of 20,000 leaves of weight 1, each leaf with an arc to one
      sink, queues every leaf at distance 1 from the centre (more than a
      ring slot of the source kernel holds at first) and gives the sink
      20,000 in-arcs: BC(leaf) = 1 / 20,000, BC(centre) = BC(sink) = 0.
    - The same star with arcs to two sinks, and every row longer than one
      arc cut into chunks: two chunks per leaf at distance 1 (more than the
      source kernel's chunk list holds at first); BC(leaf) = 2 / 20,000."""
    n = 10000
    w = gg.uniform_weights(n - 1, 1, 2, 9)
    path = csr(n, [(i, i + 1) for i in range(n - 1)], w.tolist())
    dg = make(bcd, path, weighted_kernel=kernel)
    rs = [1, 300, 2000]
    out, _ = bcd.bc_batch(dg, [{"r": r} for r in rs])
    for r, o in zip(rs, out):
        assert o["status"] == 0 and o["bc"] == float(r * (n - 1 - r)), (r, o)
    dg.close()
    L = 20000
    arcs = [(0, 1 + i) for i in range(L)] + [(1 + i, L + 1) for i in range(L)]
    star = csr(L + 2, arcs, [1] * len(arcs))
    dg = make(bcd, star, weighted_kernel=kernel)
    out, _ = bcd.bc_batch(dg, [{"r": 1}, {"r": 777}, {"r": 0}, {"r": L + 1}])
    assert [o["bc"] for o in out] == [1.0 / L, 1.0 / L, 0.0, 0.0], out
    dg.close()
    arcs2 = [(0, 1 + i) for i in range(L)] + [(1 + i, L + 1) for i in range(L)] + [(1 + i, L + 2) for i in range(L)]
    star2 = csr(L + 3, arcs2, [1] * len(arcs2))
    dg = make(bcd, star2, weighted_kernel=kernel, weighted_short_row=1, chunk_arcs=32)
    out, _ = bcd.bc_batch(dg, [{"r": 1}, {"r": L}, {"r": L + 2}])
    assert [o["bc"] for o in out] == [2.0 / L, 2.0 / L, 0.0], out
    dg.close()


def test_device_input_arrays(bcd, er1):
    torch = pytest.importorskip("torch")
    g, og = er1
    off = torch.from_numpy(g.offsets).cuda()
    col = torch.from_numpy(g.cols).cuda()
    dg = bcd.bc_graph_create(g.n, off, col)
    r = 11
    assert close(bcd.bc_exact(dg, r)[0], O.bc_exact(og, r, 0)[0])


@pytest.mark.parametrize("nshards", [1, 2, 3, 5])
def test_batch_shards_add_up(bcd, er1, nshards):
    """bc_batch_shard: the shards' partial scores of a mixed batch (exact,
    sampled, hybrid; 128-source tiles, so each group has several tiles) add
    up, in shard order, to the oracle's scores; rv_size, samples and status
    agree on every shard."""
    from paper_1708_08739_gb300 import shard as sh
    g, og = er1
    dg = make(bcd, g, tile_words=2)
    rs = gg.random_vertices(g.n, 12, 41).tolist()
    specs = []
    for i, r in enumerate(rs):
        if i % 3 == 0:
            specs.append({"r": r, "kind": bcd.BC_QUERY_EXACT})
        elif i % 3 == 1:
            specs.append({"r": r, "kind": bcd.BC_QUERY_APPROX_T, "T": 900, "seed": 7})
        else:
            specs.append({"r": r, "kind": bcd.BC_QUERY_HYBRID, "T": 1000, "seed": 3})
    parts = {}
    outs = []
    for k in range(nshards):
        out, info = bcd.bc_batch_shard(dg, specs, k, nshards)
        parts[k] = [o["bc"] for o in out]
        outs.append(out)
    tot = sh.reduce_in_shard_order(parts, nshards, len(specs))
    for i, s in enumerate(specs):
        r = s["r"]
        rvk = O.rv(og, r).shape[0]
        if s["kind"] == bcd.BC_QUERY_EXACT or (s["kind"] == bcd.BC_QUERY_HYBRID and rvk <= s["T"]):
            want = O.bc_exact(og, r, 0)[0]
        else:
            want = O.bc_approx(og, r, s["T"], s["seed"], 0)[0]
        assert close(tot[i], want), (nshards, s, tot[i], want)
        for out in outs:
            assert out[i]["status"] == 0 and out[i]["rv_size"] == outs[0][i]["rv_size"]
            assert out[i]["samples"] == outs[0][i]["samples"]
    with pytest.raises(bcd.BCError):
        bcd.bc_batch_shard(dg, specs, nshards, nshards)


@pytest.mark.parametrize("nshards", [1, 3])
def test_weighted_batch_shards_add_up(bcd, wer, nshards):
    """bc_batch_shard on a weighted graph (the source kernel, 64-source
    tiles): exact and sampled queries, the shards' partial scores summed in
    shard order equal the oracle's."""
    from paper_1708_08739_gb300 import shard as sh
    g, og = wer[1]
    dg = make(bcd, g, weighted_words=1)
    rs = gg.random_vertices(g.n, 8, 42).tolist()
    specs = [{"r": r, "kind": bcd.BC_QUERY_EXACT} if i % 2 == 0 else
             {"r": r, "kind": bcd.BC_QUERY_APPROX_T, "T": 500, "seed": 9} for i, r in enumerate(rs)]
    parts = {}
    for k in range(nshards):
        out, _ = bcd.bc_batch_shard(dg, specs, k, nshards)
        assert all(o["status"] == 0 for o in out)
        parts[k] = [o["bc"] for o in out]
    tot = sh.reduce_in_shard_order(parts, nshards, len(specs))
    for i, s in enumerate(specs):
        if s["kind"] == bcd.BC_QUERY_EXACT:
            want = O.bc_exact(og, s["r"], 0)[0]
        else:
            want = O.bc_approx(og, s["r"], s["T"], s["seed"], 0)[0]
        assert close(tot[i], want), (nshards, s, tot[i], want)


# ---------------------------------------------------------------- bottom-up levels

@pytest.mark.parametrize("cfg", [{"pull_permille": 1}, {"pull_permille": 1, "tile_words": 1},
                                 {"pull_permille": 1, "tile_words": 2, "chunk_arcs": 32},
                                 {"pull_permille": 1, "tile_words": 4, "blocks_per_sm": 1},
                                 {"pull_permille": 50}])
def test_bottom_up_levels_bit_exact(bcd, er1, cfg):
    """Forward levels run bottom-up (every level from 1 on with 1 permille):
    distances and sigma stay bit-exact, dependencies and scores within the
    bar, in both accumulations."""
    g, og = er1
    dg = make(bcd, g, **cfg)
    srcs = np.array(sorted(set(gg.random_vertices(g.n, 40, 7).tolist())), dtype=np.int32)[:37]
    tgts = np.array(list(dict.fromkeys(gg.random_vertices(g.n, 20, 8).tolist())), dtype=np.int32)
    dist, sig, dep, flags = bcd.bc_spd_probe(dg, srcs, tgts)
    for i, s in enumerate(srcs.tolist()):
        st = O.source_state(og, s)
        assert np.array_equal(dist[i], st["dist"]), s
        assert np.array_equal(sig[i], st["sigma"]), s
        for j, t in enumerate(tgts.tolist()):
            if t != s:
                assert close(dep[i, j], st["delta"][t]), (s, t, dep[i, j], st["delta"][t])
    qs = gg.random_vertices(g.n, 10, 102).tolist()
    out, info = bcd.bc_batch(dg, [{"r": r} for r in qs])
    assert info["pull_levels"] > 0
    for r, o in zip(qs, out):
        assert close(o["bc"], O.bc_exact(og, r, 0)[0]), r
    bcd.bc_set_config(dg, accumulation=2)
    got, _ = bcd.bc_exact(dg, qs[0])
    assert close(got, O.bc_exact(og, qs[0], 0)[0])


def test_bottom_up_heavy_rows(bcd):
    """A hub with 20,000 in-arcs: its in-arc row is cut into chunks whose
    sigma sums meet in atomic adds; path counts on a diamond chain reach
    2^52 through bottom-up levels."""
    n = 20001
    arcs = [(0, i) for i in range(1, n)] + [(i, 0) for i in range(1, n)]
    arcs += [(i, i + 1) for i in range(1, n - 1)]
    g = csr(n, arcs)
    og = O.Graph.from_csr(g)
    for cfg in [{"pull_permille": 1}, {"pull_permille": 1, "chunk_arcs": 32}]:
        dg = make(bcd, g, **cfg)
        for r in [0, 5, 19999]:
            assert close(bcd.bc_exact(dg, r)[0], O.bc_exact(og, r, 0)[0]), (cfg, r)
        dist, sig, _, _ = bcd.bc_spd_probe(dg, [3, 0, 700], [0])
        for i, s in enumerate([3, 0, 700]):
            st = O.source_state(og, s)
            assert np.array_equal(dist[i], st["dist"]) and np.array_equal(sig[i], st["sigma"]), (cfg, s)
    k = 52
    arcs = []
    for i in range(k):
        a, b, c, d = 3 * i, 3 * i + 1, 3 * i + 2, 3 * i + 3
        arcs += [(a, b), (a, c), (b, d), (c, d)]
    g = csr(3 * k + 1, arcs)
    og = O.Graph.from_csr(g)
    dg = make(bcd, g, pull_permille=1)
    dist, sig, _, flags = bcd.bc_spd_probe(dg, [0], [3 * k])
    st = O.source_state(og, 0)
    assert np.array_equal(sig[0], st["sigma"]) and sig[0, 3 * k] == 2.0 ** k and flags[0] == 0
