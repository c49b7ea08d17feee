"""Pins of the CPU oracle against things other than itself.

Each test ties one part of the oracle to mathematics the paper fixes, to a
library routine, or to brute force, so that a dropped term, a wrong sign or
index, or a transposed operand fails at least one of them:

* Eq. 1 (BC definition): brute-force enumeration of all simple paths on
  every 3- and 4-vertex digraph and on random small weighted/unweighted
  digraphs; networkx's Brandes implementation on random digraphs.
* Section 2 (d, sigma): scipy BFS/Dijkstra distances; closed-form path counts
  (diamond chain sigma = 2^k, grid DAG sigma = binomial).
* Eq. 4 (recursion): closed forms on paths, cycles, stars, diamonds; an
  independent dependency formula (pair dependencies of Eq. 2) from two BFS
  runs, and from two Dijkstra runs on weighted graphs; the global sum
  identity.
* Prop. 1 / Eq. 5 (pruning), Prop. 2 (RV via R(G)): all-sources equality and
  forward reachability through scipy.
* Algorithm 2 / Props. 3-4: Philox against numpy's Philox, unbiasedness over
  seeds, Hoeffding coverage, and the sample-count formula.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import graphgen as gg
import oracle as O
from helpers import arcs_of, bfs_dist_sigma, brute_force_bc, csr, dijkstra_dist_sigma, random_digraph

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def og(g):
    return O.Graph.from_csr(g)


# --------------------------------------------------------------------------
# Eq. 1 against brute force
# --------------------------------------------------------------------------

def _check_against_brute(g, tol=1e-12):
    G = og(g)
    brute = brute_force_bc(g)
    allbc = O.bc_all(G)
    for r in range(g.n):
        exact, _, _ = O.bc_exact(G, r, nthreads=1)
        want = float(brute[r])
        assert abs(exact - want) <= tol * max(1.0, abs(want)), (r, exact, want, arcs_of(g))
        assert abs(allbc[r] - want) <= tol * max(1.0, abs(want)), (r, allbc[r], want)


@pytest.mark.parametrize("n", [3, 4])
def test_all_small_digraphs_match_brute_force(n):
    pairs = [(u, v) for u in range(n) for v in range(n) if u != v]
    step = 1 if n == 3 else 3  # every 3-vertex digraph; every third 4-vertex one
    for mask in range(0, 1 << len(pairs), step):
        arcs = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        _check_against_brute(csr(n, arcs))


@pytest.mark.parametrize("seed", range(12))
def test_random_unweighted_match_brute_force(seed):
    n = 6 + seed % 3
    _check_against_brute(random_digraph(n, 0.3, seed))


@pytest.mark.parametrize("seed", range(12))
def test_random_weighted_match_brute_force(seed):
    n = 6 + seed % 3
    _check_against_brute(random_digraph(n, 0.35, 100 + seed, weighted=True, wmax=3))


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("seed", range(4))
def test_networkx_brandes(weighted, seed):
    nx = pytest.importorskip("networkx")
    g = random_digraph(40, 0.08, 500 + seed, weighted=weighted, wmax=5)
    D = nx.DiGraph()
    D.add_nodes_from(range(g.n))
    t, h = g.arcs()
    for i in range(g.m):
        D.add_edge(int(t[i]), int(h[i]), weight=int(g.weights[i]) if weighted else 1)
    want = nx.betweenness_centrality(D, normalized=False, weight="weight" if weighted else None)
    G = og(g)
    for r in range(g.n):
        got, _, _ = O.bc_exact(G, r, nthreads=2)
        assert got == pytest.approx(want[r], rel=1e-12, abs=1e-12)


# --------------------------------------------------------------------------
# Closed forms
# --------------------------------------------------------------------------

def test_directed_path():
    n = 9
    g = csr(n, [(i, i + 1) for i in range(n - 1)])
    G = og(g)
    for i in range(n):  # 0-based i: (i) * (n - 1 - i)
        assert O.bc_exact(G, i, 1)[0] == i * (n - 1 - i)


def test_directed_cycle():
    n = 7
    g = csr(n, [(i, (i + 1) % n) for i in range(n)])
    G = og(g)
    for v in range(n):
        assert O.bc_exact(G, v, 1)[0] == (n - 1) * (n - 2) / 2


def test_stars_and_complete():
    n = 6
    bidir = csr(n, [(0, i) for i in range(1, n)] + [(i, 0) for i in range(1, n)])
    G = og(bidir)
    assert O.bc_exact(G, 0, 1)[0] == (n - 1) * (n - 2)
    assert all(O.bc_exact(G, v, 1)[0] == 0 for v in range(1, n))
    out_star = og(csr(n, [(0, i) for i in range(1, n)]))
    in_star = og(csr(n, [(i, 0) for i in range(1, n)]))
    assert O.bc_exact(out_star, 0, 1)[0] == 0  # no in-arcs: RV(0) empty
    assert O.bc_exact(in_star, 0, 1)[0] == 0   # no out-arcs: Prop. 1
    assert O.bc_exact(out_star, 0, 1)[1] == 0
    comp = og(csr(n, [(u, v) for u in range(n) for v in range(n) if u != v]))
    assert all(O.bc_exact(comp, v, 1)[0] == 0 for v in range(n))


def test_diamond_and_weighted_tie():
    d = og(csr(4, [(0, 1), (0, 2), (1, 3), (2, 3)]))
    assert O.bc_exact(d, 1, 1)[0] == 0.5
    assert O.bc_exact(d, 2, 1)[0] == 0.5
    # a->b weight 2, a->c weight 1, c->b weight 1: two shortest a->b paths
    wt = og(csr(3, [(0, 1), (0, 2), (2, 1)], [2, 1, 1]))
    assert O.bc_exact(wt, 2, 1)[0] == 0.5
    # same graph unweighted: a->b direct is the only shortest path
    uw = og(csr(3, [(0, 1), (0, 2), (2, 1)]))
    assert O.bc_exact(uw, 2, 1)[0] == 0.0


def diamond_chain(k):
    """k diamonds in series: vertices 0..3k, sigma(source -> sink) = 2^k."""
    arcs = []
    for i in range(k):
        a, b, c, d = 3 * i, 3 * i + 1, 3 * i + 2, 3 * i + 3
        arcs += [(a, b), (a, c), (b, d), (c, d)]
    return csr(3 * k + 1, arcs)


@pytest.mark.parametrize("k", [1, 5, 30, 53, 54, 60])
def test_sigma_diamond_chain(k):
    g = diamond_chain(k)
    st = O.source_state(og(g), 0)
    sink = 3 * k
    assert O.sigma_exact(st, sink) == 2 ** k
    assert int(st["dist"][sink]) == 2 * k
    if k <= 53:
        assert st["sigma"][sink] == float(2 ** k)
    if k < 53:
        assert st["flags"] == 0
    else:  # 2^53 and beyond: fp64 sums can no longer be certified exact
        assert st["flags"] & O.FLAG_SIGMA_GT_2_53


def test_sigma_grid_dag():
    k = 8
    idx = lambda i, j: i * k + j
    arcs = []
    for i in range(k):
        for j in range(k):
            if i + 1 < k:
                arcs.append((idx(i, j), idx(i + 1, j)))
            if j + 1 < k:
                arcs.append((idx(i, j), idx(i, j + 1)))
    st = O.source_state(og(csr(k * k, arcs)), 0)
    for i in range(k):
        for j in range(k):
            assert O.sigma_exact(st, idx(i, j)) == math.comb(i + j, i)
            assert int(st["dist"][idx(i, j)]) == i + j


# --------------------------------------------------------------------------
# Distances and RV against scipy; Prop. 1 and Prop. 2
# --------------------------------------------------------------------------

def _scipy_matrix(g, weighted):
    from scipy.sparse import csr_matrix
    data = g.weights.astype(np.float64) if weighted else np.ones(g.m)
    return csr_matrix((data, g.cols, g.offsets), shape=(g.n, g.n))


@pytest.mark.parametrize("weighted", [False, True])
def test_distances_match_scipy(weighted):
    from scipy.sparse.csgraph import shortest_path
    g = gg.erdos_renyi(300, 900, 11)
    if weighted:
        g = g.with_weights(gg.uniform_weights(g.m, 1, 255, 3))
    D = shortest_path(_scipy_matrix(g, weighted), method="D", directed=True,
                      unweighted=not weighted, indices=[0, 7, 123])
    G = og(g)
    for row, s in enumerate([0, 7, 123]):
        st = O.source_state(G, s)
        d = st["dist"]
        ref = D[row]
        reach = np.isfinite(ref)
        assert np.array_equal(d != np.iinfo(np.uint64).max, reach)
        assert np.array_equal(d[reach].astype(np.float64), ref[reach])


def test_rv_is_set_of_vertices_reaching_r():
    from scipy.sparse.csgraph import shortest_path
    g = gg.erdos_renyi(400, 700, 5)
    D = shortest_path(_scipy_matrix(g, False), directed=True, unweighted=True)
    G = og(g)
    for r in [0, 3, 77, 399]:
        want = np.array([v for v in range(g.n) if v != r and np.isfinite(D[v, r])], dtype=np.int32)
        assert np.array_equal(O.rv(G, r), want)


@pytest.mark.parametrize("weighted", [False, True])
def test_pruned_equals_all_sources(weighted):
    g = gg.erdos_renyi(150, 400, 17)
    if weighted:
        g = g.with_weights(gg.uniform_weights(g.m, 1, 9, 4))
    G = og(g)
    allbc = O.bc_all(G)
    outd = g.out_degree()
    ind = g.in_degree()
    for r in range(g.n):
        bc, k, _ = O.bc_exact(G, r, 2)
        assert bc == pytest.approx(allbc[r], rel=1e-12, abs=1e-12)
        if outd[r] == 0 or ind[r] == 0:
            assert bc == 0.0
        if ind[r] == 0 and outd[r] > 0:
            assert k == 0


def test_reverse_graph_definition():
    g = gg.erdos_renyi(200, 1200, 9)
    G = og(g)
    fwd = set(arcs_of(g))
    rev = set()
    for u in range(g.n):
        for e in range(G.roff[u], G.roff[u + 1]):
            rev.add((u, int(G.rcol[e])))
    assert rev == {(v, u) for (u, v) in fwd}
    for u in range(g.n):  # rows ascend
        row = G.rcol[G.roff[u]:G.roff[u + 1]]
        assert np.all(np.diff(row) > 0)


# --------------------------------------------------------------------------
# Eq. 4 against an independent formula, and a global identity
# --------------------------------------------------------------------------

def test_dependency_matches_pair_formula():
    """delta_s.(r) = sigma_sr * sum_t [d(s,r)+d(r,t) = d(s,t)] sigma_rt/sigma_st,
    with sigma_st(r) = sigma_sr * sigma_rt (Bellman criterion)."""
    g = gg.erdos_renyi(120, 420, 23)
    G = og(g)
    for r in [1, 50, 99]:
        dr, sr = bfs_dist_sigma(g, r)
        srcs = O.rv(G, r)[:25]
        dep, _, _ = O.dependencies(G, srcs, [r], nthreads=2)
        for i, s in enumerate(srcs.tolist()):
            ds, ss = bfs_dist_sigma(g, s)
            tot = Fraction(0)
            for t in range(g.n):
                if t in (s, r) or ds[t] < 0 or dr[t] < 0:
                    continue
                if ds[r] + dr[t] == ds[t]:
                    tot += Fraction(ss[r] * sr[t], ss[t])
            assert dep[i, 0] == pytest.approx(float(tot), rel=1e-12, abs=1e-12)


def test_weighted_dependency_matches_pair_formula():
    """The same identity with weighted distances (weights 1..3: many ties, so
    sigma > 1): Eq. 4 in the oracle against the pair dependencies of Eq. 2
    from two Dijkstra runs, the formula the weighted vertex scan sums."""
    g = gg.erdos_renyi(100, 400, 29).with_weights(gg.uniform_weights(400, 1, 3, 5))
    G = og(g)
    checked = 0
    for r in [2, 40, 77]:
        dr, sr = dijkstra_dist_sigma(g, r)
        srcs = O.rv(G, r)[:20]
        dep, _, _ = O.dependencies(G, srcs, [r], nthreads=2)
        for i, s in enumerate(srcs.tolist()):
            ds, ss = dijkstra_dist_sigma(g, s)
            tot = Fraction(0)
            for t in range(g.n):
                if t in (s, r) or ds[t] < 0 or dr[t] < 0:
                    continue
                if ds[r] + dr[t] == ds[t]:
                    tot += Fraction(ss[r] * sr[t], ss[t])
            assert dep[i, 0] == pytest.approx(float(tot), rel=1e-12, abs=1e-12)
            checked += tot > 0
    assert checked > 5


def test_sum_identity_unweighted():
    """sum_v BC(v) = sum over ordered reachable s != t of (d(s,t) - 1)."""
    g = gg.erdos_renyi(90, 300, 31)
    G = og(g)
    total = sum(O.bc_exact(G, r, 2)[0] for r in range(g.n))
    want = 0
    for s in range(g.n):
        d, _ = bfs_dist_sigma(g, s)
        want += sum(x - 1 for t, x in enumerate(d) if t != s and x > 0)
    assert total == pytest.approx(want, rel=1e-11)


def test_sum_identity_weighted():
    """sum_v BC(v) = sum_{s,t} (H_st / sigma_st - 1), H_st the total hop
    count over shortest s-t paths (forward DP over the SPD)."""
    import heapq
    g = gg.erdos_renyi(70, 260, 37).with_weights(gg.uniform_weights(260, 1, 4, 8))
    G = og(g)
    total = sum(O.bc_exact(G, r, 2)[0] for r in range(g.n))
    want = Fraction(0)
    for s in range(g.n):
        dist = {s: 0}
        pq = [(0, s)]
        order = []
        done = set()
        while pq:
            d, x = heapq.heappop(pq)
            if x in done:
                continue
            done.add(x)
            order.append(x)
            for e in range(g.offsets[x], g.offsets[x + 1]):
                y, w = int(g.cols[e]), int(g.weights[e])
                if y not in dist or d + w < dist[y]:
                    dist[y] = d + w
                    heapq.heappush(pq, (d + w, y))
        sig = {s: 1}
        hop = {s: 0}
        for x in order[1:]:
            sig[x] = 0
            hop[x] = 0
        for x in order:  # push along tight arcs, in distance order
            for e in range(g.offsets[x], g.offsets[x + 1]):
                y, w = int(g.cols[e]), int(g.weights[e])
                if dist[x] + w == dist[y]:
                    sig[y] += sig[x]
                    hop[y] += hop[x] + sig[x]
        for t in order[1:]:
            want += Fraction(hop[t], sig[t]) - 1
    assert total == pytest.approx(float(want), rel=1e-11)


# --------------------------------------------------------------------------
# Sampling: Philox, index map, T, Props. 3-4
# --------------------------------------------------------------------------

@pytest.mark.parametrize("key", [0, 7, 2**64 - 1, 0x0123456789ABCDEF + (0xFEDCBA9876543210 << 64)])
def test_philox_matches_numpy(key):
    for ctr in [0, 1, 2**64 - 1, 2**64, (5 << 130) + 17]:
        # numpy advances the 256-bit counter by one before each block
        ref = np.random.Philox(key=key, counter=ctr).random_raw(4)
        nxt = ctr + 1
        words = [(nxt >> (64 * i)) & (2**64 - 1) for i in range(4)]
        mine = O.philox4x64_10(words, [key & (2**64 - 1), key >> 64])
        assert np.array_equal(mine, ref), (key, ctr)


def test_sample_index_mapping():
    for seed in [7, 99]:
        for k in [1, 2, 3, 1000, 2**31 - 1]:
            for t in [0, 1, 14978]:
                x0 = int(np.random.Philox(key=seed, counter=t - 1 if t > 0 else 2**256 - 1)
                         .random_raw(1)[0])
                assert O.sample_index(seed, t, k) == (x0 * k) >> 64


def test_sample_count_formula():
    assert O.samples_for(0.01, 0.1) == 14979
    assert O.samples_for(0.02, 0.1) == 3745
    assert O.samples_for(0.5, 0.5) == math.ceil(math.log(4) / 0.5)
    with pytest.raises(ValueError):
        O.samples_for(0.0, 0.1)
    with pytest.raises(ValueError):
        O.samples_for(0.1, 1.0)


def test_approx_samples_are_the_stream():
    g = gg.erdos_renyi(200, 800, 41)
    G = og(g)
    r = 10
    rvl = O.rv(G, r)
    bc, draws, k, _ = O.bc_approx(G, r, 500, 7, 2)
    assert k == rvl.shape[0]
    want = np.array([rvl[O.sample_index(7, t, k)] for t in range(500)], dtype=np.int32)
    assert np.array_equal(draws, want)
    dep, _, _ = O.dependencies(G, want, [r], 2)
    assert bc == pytest.approx(float(np.sum(dep[:, 0]) * k / 500), rel=1e-12)


def test_approx_unbiased_prop3():
    g = gg.erdos_renyi(60, 200, 43)
    G = og(g)
    r = int(np.argmax(g.in_degree() * g.out_degree()))
    exact, k, _ = O.bc_exact(G, r, 2)
    assert k > 5
    T = 8
    ests = np.array([O.bc_approx(G, r, T, seed, 1)[0] for seed in range(3000)])
    se = ests.std(ddof=1) / math.sqrt(len(ests))
    assert abs(ests.mean() - exact) < 4 * se + 1e-9


def test_hoeffding_coverage_prop4():
    g = gg.erdos_renyi(50, 170, 47)
    G = og(g)
    r = int(np.argmax(g.in_degree() * g.out_degree()))
    exact, k, _ = O.bc_exact(G, r, 2)
    rvl = O.rv(G, r)
    dep, _, _ = O.dependencies(G, rvl, [r], 2)
    K = float(dep.max())  # the maximum dependency on r
    eps_rel, delta = 0.2, 0.2
    T = O.samples_for(eps_rel, delta)
    bad = 0
    N = 400
    for seed in range(N):
        est = O.bc_approx(G, r, T, 1000 + seed, 1)[0]
        bad += abs(est - exact) > eps_rel * K * k
    # P[fail] <= delta; allow binomial slack of 4 standard deviations
    assert bad <= N * delta + 4 * math.sqrt(N * delta * (1 - delta))


def test_zero_out_degree_short_circuit():
    g = csr(4, [(0, 1), (1, 2), (3, 2)])
    G = og(g)
    assert O.bc_exact(G, 2, 1) == (0.0, 0, 0)  # Algorithm 1: out-degree 0
    bc, draws, k, _ = O.bc_approx(G, 2, 10, 7, 1)
    assert bc == 0.0 and k == 0 and draws.shape[0] == 0
    assert O.bc_exact(G, 1, 1)[0] == 1.0
