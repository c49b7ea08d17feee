"""Serving loop (continuous batching): every result is the same alone and in
the mix, within the parity tolerance, including queries submitted while
others are running; sampled queries keep their own draw streams."""
import time

import numpy as np
import pytest

import graphgen as gg
import oracle as O
from helpers import close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import paper_1708_08739_gb300 as bcd
    g = gg.rmat(13, 8, seed=13)
    og = O.Graph.from_csr(g)
    rng = np.random.default_rng(3)
    rs = gg.zipf_vertices(g.n, 60, 1.1, 55).tolist() + gg.top_inout_vertices(g, 3).tolist()
    specs = []
    for i, r in enumerate(rs):
        k = i % 3
        if k == 0:
            specs.append({"r": r, "kind": bcd.BC_QUERY_EXACT})
        elif k == 1:
            specs.append({"r": r, "kind": bcd.BC_QUERY_APPROX_T, "T": 400, "seed": int(rng.integers(1, 1000))})
        else:
            specs.append({"r": r, "kind": bcd.BC_QUERY_APPROX, "eps": 0.1, "delta": 0.1, "seed": 7})
    return bcd, g, og, specs


def alone(bcd, dg, s):
    if s["kind"] == bcd.BC_QUERY_EXACT:
        return bcd.bc_exact(dg, s["r"])[0]
    if s["kind"] == bcd.BC_QUERY_APPROX_T:
        return bcd.bc_approx_T(dg, s["r"], s["T"], s["seed"])[0]
    return bcd.bc_approx(dg, s["r"], s["eps"], s["delta"], s["seed"])[0]


def test_server_mix_equals_alone(setup):
    bcd, g, og, specs = setup
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols)
    want = [alone(bcd, dg, s) for s in specs]
    srv = bcd.Server(dg, tiles_per_slice=2)
    # a first wave, then the rest while the first is running
    tickets = [srv.submit(s) for s in specs[:20]]
    time.sleep(0.05)
    tickets += [srv.submit(s) for s in specs[20:]]
    got = [None] * len(specs)
    lat = [None] * len(specs)
    deadline = time.time() + 300
    while any(x is None for x in got) and time.time() < deadline:
        for i, t in enumerate(tickets):
            if got[i] is None:
                r = srv.poll(t, timeout_us=1000)
                if r is not None:
                    got[i], lat[i] = r
    st = srv.stats()
    srv.close()
    assert all(x is not None for x in got)
    for s, gres, w in zip(specs, got, want):
        assert gres["status"] == 0
        assert close(gres["bc"], w), (s, gres["bc"], w)
    assert st["completed"] == len(specs) and st["slices"] > 0
    assert all(x >= 0.0 for x in lat)
    # spot checks against the oracle
    for s, gres in list(zip(specs, got))[:6]:
        if s["kind"] == bcd.BC_QUERY_EXACT:
            assert close(gres["bc"], O.bc_exact(og, s["r"], 0)[0])
        elif s["kind"] == bcd.BC_QUERY_APPROX_T:
            assert close(gres["bc"], O.bc_approx(og, s["r"], s["T"], s["seed"], 0)[0])


@pytest.mark.parametrize("kernel", [1, 2])
def test_server_weighted_mix_equals_alone(setup, kernel):
    """The same mix on the graph with weights 1..255 (seed 3), under the
    weighted tile kernel (1) and the source kernel (2): every served result
    equals the query alone, and spot checks equal the oracle."""
    bcd, g, og, specs = setup
    gw = g.with_weights(gg.uniform_weights(g.m, 1, 255, 3))
    ogw = O.Graph.from_csr(gw)
    dg = bcd.bc_graph_create(gw.n, gw.offsets, gw.cols, gw.weights)
    bcd.bc_set_config(dg, weighted_kernel=kernel)
    sub = specs[:30]
    want = [alone(bcd, dg, s) for s in sub]
    srv = bcd.Server(dg, tiles_per_slice=2)
    tickets = [srv.submit(s) for s in sub]
    got = [None] * len(sub)
    deadline = time.time() + 300
    while any(x is None for x in got) and time.time() < deadline:
        for i, t in enumerate(tickets):
            if got[i] is None:
                r = srv.poll(t, timeout_us=1000)
                if r is not None:
                    got[i] = r[0]
    srv.close()
    assert all(x is not None for x in got)
    for s, gres, w in zip(sub, got, want):
        assert gres["status"] == 0 and close(gres["bc"], w), (s, gres["bc"], w)
    for s, gres in list(zip(sub, got))[:6]:
        if s["kind"] == bcd.BC_QUERY_EXACT:
            assert close(gres["bc"], O.bc_exact(ogw, s["r"], 0)[0])
        elif s["kind"] == bcd.BC_QUERY_APPROX_T:
            assert close(gres["bc"], O.bc_approx(ogw, s["r"], s["T"], s["seed"], 0)[0])


def test_server_rejects_and_drains(setup):
    bcd, g, og, specs = setup
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols)
    srv = bcd.Server(dg, max_active=4, tiles_per_slice=1, max_queue=8)
    with pytest.raises(bcd.BCError):
        srv.submit({"r": g.n + 5})
    with pytest.raises(bcd.BCError):
        srv.submit({"r": 1, "kind": bcd.BC_QUERY_APPROX, "eps": 0.0, "delta": 0.1})
    ts = []
    busy = 0
    for s in specs[:30]:
        try:
            ts.append((s, srv.submit(s)))
        except bcd.BCError as e:
            assert e.status == bcd.BC_E_BUSY
            busy += 1
    results = []
    for s, t in ts:
        r = None
        while r is None:
            r = srv.poll(t, timeout_us=100000)
        assert r[0]["status"] == 0
        results.append((s, r[0]["bc"]))
    srv.close()
    assert len(ts) + busy == 30
    for s, bc in results:  # the graph is free again once the server is closed
        assert close(bc, alone(bcd, dg, s))


def test_server_memory_budget(setup):
    """Admission by device bytes, on a sparse ER graph (3,000 vertices,
    3,600 arcs: RV sizes from 1 to about 850). The budget fits either of two
    small exact queries but not both, and not the big one: the big query
    completes with BC_E_BUSY, the two small ones run one after the other and
    answer as alone."""
    bcd = setup[0]
    g = gg.erdos_renyi(3000, 3600, 2)
    og = O.Graph.from_csr(g)
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols)
    S = 64 * bcd.bc_get_config(dg)["tile_words"]
    sizes = {}
    for r in range(0, g.n, 7):
        if g.out_degree()[r] > 0:
            sizes[r] = bcd.bc_rv_compute(dg, r).shape[0]
    big = max(sizes, key=sizes.get)
    small = [r for r, k in sizes.items() if 50 <= k <= 110][:2]
    assert sizes[big] > 700 and len(small) == 2, sizes

    def staged(k):  # the header's count: 12 bytes per source, 512 per tile
        return 12 * k + (k + S - 1) // S * 512

    budget = max(staged(sizes[r]) for r in small) + min(staged(sizes[r]) for r in small) - 1
    assert staged(sizes[big]) > budget
    srv = bcd.Server(dg, max_device_bytes=budget)
    try:
        tb = srv.submit({"r": big, "kind": bcd.BC_QUERY_EXACT})
        ts = [srv.submit({"r": r, "kind": bcd.BC_QUERY_EXACT}) for r in small]
        res = {}
        deadline = time.time() + 120
        while len(res) < 3 and time.time() < deadline:
            for t in [tb] + ts:
                if t not in res:
                    x = srv.poll(t, timeout_us=2000)
                    if x is not None:
                        res[t] = x[0]
        assert len(res) == 3
        assert res[tb]["status"] == bcd.BC_E_BUSY
        for t, r in zip(ts, small):
            want = O.bc_exact(og, r, 0)[0]
            assert res[t]["status"] == 0 and res[t]["rv_size"] == sizes[r]
            assert close(res[t]["bc"], want), (r, res[t]["bc"], want)
        assert srv.stats()["admitted"] == 2
    finally:
        srv.close()
