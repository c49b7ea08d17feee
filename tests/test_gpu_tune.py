"""The autotuner (bc_tune) on the GPU: it times candidates on a probe batch,
applies the fastest, and the tuned configuration answers the real batch as
the oracle does (within the parity bar), on an unweighted and a weighted
R-MAT graph; the tuning table stores and re-applies its answer."""
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


@pytest.mark.parametrize("weighted", [False, True])
def test_tuned_config_matches_oracle(bcd, weighted, tmp_path):
    from paper_1708_08739_gb300 import tuning
    g = gg.rmat(13, 8, seed=13)
    if weighted:
        g = g.with_weights(gg.uniform_weights(g.m, 1, 255, 3))
    og = O.Graph.from_csr(g)
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols, g.weights)
    qs = [int(x) for x in gg.random_vertices(g.n, 6, 33)] + [int(x) for x in gg.top_inout_vertices(g, 2)]
    specs = [{"r": r, "kind": bcd.BC_QUERY_APPROX_T, "T": 300, "seed": 7} for r in qs]
    path = str(tmp_path / "tune.json")
    cfg, entry = tuning.tuned(dg, g.offsets, specs, path, probe_T=64)
    rep = entry["report"]
    assert rep["candidates"] >= 8 and rep["ms_best"] <= rep["ms_default"]
    got = bcd.bc_get_config(dg)
    assert all(got[k] == v for k, v in cfg.items()), (got, cfg)
    out, _ = bcd.bc_batch(dg, specs)
    threads = os.cpu_count() or 1
    for s, o in zip(specs, out):
        want = O.bc_approx(og, s["r"], s["T"], s["seed"], threads)[0]
        assert o["status"] == 0 and close(o["bc"], want), (cfg, s, o["bc"], want)
    # a second handle of the same graph takes the stored answer
    dg2 = bcd.bc_graph_create(g.n, g.offsets, g.cols, g.weights)
    cfg2, _ = tuning.tuned(dg2, g.offsets, specs, path, probe_T=64)
    assert cfg2 == cfg and all(bcd.bc_get_config(dg2)[k] == v for k, v in cfg.items())
