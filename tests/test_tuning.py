"""The tuning table (paper_1708_08739_gb300.tuning) on the host: keys from
graph statistics, a first call that runs the tuner and stores its answer, a
second call on a graph of the same kind that applies the stored answer
without timing anything. The tuner and the config call are fakes here; the
library's bc_tune runs in tests/test_gpu_tune.py."""
import json

import numpy as np

import graphgen as gg
from paper_1708_08739_gb300 import tuning


class FakeGraph:
    def __init__(self, g):
        self.n, self.m, self.weighted = g.n, g.m, g.weights is not None


def test_keys_follow_graph_statistics():
    a = gg.rmat(12, 8, seed=1)
    b = gg.rmat(12, 8, seed=2)
    c = gg.erdos_renyi(4096, 32768, 3)
    ka = tuning.graph_key(a.n, a.offsets, False, [{"r": 1}, {"r": 2}])
    assert ka == tuning.graph_key(b.n, b.offsets, False, [{"r": 5}, {"r": 9}])  # same kind of graph
    assert ka != tuning.graph_key(c.n, c.offsets, False, [{"r": 1}, {"r": 2}])  # no hub: lower skew
    assert ka != tuning.graph_key(a.n, a.offsets, True, [{"r": 1}, {"r": 2}])
    assert ka != tuning.graph_key(a.n, a.offsets, False, [{"r": 1}, {"r": 1}])  # one query vertex
    assert ka.startswith("w0-n12-")


def test_table_roundtrip(tmp_path):
    path = str(tmp_path / "tune.json")
    g = gg.rmat(12, 8, seed=1)
    calls = {"tune": 0, "set": []}

    def fake_tune(dg, specs, probe_T):
        calls["tune"] += 1
        return ({"tile_words": 2, "blocks_per_sm": 1, "chunk_arcs": 64, "pull_permille": -1, "accumulation": 4,
                 "weighted_words": 1, "weighted_short_row": 32, "weighted_kernel": 2, "block_threads": 512},
                {"candidates": 9, "probe_queries": 2, "ms_default": 10.0, "ms_best": 8.0})

    def fake_set(dg, **cfg):
        calls["set"].append(cfg)

    specs = [{"r": 3}, {"r": 4}]
    cfg, entry = tuning.tuned(FakeGraph(g), g.offsets, specs, path, 128, fake_tune, fake_set)
    assert calls["tune"] == 1 and calls["set"] == [] and cfg["tile_words"] == 2
    stored = json.load(open(path))
    assert list(stored) == [tuning.graph_key(g.n, g.offsets, False, specs)]
    assert stored[list(stored)[0]]["report"]["ms_best"] == 8.0
    g2 = gg.rmat(12, 8, seed=7)
    cfg2, _ = tuning.tuned(FakeGraph(g2), g2.offsets, [{"r": 9}, {"r": 10}], path, 128, fake_tune, fake_set)
    assert calls["tune"] == 1 and calls["set"] == [cfg2] and cfg2 == cfg
    assert set(cfg) == set(tuning.TUNED_FIELDS)
