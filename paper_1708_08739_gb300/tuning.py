"""Tuning table of the batched traversal's launch parameters.

bc_tune (the library's autotuner) times candidate configurations on a probe
of a batch and applies the fastest. This module keeps its answers in a JSON
table keyed by the statistics of a graph that decide the best launch shape,
so a graph of the same kind reuses them without timing anything:

  weighted       the weighted (Dial buckets) or unweighted (bit-mask) kernel
  log2 n         size class of the vertex set
  mean degree    m / n, rounded to a power of two
  degree skew    largest out-degree over the mean, rounded to a power of two
  query vertices distinct query vertices of the probe batch (1, or several:
                 one-vertex groups take the vertex scan)

Host logic only: the timing runs in the library.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

DEFAULT_TABLE = os.path.join(os.path.expanduser("~"), ".cache", "bcd", "tune.json")
TUNED_FIELDS = ("tile_words", "blocks_per_sm", "chunk_arcs", "pull_permille", "accumulation", "weighted_words",
                "weighted_short_row", "weighted_kernel")


def _pow2_class(x: float) -> int:
    return int(round(math.log2(x))) if x > 0 else -1


def graph_key(n: int, offsets, weighted: bool, specs=None) -> str:
    """The table key of a graph (CSR row offsets) and a kind of batch."""
    off = np.asarray(offsets, dtype=np.int64)
    m = int(off[-1])
    deg = np.diff(off)
    mean = m / max(n, 1)
    skew = (float(deg.max()) / mean) if m > 0 else 0.0
    roots = len({int(s["r"]) for s in specs}) if specs else 1
    return "w%d-n%d-d%d-s%d-q%s" % (int(bool(weighted)), _pow2_class(n), _pow2_class(mean), _pow2_class(skew),
                                     "1" if roots == 1 else "many")


def load(path: str = DEFAULT_TABLE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save(table: dict, path: str = DEFAULT_TABLE):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuned(g, offsets, specs, path: str = DEFAULT_TABLE, probe_T: int = 2048, tune_fn=None, set_fn=None):
    """Applies the table's configuration for this graph and batch kind to g,
    running the autotuner first when the table has none. Returns (config,
    entry) where entry records the probe times. The probe should span a few
    dozen tiles (probe_T draws per query): with only a handful, the one tile
    on which accumulation 4 tries the vertex scan weighs too much. tune_fn /
    set_fn default to the library's bc_tune / bc_set_config."""
    if tune_fn is None or set_fn is None:
        import paper_1708_08739_gb300 as bcd
        tune_fn = tune_fn or bcd.bc_tune
        set_fn = set_fn or bcd.bc_set_config
    key = graph_key(g.n, offsets, g.weighted, specs)
    table = load(path)
    entry = table.get(key)
    if entry is None:
        cfg, rep = tune_fn(g, specs, probe_T)
        entry = {"config": {k: int(cfg[k]) for k in TUNED_FIELDS if k in cfg}, "report": rep, "probe_T": probe_T}
        table[key] = entry
        save(table, path)
    else:
        set_fn(g, **entry["config"])
    return entry["config"], entry
