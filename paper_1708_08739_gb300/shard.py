"""Source sharding of one batch over several GPUs, one process per GPU.

The sources of a batch are independent terms of the sums of Algorithm 1 and
Algorithm 2 (and of the set version of Section 4.2): BC(r) is a sum over the
sources in RV(r) of delta_s.(r), and A-BCD's estimate a sum over its draws.
So a batch splits into `nshards` contiguous shards of its tiles (in the
library's tile order, bc_batch_shard), each run on one GPU against its own
replica of the graph; the only exchange is one fp64 partial score per query
and shard, summed on the host in shard order.

If a rank leaves between steps (it announces this on the host, for example
in the process group's key-value store), its shards go to the ranks that
remain: the number of shards, the split and the order of the final sum do
not change, so the scores are the same as before, bit for bit.

Host logic only: no device code and no arithmetic of the method.
"""
from __future__ import annotations

import numpy as np


def shard_bounds(nunits: int, k: int, nshards: int):
    """Units [lo, hi) of shard k of nshards contiguous shards: the split of
    bc_batch_shard (lo = nunits * k // nshards)."""
    if not (0 <= k < nshards):
        raise ValueError("need 0 <= k < nshards")
    return nunits * k // nshards, nunits * (k + 1) // nshards


def assign_shards(nshards: int, alive):
    """Shard -> rank that runs it: shard k goes to rank k while that rank is
    alive, else to the live ranks in turn."""
    alive = sorted(set(int(r) for r in alive))
    if not alive:
        raise ValueError("no live rank")
    out = {}
    spare = [k for k in range(nshards) if k not in alive]
    for k in range(nshards):
        if k in alive:
            out[k] = k
    for i, k in enumerate(spare):
        out[k] = alive[i % len(alive)]
    return out


def shards_of(rank: int, nshards: int, alive):
    """The shards this rank runs, ascending."""
    return sorted(k for k, r in assign_shards(nshards, alive).items() if r == rank)


def reduce_in_shard_order(parts: dict, nshards: int, nq: int) -> np.ndarray:
    """Per-query sums of the shards' partial scores, added in shard order
    0, 1, ..., nshards - 1 (every shard must be present)."""
    missing = [k for k in range(nshards) if k not in parts]
    if missing:
        raise ValueError("shards without a result: %s" % missing)
    total = np.zeros(nq, dtype=np.float64)
    for k in range(nshards):
        total += np.asarray(parts[k], dtype=np.float64)
    return total


def gather_parts(local: dict, dist=None):
    """All ranks' {shard: partial scores}, merged (every rank receives it).
    Without a process group the local dict is the whole."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return dict(local)
    got = [None] * dist.get_world_size()
    dist.all_gather_object(got, {int(k): np.asarray(v, dtype=np.float64).tolist() for k, v in local.items()})
    merged = {}
    for d in got:
        for k, v in d.items():
            if k in merged:
                raise ValueError("shard %d run twice" % k)
            merged[k] = np.asarray(v, dtype=np.float64)
    return merged


def run_sharded(solve_shard, nshards: int, rank: int, alive, nq: int, dist=None):
    """Runs this rank's shards with solve_shard(k) -> partial scores [nq],
    exchanges the partials and returns the per-query totals (on every rank
    taking part in the exchange)."""
    local = {k: np.asarray(solve_shard(k), dtype=np.float64) for k in shards_of(rank, nshards, alive)}
    return reduce_in_shard_order(gather_parts(local, dist), nshards, nq)
