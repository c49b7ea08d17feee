"""Multi-rank host logic on CPU with gloo, world size 2.

bench.py: the step time is the max over ranks and the whole-job rate counts
each query of the one batch the ranks share once.

Source sharding (paper_1708_08739_gb300.shard): the union of a batch's
source sets is split into contiguous shards, each rank evaluates its shard
(here with the oracle as the per-rank engine: RV(r), the Philox draws and
Eq. 4 dependencies from the oracle), the per-query partials are exchanged
and summed in shard order, and the result equals the oracle's single-rank
E-BCD / A-BCD within the parity bar. Then rank 1 leaves between steps,
announcing it on the host (a file store); rank 0 takes its shard, and the
scores come out bit for bit as before.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def init(rank, world, port):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)


def timing_worker(rank, world, port, out):
    init(rank, world, port)
    import bench
    local_ms = [1000.0, 1500.0][rank]
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    out[rank] = (ms, bench.job_rate(64, ms))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest():
    port = free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(timing_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1]
    ms, qs = out[0]
    assert ms == 1500.0
    assert abs(qs - 64 / 1.5) < 1e-9


# ---------------------------------------------------------------- sharding

SPECS = [(11, None), (42, 300), (7, None), (123, 200), (42, None), (250, 150)]  # (r, T): T None = exact


def oracle_engine(g, og):
    """Per-rank engine over the union D of the batch's source sets (ascending
    ids), built from the oracle: shard k's partial score of query q is
    scale_q * sum over its sources s of mult_q(s) * delta_s.(r_q)."""
    import oracle as O
    from paper_1708_08739_gb300 import shard as sh
    mult = []
    scale = []
    union = set()
    for r, T in SPECS:
        rvl = O.rv(og, r)
        if T is None:
            m = {int(v): 1 for v in rvl.tolist()}
            sc = 1.0
        else:
            m = {}
            for t in range(T):
                v = int(rvl[O.sample_index(7, t, rvl.shape[0])])
                m[v] = m.get(v, 0) + 1
            sc = rvl.shape[0] / T
        mult.append(m)
        scale.append(sc)
        union.update(m)
    D = np.array(sorted(union), dtype=np.int32)
    qv = np.array([r for r, _ in SPECS], dtype=np.int32)

    def solve(k, nshards):
        lo, hi = sh.shard_bounds(D.shape[0], k, nshards)
        part = np.zeros(len(SPECS))
        if hi > lo:
            dep, _, _ = O.dependencies(og, D[lo:hi], qv, 1)
            for q in range(len(SPECS)):
                w = np.array([mult[q].get(int(s), 0) for s in D[lo:hi]], dtype=np.float64)
                part[q] = scale[q] * float(np.dot(w, dep[:, q]))
        return part

    return solve


def shard_worker(rank, world, port, store_path, out):
    init(rank, world, port)
    import graphgen as gg
    import oracle as O
    from paper_1708_08739_gb300 import shard as sh
    g = gg.erdos_renyi(300, 2400, 5)
    og = O.Graph.from_csr(g)
    solve = oracle_engine(g, og)
    store = dist.FileStore(store_path, world)
    nshards = world
    # step 1: both ranks
    tot = sh.run_sharded(lambda k: solve(k, nshards), nshards, rank, range(world), len(SPECS), dist)
    out["step1_%d" % rank] = tot.tolist()
    dist.barrier()
    # step 2: rank 1 leaves between steps and says so on the host
    if rank == 1:
        store.set("left/1", "1")
        out["left"] = True
        return
    store.wait(["left/1"])
    alive = [0]
    assert sh.shards_of(0, nshards, alive) == [0, 1]
    tot2 = sh.run_sharded(lambda k: solve(k, nshards), nshards, 0, alive, len(SPECS), None)
    out["step2"] = tot2.tolist()
    want = []
    for r, T in SPECS:
        want.append(O.bc_exact(og, r, 0)[0] if T is None else O.bc_approx(og, r, T, 7, 0)[0])
    out["want"] = want


def test_sharded_batch_equals_single_rank(tmp_path):
    from helpers import close
    port = free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(shard_worker, args=(2, port, str(tmp_path / "store"), out), nprocs=2, join=True)
    assert out["step1_0"] == out["step1_1"]  # every rank holds the totals
    assert out["step2"] == out["step1_0"]    # same split and order after the reassignment: bit for bit
    for got, want in zip(out["step1_0"], out["want"]):
        assert close(got, want), (got, want)
    assert any(w > 0 for w in out["want"])


def test_shard_split_and_assignment():
    from paper_1708_08739_gb300 import shard as sh
    for n in (0, 1, 5, 113, 1000):
        for ns in (1, 2, 3, 8):
            b = [sh.shard_bounds(n, k, ns) for k in range(ns)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[i][1] == b[i + 1][0] for i in range(ns - 1))
            assert all(hi - lo in (n // ns, n // ns + 1) for lo, hi in b)
    assert sh.assign_shards(4, [0, 1, 2, 3]) == {0: 0, 1: 1, 2: 2, 3: 3}
    assert sh.assign_shards(4, [0, 2]) == {0: 0, 2: 2, 1: 0, 3: 2}
    assert sh.shards_of(0, 4, [0, 2]) == [0, 1]
    with pytest.raises(ValueError):
        sh.reduce_in_shard_order({0: [1.0]}, 2, 1)


class FakeLib:
    """Stands in for the CUDA binding in bench.solve_step: shard k of a
    batch answers (k + 1) * 10^-3 * (query index + 1) for every query."""

    def bc_batch(self, dg, specs):
        raise AssertionError("a sharded step must not run the whole batch")

    def bc_batch_shard(self, dg, specs, k, n):
        out = [{"bc": (k + 1) * 1e-3 * (i + 1), "status": 0, "flags": 0, "rv_size": 1, "samples": 0}
               for i in range(len(specs))]
        return out, {"shard": k}


def step_worker(rank, world, port, out):
    init(rank, world, port)
    import bench
    tot, info, res = bench.solve_step(FakeLib(), None, [{"r": 0}, {"r": 1}, {"r": 2}], rank, world, dist)
    out[rank] = (tot.tolist(), info["shard"])
    dist.destroy_process_group()


def test_bench_step_shards_and_sums():
    """bench.solve_step under two ranks: each runs its own shard and every
    rank ends with the shard-order sums of all shards."""
    port = free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(step_worker, args=(2, port, out), nprocs=2, join=True)
    want = [(1e-3 + 2e-3) * (i + 1) for i in range(3)]
    for r in (0, 1):
        tot, shard = out[r]
        assert shard == r
        assert all(abs(a - b) <= 1e-15 for a, b in zip(tot, want)), (tot, want)
