"""Benchmark: batched sampled BC(r) on a directed R-MAT scale-22 graph.

Workload (one step): one batch of 64 A-BCD queries (Algorithm 2; eps 0.01,
delta 0.1, so T = 14,979 draws each, Philox seed 7) at 64 uniform random
vertices (seed 105) of R-MAT scale 22, edge factor 8, a/b/c/d =
0.57/0.19/0.19/0.05 (seed 22), with 30 % of the arcs also added reversed
(seed 22), self-loops and repeated arcs removed, unweighted. The metric is
BC(r) queries per second; GTEPS (sum over sources of the arcs they reach, per
second) is reported too. At one GPU the line also carries the exact batch of
64 queries on R-MAT scale 20 (edge factor 16) and a short serving run
(continuous batching with Poisson arrivals, p50/p99 latency).

Arms:
  default            the CUDA library (libbcd.so). Under torchrun the ranks
                     share the one batch: rank k runs shard k of the batch's
                     source tiles (bc_batch_shard) on its own replica of the
                     graph, and the per-query partial scores are exchanged
                     and summed in shard order (strong scaling: the total
                     work is fixed as N grows).
  --impl reference   the CPU oracle as it stands, on the host cores, on a
                     bounded sample of the same batch's sources.

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402

METRIC = "GTEPS and BC(r) queries/s (exact and sampled) vs HBM roofline; p50/p99 query latency"
WORKLOAD = "rmat22_ef8_recip30_sampled64"

# DRAM bytes per (source, reached arc) of the batched traversal kernel
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch over the edges it
# traversed), measured with ncu on a small launch of the same kernel (one
# sampled query, 512 draws, on the R-MAT scale 20 graph: --case profile) and
# scaled to the bench's launch by its edge count. The figure belongs to the
# kernel sources it was taken on: when their hash differs, traffic is null.
KERNEL_SOURCES = ["bcd_traverse.cu", "bcd_device.cuh", "bcd_common.cuh"]
TRAFFIC = {"sources_sha256": "6450effc35581c4c301354863a5199a3480ebe128e9b6da6da80517b68ed4363",
           "bytes_per_reached_arc": 6.266, "tile_words": 4}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def kernel_sha():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1708_08739_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


WORKLOADS = {
    "rmat20_ef16_exact64": "R-MAT scale 20, edge factor 16, a/b/c/d 0.57/0.19/0.19/0.05, seed 20, loops and "
                           "repeats removed, unweighted; 64 exact queries: 32 uniform (seed 103) + 32 top "
                           "in-degree x out-degree",
    "rmat22_ef8_recip30_sampled64": "R-MAT scale 22, edge factor 8, seed 22, 30% of arcs also reversed (seed 22), "
                                    "repeats removed; 64 uniform queries (seed 105), A-BCD eps 0.01 delta 0.1 "
                                    "(T = 14,979) Philox seed 7",
    "rmat20_w255_exact32": "R-MAT scale 20, edge factor 16, seed 20, loops and repeats removed, arc weights uniform "
                           "in 1..255 (uint32, seed 3); 32 exact queries, uniform (seed 104)",
}


def make_workload(name=WORKLOAD):
    """(graph, query vertices, query specs as dicts for the binding)."""
    if name == "rmat20_ef16_exact64":
        g = gg.rmat(20, 16, 0.57, 0.19, 0.19, seed=20)
        qs = [int(x) for x in gg.random_vertices(g.n, 32, 103)] + [int(x) for x in gg.top_inout_vertices(g, 32)]
        return g, qs, [{"r": r} for r in qs]
    if name == "rmat20_w255_exact32":
        g = gg.rmat(20, 16, 0.57, 0.19, 0.19, seed=20)
        g = g.with_weights(gg.uniform_weights(g.m, 1, 255, 3))
        qs = [int(x) for x in gg.random_vertices(g.n, 32, 104)]
        return g, qs, [{"r": r} for r in qs]
    if name == "rmat22_ef8_recip30_sampled64":
        g = gg.add_reciprocal(gg.rmat(22, 8, seed=22), 0.3, seed=22)
        qs = [int(x) for x in gg.random_vertices(g.n, 64, 105)]
        return g, qs, [{"r": r, "kind": 1, "eps": 0.01, "delta": 0.1, "seed": 7} for r in qs]
    raise ValueError(name)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "bcd_clocks_%d_%d.csv" % (os.getpid(), index))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def oracle_union(g, qs, specs=None):
    """The union D of the batch's source sets, by the oracle: RV(r) for
    exact queries, the Philox draws for sampled ones."""
    import oracle as O
    og = O.Graph.from_csr(g)
    union = set()
    outd = g.out_degree()
    rv_cache = {}
    for i, r in enumerate(qs):
        if outd[r] == 0:
            continue
        if r not in rv_cache:
            rv_cache[r] = O.rv(og, r)
        rvl = rv_cache[r]
        spec = specs[i] if specs else {"r": r}
        if spec.get("kind", 0) == 0:
            union.update(rvl.tolist())
        elif rvl.shape[0] > 0:
            T = O.samples_for(spec["eps"], spec["delta"])
            k = rvl.shape[0]
            union.update(int(rvl[O.sample_index(spec["seed"], t, k)]) for t in range(T))
    return og, np.array(sorted(union), dtype=np.int32)


def oracle_timed(og, D, qs, threads, budget_s, seed=7, chunk=None):
    """Times the oracle on sources of the batch drawn at random from D:
    delta_s.(r_q) for every query q, in chunks of `chunk` sources (default:
    one per thread) until budget_s seconds have passed. Returns (seconds,
    sources timed)."""
    import oracle as O
    rng = np.random.default_rng(seed)
    order = rng.permutation(D.shape[0])
    chunk = chunk or threads
    qv = np.array(qs, dtype=np.int32)
    done, t0 = 0, time.time()
    while done < D.shape[0] and (time.time() - t0 < budget_s or done == 0):
        srcs = np.sort(D[order[done:done + chunk]])
        O.dependencies(og, srcs, qv, nthreads=threads)
        done += srcs.shape[0]
    return time.time() - t0, done


def max_over_ranks(value, dist=None, device="cuda"):
    """The largest value over all ranks (the job's step time); the value
    itself when not distributed."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, dist=None, device="cuda"):
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units, ms):
    """Whole-job throughput: the job's units (each query of the shared batch
    once) per second of the slowest rank."""
    return units / (ms / 1000.0)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import build as ob
    ob.build()
    g, qs, specs = make_workload(args.workload)
    threads = os.cpu_count() or 1
    og, D = oracle_union(g, qs, specs)
    nd = int(D.shape[0])
    times = []
    per_step = []
    for i in range(args.warmup + args.steps):
        el, ns = oracle_timed(og, D, qs, threads, args.ref_step_s, seed=i)
        if i >= args.warmup:
            times.append(el / ns)
            per_step.append(ns)
    t_src = sum(times) / len(times)
    qps = len(qs) / (t_src * nd)
    line = {"impl": "reference", "metric": METRIC, "value": qps, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * len(qs) / qps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "queries": len(qs), "sources_in_union": nd},
            "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": threads, "kind": "oracle",
                             "sample": "per step, random union sources in chunks of %d until %.0f s (%d..%d "
                                       "sources), delta for all %d queries; queries/s = %d / (seconds per source "
                                       "x union size %d)" % (threads, args.ref_step_s, min(per_step),
                                                             max(per_step), len(qs), len(qs), nd)},
            "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def solve_step(bcd, dg, specs, rank, world, dist):
    """One step: this rank's shard of the batch, then the exchange of the
    per-query partial scores (summed in shard order). Returns (scores, info
    of this rank's launch, results of this rank)."""
    from paper_1708_08739_gb300 import shard as sh
    if world == 1:
        out, info = bcd.bc_batch(dg, specs)
        return np.array([o["bc"] for o in out]), info, out
    box = {}

    def solve(k):
        out, info = bcd.bc_batch_shard(dg, specs, k, world)
        box["info"], box["out"] = info, out
        return [o["bc"] for o in out]

    tot = sh.run_sharded(solve, world, rank, range(world), len(specs), dist)
    return tot, box["info"], box["out"]


def algorithmic_bytes(info, weighted=False):
    """The traversal's algorithmic bytes (see the design notes): graph
    structure 2 (8 |V_B| + 4 |E_B|) summed over tiles (8 bytes per arc with
    its weight); the forward pass, 24 bytes per reached (source, vertex) pair
    (level and sigma written and read back; 32 with 8-byte distances) and 8
    per tight (source, arc) pair (sigma of the tail); the Eq. 4 backward, on
    the tiles that ran it, 16 more per reached pair (delta written and read)
    and 16 per tight pair (sigma and delta of the head); the vertex scan, 16
    per term (sigma_st and sigma_rt)."""
    arc = 8.0 if weighted else 4.0
    pair = 32.0 if weighted else 24.0
    return (2.0 * (8.0 * info["union_vertices"] + arc * info["union_arcs"]) + pair * info["reached_pairs"] +
            8.0 * info["tight_pairs"] + 16.0 * info["eq4_reached_pairs"] + 16.0 * info["eq4_tight_pairs"] +
            16.0 * info["scan_pairs"])


def run_gpu(args):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    import paper_1708_08739_gb300 as bcd

    t0 = time.time()
    g, qs, specs = make_workload(args.workload)
    log("workload built in %.1fs: n=%d m=%d" % (time.time() - t0, g.n, g.m))
    # the oracle's CPU baseline runs on the host cores meanwhile (one core is
    # left to the thread that drives the GPU), on rank 0 at N = 1 only
    cpu_box = {}
    cpu_thread = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import threading

        def cpu_job():
            threads = max(1, (os.cpu_count() or 2) - 1)
            og, D = oracle_union(g, qs, specs)
            el, ns = oracle_timed(og, D, qs, threads, args.cpu_budget_s)
            el1, ns1 = oracle_timed(og, D, qs, 1, args.cpu_budget_s / 3.0, seed=8, chunk=1)
            cpu_box.update(el=el, ns=ns, el1=el1, ns1=ns1, nd=int(D.shape[0]), threads=threads)

        cpu_thread = threading.Thread(target=cpu_job, daemon=True)
        cpu_thread.start()
    stream = torch.cuda.Stream()
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols, g.weights, stream=stream.cuda_stream)
    if g.weights is None:
        bcd.bc_set_config(dg, tile_words=args.tile_words)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    for i in range(args.warmup):
        t = time.time()
        solve_step(bcd, dg, specs, rank, world, dist)
        log("warmup %d: %.2fs" % (i, time.time() - t))
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos = []
    for i in range(args.steps):
        scores, info, out = solve_step(bcd, dg, specs, rank, world, dist)
        infos.append(info)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dist if world > 1 else None)
    nq = len(qs)
    qps = job_rate(nq, ms)
    edges = float(np.mean([i["edges_traversed"] for i in infos]))
    gteps = sum_over_ranks(edges, dist if world > 1 else None) / (ms / 1000.0) / 1e9
    trav_ms = float(np.mean([i["ms_traversal"] for i in infos]))
    launches = int(sum(i["launches"] for i in infos) / args.steps)
    algo_bytes = float(np.mean([algorithmic_bytes(i, g.weights is not None) for i in infos]))
    peak, peak_kind = peaks()
    achieved = algo_bytes / (trav_ms / 1000.0) / 1e9
    traffic = None
    if (TRAFFIC["bytes_per_reached_arc"] and TRAFFIC["sources_sha256"] == kernel_sha() and
            args.tile_words == TRAFFIC["tile_words"] and g.weights is None):
        traffic = TRAFFIC["bytes_per_reached_arc"] * edges

    # end to end through the C ABI: pinned host CSR in, results out
    off_h = torch.from_numpy(g.offsets).pin_memory()
    col_h = torch.from_numpy(g.cols).pin_memory()
    w_h = None if g.weights is None else torch.from_numpy(g.weights.view(np.int32)).pin_memory()
    barrier()
    t = time.time()
    ge = bcd.bc_graph_create(g.n, off_h.numpy(), col_h.numpy(), None if w_h is None else w_h.numpy().view(np.uint32),
                             stream=stream.cuda_stream)
    if g.weights is None:
        bcd.bc_set_config(ge, tile_words=args.tile_words)
    scores_e, _, _ = solve_step(bcd, ge, specs, rank, world, dist)
    ge.close()
    barrier()
    e2e_s = max_over_ranks(time.time() - t, dist if world > 1 else None)
    h2d = g.offsets.nbytes + g.cols.nbytes + (0 if g.weights is None else g.weights.nbytes) + nq * 40
    d2h = nq * 32

    extras = {}
    if world == 1 and not args.no_extras:
        extras = run_extras(args, bcd, dg, g, stream)
    cpu = None
    if cpu_thread is not None:
        cpu_thread.join()
        t_src = cpu_box["el"] / cpu_box["ns"]
        t_src1 = cpu_box["el1"] / cpu_box["ns1"]
        nd = cpu_box["nd"]
        cpu = {"value": nq / (t_src * nd), "unit": "queries/s", "cores": cpu_box["threads"], "kind": "oracle",
               "sample": "%d random sources of the %d in the batch's union (chunks of one source per thread for "
                         "%.0f s), delta for all %d queries; queries/s = %d / (seconds per source x union size)"
                         % (cpu_box["ns"], nd, args.cpu_budget_s, nq, nq),
               "single_thread": {"value": nq / (t_src1 * nd), "unit": "queries/s", "cores": 1,
                                 "sample": "%d sources one at a time" % cpu_box["ns1"]}}
    if rank == 0:
        line = {
            "metric": METRIC, "value": qps, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "recipe": WORKLOADS[args.workload],
                       "n": g.n, "m": g.m, "queries": nq,
                       "tile_words": args.tile_words, "sources_in_union": int(infos[-1]["sources_run"]) * world,
                       "l2": "not flushed: working set (sigma and accumulator slabs, graph, level history) well above L2",
                       "parallelism": "sources sharded: rank k runs shard k of each group's tiles, per-query "
                                      "partials summed in shard order" if world > 1 else "one GPU"},
            "gteps": gteps,
            "phases_ms": {"rv": float(np.mean([i["ms_rv"] for i in infos])),
                          "sample": float(np.mean([i["ms_sample"] for i in infos])),
                          "traversal": trav_ms,
                          "forward": float(np.mean([i["ms_forward"] for i in infos])),
                          "backward": float(np.mean([i["ms_backward"] for i in infos]))},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": ("wtrav_kernel (weighted batched SPD + dependencies)" if g.weights is not None
                                    else "trav_kernel (batched SPD + dependency traversal)"),
                         "algorithmic_bytes": algo_bytes},
            "e2e": {"value": job_rate(nq, 1000.0 * e2e_s), "unit": "queries/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk,
            "cpu_baseline": cpu,
            "check": {"bc_first": float(scores[0]),
                      "e2e_equal": all(abs(a - b) <= 1e-9 * abs(b) or a == b == 0.0 for a, b in zip(scores_e, scores))},
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    dg.close()
    if world > 1:
        dist.destroy_process_group()


def run_extras(args, bcd, dg22, g22, stream):
    """Extra keys of the one-GPU line: the exact R-MAT 20 batch and a sampled
    batch on the weighted R-MAT 20 (one warm and one timed call each), and a
    short serving run on the resident R-MAT 22 graph."""
    import torch
    out = {}
    g, qs, specs = make_workload("rmat20_ef16_exact64")
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols, stream=stream.cuda_stream)
    bcd.bc_set_config(dg, tile_words=args.tile_words)
    bcd.bc_batch(dg, specs)
    torch.cuda.synchronize()
    t = time.time()
    res, info = bcd.bc_batch(dg, specs)
    wall = time.time() - t
    ab = algorithmic_bytes(info)
    peak, _ = peaks()
    out["rmat20_ef16_exact64"] = {
        "recipe": WORKLOADS["rmat20_ef16_exact64"], "queries_per_s": len(qs) / wall, "s_per_batch": wall,
        "gteps": info["edges_traversed"] / wall / 1e9, "sources_in_union": info["sources_run"],
        "ms_traversal": info["ms_traversal"], "algorithmic_gbs": ab / (info["ms_traversal"] / 1000.0) / 1e9,
        "frac": ab / (info["ms_traversal"] / 1000.0) / 1e9 / peak, "bc_first": res[0]["bc"]}
    dg.close()
    # the weighted graph of rmat20_w255_exact32 with its 32 query vertices
    # sampled (A-BCD eps 0.05, delta 0.1: T = 600), on the weighted source kernel
    g, qs, _ = make_workload("rmat20_w255_exact32")
    specs = [{"r": r, "kind": 1, "eps": 0.05, "delta": 0.1, "seed": 7} for r in qs]
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols, g.weights, stream=stream.cuda_stream)
    bcd.bc_batch(dg, specs)
    torch.cuda.synchronize()
    t = time.time()
    res, info = bcd.bc_batch(dg, specs)
    wall = time.time() - t
    out["rmat20_w255_sampled32"] = {
        "recipe": WORKLOADS["rmat20_w255_exact32"].replace("32 exact queries", "32 queries, A-BCD eps 0.05 delta 0.1 "
                                                            "(T = 600) Philox seed 7"),
        "queries_per_s": len(qs) / wall, "s_per_batch": wall, "gteps": info["edges_traversed"] / wall / 1e9,
        "sources_in_union": info["sources_run"], "ms_traversal": info["ms_traversal"],
        "weighted_kernel": bcd.bc_get_config(dg)["weighted_kernel"], "bc_first": res[0]["bc"]}
    dg.close()
    if args.serve_extra > 0:
        specs_s, draws, rvs = serve_workload(bcd, dg22, g22, args.serve_extra, args.serve_rv_max)
        srv = bcd.Server(dg22)
        serve_run(bcd, srv, specs_s[: max(4, len(specs_s) // 8)])  # warm-up
        wall, lat = serve_run(bcd, srv, specs_s)
        sat = len(specs_s) / wall
        w2, l2 = serve_run(bcd, srv, specs_s, rate=0.8 * sat, seed=80)
        srv.close()
        t = time.time()
        for s in specs_s[:32]:
            bcd.bc_batch(dg22, [s])
        one = 32 / (time.time() - t)
        out["serving"] = {
            "workload": "R-MAT 22 + 30%% reciprocal resident; %d Zipf(1.1) queries alternating exact (|RV| <= %d) "
                        "and sampled (eps 0.02, delta 0.1, seed 7)" % (len(specs_s), args.serve_rv_max),
            "closed_loop": {"queries_per_s": sat, "p50_ms": float(np.percentile(lat, 50)),
                            "p99_ms": float(np.percentile(lat, 99))},
            "poisson_0.8x": {"arrival_rate": 0.8 * sat, "queries_per_s": len(specs_s) / w2,
                             "p50_ms": float(np.percentile(l2, 50)), "p99_ms": float(np.percentile(l2, 99))},
            "one_at_a_time_queries_per_s": one}
    return out


def serve_workload(bcd, dg, g, nq, rv_max, seed=106):
    """Zipf(1.1) query vertices over permuted ids, alternately exact and
    sampled (eps 0.02, delta 0.1, Philox seed 7). Exact queries are re-drawn
    until 1 <= |RV(r)| <= rv_max; sampled ones until |RV(r)| >= 1 (on this
    graph |RV| is either tiny or the whole giant in-component, which only
    sampling serves)."""
    # host-side screen of the synthetic workload: a vertex with no in-arc has
    # |RV| = 0, and one reachable from the hub (the vertex of largest in x out
    # degree) has every vertex that reaches the hub in its RV; only the others
    # need an RV traversal to learn their size
    import scipy.sparse as sp
    from scipy.sparse.csgraph import breadth_first_order
    hub = int(gg.top_inout_vertices(g, 1)[0])
    adj = sp.csr_matrix((np.ones(g.m, dtype=np.int8), g.cols, g.offsets), shape=(g.n, g.n))
    behind_hub = np.zeros(g.n, dtype=bool)
    behind_hub[breadth_first_order(adj, hub, directed=True, return_predecessors=False)] = True
    hub_rv = bcd.bc_rv_compute(dg, hub).shape[0]
    indeg = np.bincount(g.cols, minlength=g.n)
    sizes = {}
    out = []
    draws = 0
    rnd = 0
    while len(out) < nq and rnd < 256:
        cand = gg.zipf_vertices(g.n, 4 * nq, 1.1, seed + rnd)
        rnd += 1
        for r in cand.tolist():
            draws += 1
            if r not in sizes:
                if g.offsets[r + 1] == g.offsets[r] or indeg[r] == 0:
                    sizes[r] = 0  # out-degree 0 (BC = 0, Prop. 1) or RV empty
                elif behind_hub[r] and r != hub and hub_rv + 1 > rv_max:
                    sizes[r] = -1  # |RV| > rv_max: the hub and all that reach it are in RV
                else:
                    sizes[r] = bcd.bc_rv_compute(dg, r).shape[0]
            exact = len(out) % 2 == 0
            if (exact and 1 <= sizes[r] <= rv_max) or (not exact and (sizes[r] >= 1 or sizes[r] == -1)):
                out.append(r)
                if len(out) == nq:
                    break
    for r in set(out):
        if sizes[r] == -1:
            sizes[r] = bcd.bc_rv_compute(dg, r).shape[0]
    specs = []
    for i, r in enumerate(out):
        if i % 2 == 0:
            specs.append({"r": r, "kind": bcd.BC_QUERY_EXACT})
        else:
            specs.append({"r": r, "kind": bcd.BC_QUERY_APPROX, "eps": 0.02, "delta": 0.1, "seed": 7})
    return specs, draws, [sizes[r] for r in out]


def serve_run(bcd, srv, specs, rate=None, seed=11):
    """Submits every query (all at once, or with Poisson gaps of mean
    1/rate), waits for all; returns (wall seconds, latencies ms)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=len(specs)) if rate else np.zeros(len(specs))
    tickets = []
    t0 = time.time()
    next_t = t0
    pending = {}
    lat = []
    for s, gap in zip(specs, gaps):
        next_t += gap
        while time.time() < next_t:
            for t in list(pending):
                r = srv.poll(t)
                if r is not None:
                    lat.append(r[1])
                    del pending[t]
            time.sleep(0.0005)
        t = srv.submit(s)
        pending[t] = True
    while pending:
        for t in list(pending):
            r = srv.poll(t, timeout_us=2000)
            if r is not None:
                lat.append(r[1])
                del pending[t]
    return time.time() - t0, lat


def run_serve(args):
    """Serving: continuous batching under Poisson arrivals, p50/p99 (the
    serving shape: R-MAT 22 + 30 % reciprocal resident, Zipf(1.1) query
    vertices alternating exact and sampled; a closed loop first, then one
    wave of Poisson arrivals per rate, each a fraction of the closed-loop
    rate; one query at a time through bc_batch on the first
    args.serve_single queries)."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1708_08739_gb300 as bcd
    t0 = time.time()
    g = gg.add_reciprocal(gg.rmat(22, 8, seed=22), 0.3, seed=22)
    log("serve graph: n=%d m=%d in %.1fs" % (g.n, g.m, time.time() - t0))
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols)
    bcd.bc_set_config(dg, tile_words=args.tile_words)
    specs, draws, rvs = serve_workload(bcd, dg, g, args.serve_queries, args.serve_rv_max)
    log("serve queries: %d (from %d draws), |RV| %d..%d" % (len(specs), draws, min(rvs), max(rvs)))
    srv = bcd.Server(dg)
    serve_run(bcd, srv, specs[: max(4, min(512, len(specs) // 8))])  # warm-up
    clk = ClockSampler(0)
    clk.start()
    wall, lat = serve_run(bcd, srv, specs)
    sat = len(specs) / wall
    log("closed loop: %.1f queries/s" % sat)
    runs = {"closed_loop": {"queries_per_s": sat, "p50_ms": float(np.percentile(lat, 50)),
                            "p99_ms": float(np.percentile(lat, 99)), "wall_s": wall}}
    for f in [float(x) for x in args.serve_rates.split(",") if x]:
        w, l = serve_run(bcd, srv, specs, rate=f * sat, seed=int(100 * f))
        runs["poisson_%.1fx" % f] = {"arrival_rate": f * sat, "queries_per_s": len(specs) / w,
                                      "p50_ms": float(np.percentile(l, 50)), "p99_ms": float(np.percentile(l, 99)),
                                      "wall_s": w}
        log("poisson %.1fx: p50 %.0f ms p99 %.0f ms" % (f, runs["poisson_%.1fx" % f]["p50_ms"],
                                                      runs["poisson_%.1fx" % f]["p99_ms"]))
    clocks = clk.stop()
    st = srv.stats()
    srv.close()
    # one query at a time, the first queries of the same list
    sub = specs[: args.serve_single]
    lat1 = []
    t = time.time()
    for s1 in sub:
        t1 = time.perf_counter()
        bcd.bc_batch(dg, [s1])
        lat1.append(1000.0 * (time.perf_counter() - t1))
    single = len(sub) / (time.time() - t)
    line = {"metric": METRIC, "value": sat, "unit": "queries/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": 1000.0 * wall, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "serve_rmat22_recip30_zipf", "n": g.n, "m": g.m, "queries": len(specs),
                       "zipf_draws": draws,
                       "rv_exact_range": [min(rvs[0::2]), max(rvs[0::2])],
                       "rv_sampled_range": [min(rvs[1::2]), max(rvs[1::2])] if len(rvs) > 1 else None,
                       "mix": "alternate exact (|RV| <= %d) / sampled eps 0.02 delta 0.1 seed 7" % args.serve_rv_max},
            "serving": runs,
            "one_at_a_time": {"queries": len(sub), "queries_per_s": single, "p50_ms": float(np.percentile(lat1, 50)),
                              "p99_ms": float(np.percentile(lat1, 99))},
            "server_stats": st, "clocks": clocks}
    print(json.dumps(line), flush=True)
    dg.close()


def run_error_vs_exact(args):
    """The sampled batch against the exact scores of its query vertices: the
    64 uniform queries of the R-MAT 22 workload, A-BCD (eps 0.01, delta 0.1,
    Philox seed 7) and E-BCD in one bc_batch each, and per query the paper's
    error 100 |App - BC| / BC (Section 5), with the distribution over the
    queries whose exact score is not 0."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1708_08739_gb300 as bcd
    g, qs, specs = make_workload("rmat22_ef8_recip30_sampled64")
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols)
    t = time.time()
    app, ai = bcd.bc_batch(dg, specs)
    t_app = time.time() - t
    t = time.time()
    ex, ei = bcd.bc_batch(dg, [{"r": r} for r in qs])
    t_ex = time.time() - t
    rows = []
    for r, a, e in zip(qs, app, ex):
        err = None if e["bc"] == 0.0 else 100.0 * abs(a["bc"] - e["bc"]) / e["bc"]
        rows.append({"r": r, "rv_size": e["rv_size"], "exact": e["bc"], "sampled": a["bc"], "error_pct": err})
    errs = sorted(x["error_pct"] for x in rows if x["error_pct"] is not None)
    print(json.dumps({"experiment": "error_vs_exact", "workload": "rmat22_ef8_recip30_sampled64",
                      "sampled_s": t_app, "exact_s": t_ex, "exact_sources": ei["sources_run"],
                      "exact_tiles": ei["tiles"], "exact_scan_tiles": ei["scan_tiles"],
                      "queries_nonzero": len(errs), "queries_zero_both": sum(1 for x in rows if x["exact"] == 0.0 and
                                                                             x["sampled"] == 0.0),
                      "error_pct": {"mean": float(np.mean(errs)) if errs else None,
                                    "median": float(np.median(errs)) if errs else None,
                                    "p90": float(np.percentile(errs, 90)) if errs else None,
                                    "max": errs[-1] if errs else None},
                      "rows": rows}), flush=True)
    dg.close()


def run_profile_case(args):
    """A small launch of the same traversal kernel for ncu captures, on the
    R-MAT 20 graph: one sampled query (T = args.case_T draws, seed 7) at the
    vertex of largest in-degree x out-degree, or with --case-queries k > 1,
    k uniform queries from the giant component (seed 103) with T = args.case_T
    / k draws each (seeds 7, 8, ...), as in the bench's batch of many query
    vertices. --accumulation picks the backward (default 1: Eq. 4)."""
    import __graft_entry__
    __graft_entry__.build()
    import paper_1708_08739_gb300 as bcd
    g, qs, _ = make_workload("rmat20_ef16_exact64")
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols)
    bcd.bc_set_config(dg, tile_words=args.tile_words, accumulation=args.accumulation or 1)
    if args.case_queries <= 1:
        r = int(gg.top_inout_vertices(g, 1)[0])
        specs = [{"r": r, "kind": bcd.BC_QUERY_APPROX_T, "T": args.case_T, "seed": 7}]
    else:
        pick = []
        for r in qs[:32]:
            if g.out_degree()[r] > 0 and r not in pick and bcd.bc_rv_compute(dg, r).shape[0] > 1000:
                pick.append(r)
            if len(pick) == args.case_queries:
                break
        specs = [{"r": r, "kind": bcd.BC_QUERY_APPROX_T, "T": args.case_T // len(pick), "seed": 7 + i}
                 for i, r in enumerate(pick)]
    out, info = bcd.bc_batch(dg, specs)
    print(json.dumps({"case": "profile", "queries": [s["r"] for s in specs], "T": [s["T"] for s in specs],
                      "bc": [o["bc"] for o in out], "accumulation": bcd.bc_get_config(dg)["accumulation"],
                      "info": info}), flush=True)
    dg.close()


def run_wprofile_case(args):
    """A small launch of the weighted traversal kernel for ncu captures: one
    sampled query (T = args.case_T draws, seed 7) on the vertex of largest
    in-degree x out-degree of R-MAT scale args.case_scale (edge factor 16,
    seed 20) with weights uniform in [1, 255] (seed 3); the Eq. 4 backward, or
    the vertex scan with --accumulation 2."""
    import __graft_entry__
    __graft_entry__.build()
    import paper_1708_08739_gb300 as bcd
    g = gg.rmat(args.case_scale, 16, 0.57, 0.19, 0.19, seed=20)
    g = g.with_weights(gg.uniform_weights(g.m, 1, 255, 3))
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols, g.weights)
    bcd.bc_set_config(dg, weighted_words=args.weighted_words, accumulation=args.accumulation or 1,
                      weighted_kernel=args.weighted_kernel)
    r = int(gg.top_inout_vertices(g, 1)[0])
    out, info = bcd.bc_batch(dg, [{"r": r, "kind": bcd.BC_QUERY_APPROX_T, "T": args.case_T, "seed": 7}])
    print(json.dumps({"case": "wprofile", "scale": args.case_scale, "r": r, "T": args.case_T, "bc": out[0]["bc"],
                      "config": bcd.bc_get_config(dg), "info": info}), flush=True)
    dg.close()


def run_single(args):
    """Single-query latency, one query per bc_batch call, under both
    accumulations: 1 (the backward pass of Eq. 4, pushed along tight in-arcs)
    and 2 (the vertex scan after a traversal from r). Queries: A-BCD with
    eps 0.01, delta 0.1 (T = 14,979, seed 7) on the R-MAT 20 vertex of largest
    in-degree x out-degree and on the first uniform query (seed 105) of the
    R-MAT 22 graph with 30 % reciprocal arcs whose |RV| exceeds 1000. One
    warm-up call, then args.single_reps timed calls per accumulation (wall
    clock around the synchronous call; CUDA-event phase times from the batch
    report). Prints one JSON line per (graph, accumulation)."""
    import __graft_entry__
    __graft_entry__.build()
    import torch
    import paper_1708_08739_gb300 as bcd
    cases = []
    g20, _, _ = make_workload("rmat20_ef16_exact64")
    cases.append(("rmat20_ef16", g20, int(gg.top_inout_vertices(g20, 1)[0])))
    g22, qs22, _ = make_workload("rmat22_ef8_recip30_sampled64")
    cases.append(("rmat22_ef8_recip30", g22, None))
    for name, g, r in cases:
        dg = bcd.bc_graph_create(g.n, g.offsets, g.cols)
        bcd.bc_set_config(dg, tile_words=args.tile_words)
        if r is None:
            r = next(q for q in qs22 if bcd.bc_rv_compute(dg, q).shape[0] > 1000)
        spec = {"r": r, "kind": bcd.BC_QUERY_APPROX, "eps": 0.01, "delta": 0.1, "seed": 7}
        for acc in (1, 2):
            bcd.bc_set_config(dg, accumulation=acc)
            out, _ = bcd.bc_batch(dg, [spec])
            torch.cuda.synchronize()
            clk = ClockSampler(torch.cuda.current_device())
            clk.start()
            walls, infos = [], []
            for _ in range(args.single_reps):
                t = time.perf_counter()
                out, info = bcd.bc_batch(dg, [spec])
                walls.append(1000.0 * (time.perf_counter() - t))
                infos.append(info)
            clocks = clk.stop()
            med = float(np.median(walls))
            keys = ("ms_total", "ms_rv", "ms_sample", "ms_spd", "ms_traversal", "ms_root", "ms_forward",
                    "ms_backward")
            phases = {k: float(np.median([i[k] for i in infos])) for k in keys}
            line = {"case": "single", "graph": name, "r": r, "T": out[0]["samples"], "rv_size": out[0]["rv_size"],
                    "accumulation": acc, "bc": out[0]["bc"], "ms_per_query_median": med,
                    "ms_per_query_min": min(walls), "queries_per_s": 1000.0 / med, "reps": len(walls),
                    "phases_ms_median": phases, "sources_run": infos[-1]["sources_run"],
                    "tiles": infos[-1]["tiles"], "scan_pairs": infos[-1]["scan_pairs"],
                    "reached_pairs": infos[-1]["reached_pairs"], "tight_pairs": infos[-1]["tight_pairs"],
                    "clocks": clocks}
            print(json.dumps(line), flush=True)
        dg.close()


def run_set_experiment(args):
    """The set experiment of Section 5 (Table 6) on the R-MAT 20 graph: for
    random sets of 5, 10 and 15 vertices, BCD with tau = 1000 (HYBRID: exact
    when |RV(r)| <= 1000, else 1000 draws, seed 7) as one batch; errors
    against the exact scores (exact path, one batch over all set vertices),
    the batch's time and its RV time, |RV| statistics, and the same set run
    one query at a time."""
    import __graft_entry__
    __graft_entry__.build()
    import torch
    import paper_1708_08739_gb300 as bcd
    g, _, _ = make_workload("rmat20_ef16_exact64")
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols)
    bcd.bc_set_config(dg, tile_words=args.tile_words)
    sets = {k: [int(x) for x in gg.random_vertices(g.n, k, 200 + k)] for k in (5, 10, 15)}
    every = list(dict.fromkeys(v for vs in sets.values() for v in vs))
    t = time.time()
    ex, exi = bcd.bc_batch(dg, [{"r": r} for r in every])
    t_exact = time.time() - t
    exact = {r: o["bc"] for r, o in zip(every, ex)}
    log("set experiment: exact scores of %d vertices in %.1f s" % (len(every), t_exact))
    tau = 1000
    rows = []
    for k, vs in sets.items():
        specs = [{"r": r, "kind": bcd.BC_QUERY_HYBRID, "T": tau, "seed": 7} for r in vs]
        bcd.bc_batch(dg, specs)  # warm
        torch.cuda.synchronize()
        t = time.time()
        out, info = bcd.bc_batch(dg, specs)
        t_set = time.time() - t
        t = time.time()
        for sp in specs:
            bcd.bc_batch(dg, [sp])
        t_one = time.time() - t
        err = []
        for r, o in zip(vs, out):
            e = exact[r]
            err.append(0.0 if e == o["bc"] else 100.0 * abs(o["bc"] - e) / abs(e))
        rv = [o["rv_size"] for o in out]
        rows.append({"set_size": k, "error_pct": {"avg": sum(err) / k, "max": max(err), "min": min(err)},
                     "time_s": t_set, "time_rv_s": info["ms_rv"] / 1000.0,
                     "rv_size": {"avg": sum(rv) / k, "max": max(rv), "min": min(rv)},
                     "exact_queries": sum(1 for x in rv if x <= tau), "sources_run": info["sources_run"],
                     "one_at_a_time_s": t_one})
    print(json.dumps({"experiment": "set", "graph": WORKLOADS["rmat20_ef16_exact64"].split(";")[0], "tau": tau,
                      "exact_reference_s": t_exact, "rows": rows}), flush=True)
    dg.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--tile-words", type=int, default=4, help="64-source mask words per tile (1, 2, 4 or 8)")
    ap.add_argument("--cpu-budget-s", type=float, default=24.0,
                    help="seconds of oracle work for the all-core CPU baseline (a third of it single-threaded)")
    ap.add_argument("--ref-step-s", type=float, default=5.0, help="--impl reference: seconds of oracle work per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the R-MAT 20 exact batch and the serving run")
    ap.add_argument("--serve-extra", type=int, default=512, help="queries of the serving run among the extras")
    ap.add_argument("--case", default="", choices=["", "profile", "wprofile"],
                    help="profile / wprofile: one small sampled batch on the unweighted / weighted R-MAT (for ncu), "
                         "no JSON bench line")
    ap.add_argument("--case-scale", type=int, default=20, help="R-MAT scale of the wprofile case")
    ap.add_argument("--weighted-words", type=int, default=0, help="weighted tile width (64-source words; 0: default)")
    ap.add_argument("--weighted-kernel", type=int, default=0, choices=[0, 1, 2],
                    help="wprofile case: 1 the weighted tile kernel, 2 the source kernel (0: the library default, 2)")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--case-T", type=int, default=512)
    ap.add_argument("--case-queries", type=int, default=1, help="profile case: query vertices (1: the top vertex)")
    ap.add_argument("--serve", action="store_true", help="serving benchmark (continuous batching, p50/p99)")
    ap.add_argument("--set-experiment", action="store_true",
                    help="the set experiment of Section 5 (sets of 5, 10, 15 vertices, tau = 1000)")
    ap.add_argument("--single", action="store_true",
                    help="single-query latency under both accumulations (Eq. 4 push, vertex scan)")
    ap.add_argument("--single-reps", type=int, default=5)
    ap.add_argument("--error-vs-exact", action="store_true",
                    help="the R-MAT 22 sampled batch against the exact scores of its 64 query vertices")
    ap.add_argument("--accumulation", type=int, default=0, choices=[0, 1, 2, 3, 4],
                    help="profile / wprofile cases: 1 Eq. 4 backward (their default), 2 vertex scan, 3 scan over "
                         "several vertices, 4 chosen per group")
    ap.add_argument("--serve-queries", type=int, default=10000)
    ap.add_argument("--serve-rates", default="0.5,0.8,1.0", help="Poisson arrival rates as fractions of saturation")
    ap.add_argument("--serve-single", type=int, default=256, help="queries run one at a time for the comparison")
    ap.add_argument("--serve-rv-max", type=int, default=100000)
    args = ap.parse_args()
    if args.warmup < 3:
        log("warm-up raised to 3 steps")
        args.warmup = 3
    if args.serve:
        run_serve(args)
    elif args.error_vs_exact:
        run_error_vs_exact(args)
    elif args.single:
        run_single(args)
    elif args.set_experiment:
        run_set_experiment(args)
    elif args.case == "profile":
        run_profile_case(args)
    elif args.case == "wprofile":
        run_wprofile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
