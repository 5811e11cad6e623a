#!/usr/bin/env python
"""Benchmark of the GB300 Cluster-BFS hot path.

Workload (one step): batched C-BFS of 256 star clusters (1-64 sources each,
seeded random centres and neighbour subsets, d = 2) on an undirected R-MAT
scale-22 graph (edge factor 16, a = 0.57, b = c = 0.19), then the vertex-major
label append of those 256 clusters and one 65,536-pair distance query.
Inputs are device-resident when the timed region starts; the CSR (0.5 GB)
and the outputs (18 GB) are far larger than L2, so no flush is needed.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
(Algorithm 1, sequential C, one cluster per host core) on a bounded sample of
the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2410_17226_gb300 import inputs as I  # noqa: E402

METRIC = "C-BFS source-edge GTEPS + HBM roofline fraction; label-query p50/p99 latency"
def workload_text(scale: int, clusters: int) -> str:
    return (f"batched C-BFS: undirected R-MAT scale {scale} (edge factor 16, a=0.57 b=c=0.19, int32 CSR), "
            f"{clusters} star clusters of 1-64 sources (seeded random centres + random neighbour subsets), d=2, "
            "autotuned push/pull; + label append + 65,536-pair query")
ARC_BYTES = 13      # per arc scanned: 4 B neighbour id + 1 B Delta_v check + 8 B subset OR
VERTEX_BYTES = 41   # per frontier appearance: 8 B offsets + 33 B vertex-phase reads/writes


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cbfs", "reference"], default="cbfs")
    ap.add_argument("--scale", type=int, default=22)
    ap.add_argument("--clusters", type=int, default=256)
    ap.add_argument("--query-batch", type=int, default=65536)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--latency-requests", type=int, default=200)
    ap.add_argument("--serve-s", type=float, default=2.0, help="seconds per offered serving load (0: skip)")
    ap.add_argument("--no-single-compare", dest="single_compare", action="store_false",
                    help="skip timing the clusters one call each")
    ap.add_argument("--fixed-tune", default="", help="'alpha,slots[,small_deg,mid_deg]' instead of the autotuner (profiling runs)")
    ap.add_argument("--no-next", dest="next_rows", action="store_false",
                    help="skip the single-source BFS comparison and the d sweep")
    ap.add_argument("--no-configs", dest="configs", action="store_false",
                    help="skip timing the single-cluster (scale 14) and label-construction (scale 24) workloads")
    ap.add_argument("--record-traffic", default="",
                    help="comma-separated ncu CSVs (dram__bytes_read/write.sum of the traversal kernels of one "
                         "`runcli --host-loop` call) to turn into profiles/traffic.json for the current kernel "
                         "sources, then exit")
    ap.add_argument("--traffic-run", default="", help="the runcli output line of the captured call")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(rank: int) -> int:
    """Cluster seed of a rank: weak scaling gives every rank its own 256 clusters."""
    return I.MASTER_SEED + 1 + 1000 * rank


def max_over_ranks(x: float, pg, device) -> float:
    """The slowest rank's time (the job's time): all-reduce MAX; x itself at N = 1."""
    if pg is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: int, ranks: int, t_max_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time, in G/s."""
    return units_per_rank * ranks / (t_max_ms / 1e3) / 1e9


def bench_config(scale: int, C: int, d: int, n: int, nnz: int, sources: int, query_batch: int) -> dict:
    """The workload's description, the same in both arms' lines."""
    return {"workload": workload_text(scale, C), "graph": f"rmat-s{scale}-ef16", "n": int(n), "nnz": int(nnz),
            "clusters": int(C), "sources": int(sources), "d": int(d), "query_batch": int(query_batch),
            "l2": "inputs larger than L2 (0.5 GB CSR, 18 GB outputs, 18 GB labels)"}


def workload(scale: int, C: int, rank: int):
    off, adj = I.rmat(scale)
    clusters, d = I.star_clusters(off, adj, C, seed=rank_seed(rank), size="uniform")
    return off, adj, clusters, d


# ------------------------------------------------------------ CPU oracle leg

_CPU_G = None  # (off, adj) inherited by forked workers


def _oracle_one(args):
    import oracle

    S, d = args
    off, adj = _CPU_G
    t0 = time.perf_counter()
    _, _, cnt = oracle.cbfs_alg1(off, adj, S, d, with_counters=True)
    return len(S) * cnt["reached_arcs"] // 2, time.perf_counter() - t0


def cpu_oracle_sample(off, adj, clusters, d, budget_s: float):
    """Times the oracle on the host cores (one cluster per worker) until the
    budget is used; returns (GTEPS, cores, clusters done, wall seconds)."""
    global _CPU_G
    import oracle

    oracle.build()
    _CPU_G = (off, adj)
    cores = len(os.sched_getaffinity(0))
    workers = max(1, min(cores, 64))
    ctx = mp.get_context("fork")  # forked before any CUDA call in this process
    done, edges, t0 = 0, 0, time.perf_counter()
    with ctx.Pool(workers) as pool:
        while done < len(clusters) and time.perf_counter() - t0 < budget_s:
            batch = [(clusters[i], d) for i in range(done, min(len(clusters), done + workers))]
            for e, _ in pool.map(_oracle_one, batch, chunksize=1):
                edges += e
            done += len(batch)
    wall = time.perf_counter() - t0
    _CPU_G = None
    return edges / wall / 1e9, workers, done, wall


# ------------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for nm, val in zip(names, p[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- helpers


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the CUDA sources' code: comments and whitespace are left out,
    so that a traffic record stays valid across comment-only edits."""
    import re

    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2410_17226_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, fn), encoding="utf-8") as f:
                text = f.read()
            # string literals kept whole, comments dropped, whitespace runs folded
            code = re.sub(r'("(?:\\.|[^"\\])*")|/\*.*?\*/|//[^\n]*',
                          lambda m: m.group(1) or " ", text, flags=re.S)
            h.update(fn.encode())
            h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, alg_bytes: int):
    """DRAM bytes of a launch of `alg_bytes` algorithmic bytes, from the
    committed ncu record (physical bytes per algorithmic byte of a captured
    wave), or None when the kernels changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    e = t.get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash() or "dram_bytes_per_alg_byte" not in e:
        return None
    return int(e["dram_bytes_per_alg_byte"] * alg_bytes)


# ------------------------------------------------- single-source BFS and d


def timed_ms(fn, reps: int = 3) -> float:
    """Median wall time of fn() (each call synchronises its stream)."""
    import torch

    fn()
    out = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        out.append((time.perf_counter() - t0) * 1e3)
    return statistics.median(out)


def comparison_clusters(off, adj, seed: int, count: int = 10):
    """The microbenchmark clusters of Section 5.1: a vertex and up to 63 of
    its neighbours (d = 2)."""
    return I.star_clusters(off, adj, count, seed=seed, size="max", min_deg=63)


def seq_bfs_sample(off, adj, seed: int, sample: int = 8):
    """Plain sequential BFS (the paper's "Seq-BFS" baseline) on one host core:
    the oracle's BFS from a sample of the comparison clusters' sources, in ms
    per 64 sources.  Part of the CPU baseline; runs before CUDA starts."""
    import oracle

    oracle.build()
    clusters, _ = comparison_clusters(off, adj, seed)
    t0 = time.perf_counter()
    done = 0
    for S in clusters[:2]:
        for s in S[:sample // 2]:
            oracle.bfs(off, adj, int(s))
            done += 1
    ms = (time.perf_counter() - t0) * 1e3 / max(done, 1) * 64
    return {"ms_per_64_sources": round(ms, 1), "cores": 1, "kind": "oracle",
            "sample": f"{done} plain BFSs (oracle) from the comparison clusters' sources, scaled to 64"}


def bfs_comparison(g, off, adj, seed: int, seq=None):
    """The paper's microbenchmark framing (Section 5.1) on this GPU: C-BFS of
    a 64-vertex star cluster (d = 2) against the plain BFSs of its sources,
    both through the same kernels (a BFS is C-BFS with k = 1, d = 0,
    direction-optimising as in Algorithm "EdgeMap")."""
    clusters, d = comparison_clusters(off, adj, seed)
    deg = np.diff(off)
    cb_ms, bfs_ms, bfs8_ms = [], [], []
    for S in clusters:
        singles = [np.array([s], np.int32) for s in S]
        cb_ms.append(timed_ms(lambda: g.run_batched([S], d, tune={"slots": 1})))
        # separate BFSs: one source per slot word (packing would make them one C-BFS)
        bfs_ms.append(timed_ms(lambda: g.run_batched(singles, 0, tune={"slots": 1, "pack": -1})))
        bfs8_ms.append(timed_ms(lambda: g.run_batched(singles, 0, tune={"slots": 8, "pack": -1})))
    # undirected edges of the reached component (the same for every source of a cluster)
    hd, _ = g.run([int(clusters[0][0])], 0)
    comp_edges = int(deg[hd.cpu().numpy() != 255].sum()) // 2
    cb, bf, b8 = statistics.mean(cb_ms), statistics.mean(bfs_ms), statistics.mean(bfs8_ms)
    k = statistics.mean(len(S) for S in clusters)
    out = {"clusters": len(clusters), "mean_sources": round(k, 1), "d": d,
           "cbfs_ms_per_cluster": round(cb, 3),
           "bfs_all_k_sources_ms_one_per_wave": round(bf, 3),
           "bfs_all_k_sources_ms_eight_per_wave": round(b8, 3),
           "bit_level_gain": round(bf / cb, 2),
           "bfs_gteps_one_per_wave": round(k * comp_edges / (bf / 1e3) / 1e9, 3),
           "cbfs_gteps": round(k * comp_edges / (cb / 1e3) / 1e9, 3)}
    if seq:
        out["speedup_over_seq_bfs"] = round(seq["ms_per_64_sources"] * k / 64 / cb, 1)
    return out


def d_sweep(cbfs, g, off, adj, seed: int, per_d: int = 8, ds=(2, 3, 4, 5, 6), min_deg: int = 1):
    """C-BFS cost against the diameter bound d (Theorem 1: work grows with d):
    per d, clusters of 64 vertices within d of each other by construction
    (``inputs.radius_cluster`` around random centres, hop counts from this
    library's own BFS), each run alone and batched.  The exact diameters,
    decoded from the outputs, are reported beside d.  (On a power-law graph
    hubs keep every cluster's spread small, so the cost hardly moves; the
    road grid shows the growth.)"""
    import torch

    deg = np.diff(off)
    cand = np.flatnonzero(deg >= max(min_deg, 1))
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {}
    for d in ds:
        clusters = []
        for _ in range(50 * per_d):
            if len(clusters) == per_d:
                break
            ctr = int(cand[rng.integers(0, cand.size)])
            hd, _ = g.run([ctr], 0)
            hops = hd.cpu().numpy().astype(np.int64)
            hops[hops == 255] = -1
            S = I.radius_cluster(hops, ctr, d, k=64, seed=int(rng.integers(1 << 62)))
            if S.size >= 2:  # small balls (a grid at small d) give fewer than 64
                clusters.append(S)
        ks = [int(S.size) for S in clusters]
        alone = statistics.mean(timed_ms(lambda: g.run_batched([S], d, tune={"slots": 1})) for S in clusters)
        dist, masks = g.run_batched(clusters, d, tune={"slots": 4})
        batched = timed_ms(lambda: g.run_batched(clusters, d, dist, masks, tune={"slots": 4}))
        st = g.output_stats(dist, masks, ks, d)
        # exact diameters: delta_j(S[i]) = Delta + offset of bit j at vertex S[i]
        diam = []
        dist_h = dist.cpu().numpy()
        masks_h = masks.cpu().numpy().view(np.uint64)
        for c, S in enumerate(clusters):
            best = 0
            for v in S:
                seen = np.uint64(0)
                for t in range(d):
                    m = masks_h[c, t, v]
                    if m & ~seen:
                        best = max(best, int(dist_h[c, v]) + t)
                    seen |= m
                if seen != np.uint64((1 << ks[c]) - 1):
                    best = max(best, int(dist_h[c, v]) + d)
            diam.append(best)
        out[str(d)] = {"mean_sources": round(statistics.mean(ks), 1),
                       "ms_per_cluster_alone": round(alone, 3), "ms_per_cluster_batched": round(batched / len(clusters), 3),
                       "arcs_scanned_per_cluster": int(st[:, 1].mean()), "rounds": int(st[:, 3].max()),
                       "exact_diameters": sorted(set(diam))}
        del dist, masks
        torch.cuda.empty_cache()
    return {"clusters_per_d": per_d, "sizes": 64, "by_d": out}


def ll_quality(cbfs, g, off, adj, seed: int, budget: int = 1024, n_src: int = 32, pairs_per_src: int = 3125,
               local_pairs: int = 20000):
    """Landmark-labeling index quality against word size (Section 5.3,
    table "ApproxLL" on this synthetic graph): plain landmarks and clusters of
    w = 8, 16, 32, 64 (d = 2) under one budget of bytes per vertex; index
    time, label bytes, distortion epsilon over 100,000 pairs of the largest
    component and query time.  Exact distances come from this library's BFS
    (k = 1, d = 0) from each pair's first vertex."""
    import torch

    from paper_2410_17226_gb300 import ll

    n = off.size - 1
    deg = np.diff(off)
    hub = int(np.argmax(deg))
    comp_d, _ = g.run([hub], 0)
    comp = np.flatnonzero(comp_d.cpu().numpy() != 255)
    rng = np.random.Generator(np.random.PCG64(seed))
    us = comp[rng.integers(0, comp.size, n_src)].astype(np.int32)
    tru, _ = g.run_batched([np.array([u], np.int32) for u in us], 0, tune={"slots": 8})
    tru = tru.cpu().numpy()
    vs = comp[rng.integers(0, comp.size, (n_src, pairs_per_src))]
    pairs = np.stack([np.repeat(us, pairs_per_src), vs.reshape(-1)], axis=1).astype(np.int32)
    exact = tru[np.repeat(np.arange(n_src), pairs_per_src), vs.reshape(-1)].astype(np.int64)
    exact[exact == 255] = -1
    pairs_dev = torch.from_numpy(pairs).cuda()
    out = {}
    for name, w in (("plain", 1), ("w8", 8), ("w16", 16), ("w32", 32), ("w64", 64)):
        clusters, d = ll.select(off, adj, budget, w=w)
        L, build_ms = ll.build(g, clusters, d, w)
        ans = L.query(pairs_dev)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        L.query(pairs_dev, out=ans)
        e1.record()
        torch.cuda.synchronize()
        q_ms = e0.elapsed_time(e1)
        dd = ll.distortion(cbfs.as_numpy_u16(ans), exact)
        out[name] = {"clusters": len(clusters), "landmarks": int(sum(len(S) for S in clusters)), "d": d,
                     "row_bytes_per_vertex": cbfs.Labels.bytes_per_vertex(len(clusters), d, max(w, 8) if d else 64),
                     "index_ms": round(build_ms, 2), "epsilon_pct": round(100 * dd["epsilon"], 3),
                     "exact_share": round(dd["exact_share"], 4), "unanswered": dd["unanswered"],
                     "query_ns_per_pair": round(q_ms * 1e6 / len(pairs), 2)}
        if name == "w64":
            # the bounded bidirectional search fused into the query (Appendix B), on a sample
            m = min(len(pairs), local_pairs)
            sub = pairs_dev[:m].contiguous()
            local = {}
            for tau in (128, 512, 2048):
                la = g.query_local(sub, tau, labels=L)
                torch.cuda.synchronize()
                e0.record()
                g.query_local(sub, tau, labels=L, out=la)
                e1.record()
                torch.cuda.synchronize()
                dl = ll.distortion(cbfs.as_numpy_u16(la), exact[:m])
                base = ll.distortion(cbfs.as_numpy_u16(ans[:m]), exact[:m])
                local[str(tau)] = {"epsilon_pct": round(100 * dl["epsilon"], 3),
                                   "epsilon_pct_labels_only": round(100 * base["epsilon"], 3),
                                   "exact_share": round(dl["exact_share"], 4),
                                   "query_ns_per_pair": round(e0.elapsed_time(e1) * 1e6 / m, 1)}
            out[name]["local_search"] = {"pairs": m, "by_tau": local}
        L.close()
        torch.cuda.empty_cache()
    return {"budget_bytes_per_vertex": budget, "pairs": int(len(pairs)), "sources_of_pairs": n_src,
            "pairs_from": "the component of the highest-degree vertex", "by_index": out}


def road_grid_throughput(cbfs, seed: int, side: int = 4096, count: int = 64, per_launch: int = 16):
    """The high-diameter road-like workload (4096 x 4096 grid, 10 % of edges
    deleted, 1 % shortcuts; 64 BFS-ball clusters of 64 sources, d = their
    largest exact diameter), timed in launches of `per_launch` clusters:
    source-edge GTEPS and the algorithmic-byte rate beside the HBM peak."""
    import torch

    from paper_2410_17226_gb300 import tune

    off, adj = I.road_grid(side, seed=I.MASTER_SEED + 2)
    clusters, ds = I.ball_clusters(off, adj, count, 64, seed=seed)
    d = max(ds)
    deg = np.diff(off)
    with cbfs.Graph(off, adj) as g:
        n = g.n
        # this graph's own switch factor, clusters per wave and degree classes
        tn = tune.autotune(g, clusters, d, sample=per_launch, key_extra=f"grid-{side}-{tune.signature(off)}")
        tset = {k: tn.get(k, 0) for k in ("pull_alpha", "slots", "small_deg", "mid_deg", "fused_pull")}
        dist = torch.empty((per_launch, n), dtype=torch.uint8, device="cuda")
        masks = torch.empty((per_launch, d, n), dtype=torch.int64, device="cuda")
        total_ms, A, V, src_edges, rounds = 0.0, 0, 0, 0, 0
        lock = {"waves": 0, "words": 0, "wave_rounds": 0, "word_rounds": 0, "cluster_rounds": 0}
        for b in range(0, count, per_launch):
            part = clusters[b:b + per_launch]
            k = len(part)
            run = lambda: g.run_batched(part, d, dist[:k], masks[:k], tune=tset)  # noqa: E731
            total_ms += timed_ms(run, reps=2)
            st = g.output_stats(dist[:k], masks[:k], [len(S) for S in part], d)
            A += int(st[:, 1].sum())
            V += int(st[:, 0].sum())
            rounds = max(rounds, int(st[:, 3].max()))
            ls = lockstep_rounds([len(S) for S in part], st[:, 3], tset["slots"])
            for key in lock:
                lock[key] += ls[key]
            reached = dist[:k].cpu().numpy() != 255
            for c, S in enumerate(part):
                src_edges += len(S) * int(deg[reached[c]].sum()) // 2
        alg = ARC_BYTES * A + VERTEX_BYTES * V + count * n * (1 + 8 * d)
        del dist, masks
        torch.cuda.empty_cache()
    peak, _ = measured_peak_hbm()
    return {"graph": f"road grid {side}x{side}, 10% deleted, 1% shortcuts", "n": int(n), "nnz": int(adj.size),
            "clusters": count, "d": d, "per_launch": per_launch, "tune": dict(tset, cached=tn.get("cached")),
            "ms_all_clusters": round(total_ms, 2),
            "gteps": round(src_edges / (total_ms / 1e3) / 1e9, 2), "max_rounds": rounds,
            "lockstep": dict(lock, busy_slot_round_share=round(
                lock["word_rounds"] / max(lock["wave_rounds"] * max(int(tset["slots"]), 1), 1), 4)),
            "arcs_per_s": round(A / (total_ms / 1e3), 1),
            "alg_gbs": round(alg / (total_ms / 1e3) / 1e9, 1), "alg_frac": round(alg / (total_ms / 1e3) / 1e9 / peak, 4)}


def single_cluster_config(cbfs, reps: int = 20):
    """Single C-BFS, plain form: R-MAT scale 14, clusters of a seeded random
    vertex and up to 63 of its neighbours, d = 2 (the state fits L2: time and
    GTEPS, no HBM roofline).  Ten seeded clusters with uniform random centres
    (most centres have few neighbours, so k is small) and ten whose centres
    have degree >= 63 (k = 64); per cluster the device time of a call
    (stream-ordered calls back to back, CUDA events) and the host latency of
    a blocking call."""
    import torch

    off, adj = I.rmat(14)
    deg = np.diff(off)
    out = {"graph": "R-MAT scale 14", "d": 2}
    with cbfs.Graph(off, adj) as g:
        dist = torch.empty(g.n, dtype=torch.uint8, device="cuda")
        masks = torch.empty((2, g.n), dtype=torch.int64, device="cuda")
        stream = torch.cuda.current_stream()
        for name, kw in (("random_centres", {}), ("centres_deg_ge_63", {"min_deg": 63})):
            clusters, d = I.star_clusters(off, adj, 10, seed=I.MASTER_SEED, size="max", **kw)
            edges = 0
            for S in clusters:  # warm-up (records each call shape's graph) and the reached edges
                g.run(S, d, dist, masks)
                edges += len(S) * int(deg[dist.cpu().numpy() != 255].sum()) // 2
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                for S in clusters:
                    g.run(S, d, dist, masks, check=False)
            e1.record(stream)
            torch.cuda.synchronize()
            if cbfs.sync_status(stream) != cbfs.OK:
                raise RuntimeError("single-cluster calls reported an error")
            dev_ms = e0.elapsed_time(e1) / (reps * len(clusters))
            lat = []
            for _ in range(3):
                for S in clusters:
                    t0 = time.perf_counter()
                    g.run(S, d, dist, masks)  # blocking: waits for the stream and checks the status
                    lat.append((time.perf_counter() - t0) * 1e3)
            out[name] = {"clusters": len(clusters), "mean_sources": round(statistics.mean(len(S) for S in clusters), 1),
                         "ms_per_call_device": round(dev_ms, 4), "ms_per_call_host_p50": round(statistics.median(lat), 4),
                         "gteps": round(edges / len(clusters) / (dev_ms / 1e3) / 1e9, 2)}
    return out


def label_construction_config(cbfs, budget_bytes_per_vertex: int = 1024, count: int = 1024, per_launch: int = 32):
    """Label construction at scale: R-MAT scale 24 (int64 offsets), 1024
    degree-ordered clusters of 64 (Section 4.2 selection), 32 per launch, the
    labels that fit 1024 B/vertex kept on the device (the rest computed and
    dropped).  Reports the traversal rate over all 1024 clusters: source-edge
    GTEPS, arcs scanned per second (Sigma A / t) and the algorithmic-byte
    rate, from CUDA events around each launch."""
    import torch

    t_gen = time.perf_counter()
    off, adj = I.rmat(24)
    clusters, d = I.degree_clusters(off, adj, count)
    gen_s = time.perf_counter() - t_gen
    deg = np.diff(off)
    with cbfs.Graph(off, adj) as g:
        n = g.n
        cap = budget_bytes_per_vertex * n // (n * (1 + 8 * d))
        L = cbfs.Labels(n, int(cap), d, budget_bytes=budget_bytes_per_vertex * n)
        dist = torch.empty((per_launch, n), dtype=torch.uint8, device="cuda")
        masks = torch.empty((per_launch, d, n), dtype=torch.int64, device="cuda")
        g.run_batched(clusters[:per_launch], d, dist, masks)  # warm-up
        stream = torch.cuda.current_stream()
        kept, A, V, trav_ms = 0, 0, 0, 0.0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for b in range(0, len(clusters), per_launch):
            part = clusters[b:b + per_launch]
            k = len(part)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.run_batched(part, d, dist[:k], masks[:k], check=False)
            e1.record(stream)
            take = min(k, int(cap) - kept)
            if take > 0:
                L.append(dist[:take], masks[:take], [len(S) for S in part[:take]])
                kept += take
            e1.synchronize()
            trav_ms += e0.elapsed_time(e1)
            st = g.output_stats(dist[:k], masks[:k], [len(S) for S in part], d)  # untimed: outside the events
            A += int(st[:, 1].sum())
            V += int(st[:, 0].sum())
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        if cbfs.sync_status(stream) != cbfs.OK:
            raise RuntimeError("label construction reported an error")
        reached = dist[0].cpu().numpy() != 255  # the degree clusters all sit in the giant component
        comp_edges = int(deg[reached].sum()) // 2
        src_edges = sum(len(S) for S in clusters) * comp_edges
        del dist, masks, L
        torch.cuda.empty_cache()
    alg = ARC_BYTES * A + VERTEX_BYTES * V + len(clusters) * n * (1 + 8 * d)
    peak, _ = measured_peak_hbm()
    return {"graph": "R-MAT scale 24 (int64 offsets)", "n": int(n), "nnz": int(adj.size), "clusters": len(clusters),
            "per_launch": per_launch, "labels_kept": int(kept), "label_budget_bytes_per_vertex": budget_bytes_per_vertex,
            "ms_all_clusters": round(ms, 1), "traversal_ms": round(trav_ms, 1),
            "gteps": round(src_edges / (trav_ms / 1e3) / 1e9, 1),
            "arcs_per_s": round(A / (trav_ms / 1e3), 1), "alg_gbs": round(alg / (trav_ms / 1e3) / 1e9, 1),
            "alg_frac": round(alg / (trav_ms / 1e3) / 1e9 / peak, 4), "graph_generation_s": round(gen_s, 1)}


# ---------------------------------------------------------------- arms


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    off, adj, clusters, d = workload(args.scale, args.clusters, 0)
    per_step = []
    edges_total, wall_total = 0, 0.0
    cores = 0
    for k in range(args.warmup + args.steps):
        sample = clusters[(k * 16) % len(clusters):][:16]
        g, cores, done, wall = cpu_oracle_sample(off, adj, sample, d, budget_s=args.cpu_budget_s)
        if k >= args.warmup:
            per_step.append(wall)
            edges_total += g * wall * 1e9
            wall_total += wall
    value = edges_total / wall_total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GTEPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * wall_total / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": bench_config(args.scale, len(clusters), d, off.size - 1, adj.size, sum(len(S) for S in clusters),
                               args.query_batch),
        "cpu_baseline": {"value": round(value, 4), "unit": "GTEPS", "cores": cores, "kind": "oracle",
                         "sample": f"each step: 16 of the {len(clusters)} clusters, Algorithm 1 in plain C, "
                                   "one cluster per core"},
        "e2e": {"value": round(value, 4), "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_cbfs(args, ws, rank, local):
    off, adj, clusters, d = workload(args.scale, args.clusters, rank)
    C = len(clusters)
    ks = np.array([len(S) for S in clusters], dtype=np.int32)
    pairs = I.random_pairs(off.size - 1, args.query_batch, seed=rank_seed(rank) + 7)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        g_cpu, cores, done, wall = cpu_oracle_sample(off, adj, clusters, d, budget_s=args.cpu_budget_s)
        cpu = {"value": round(g_cpu, 4), "unit": "GTEPS", "cores": cores, "kind": "oracle",
               "sample": f"{done} of the {C} clusters ({wall:.1f} s wall), Algorithm 1 in plain C, "
                         f"one cluster per host core"}
        if args.next_rows:
            cpu["seq_bfs"] = seq_bfs_sample(off, adj, seed=rank_seed(rank) + 21)

    import torch

    from paper_2410_17226_gb300 import build as B
    from paper_2410_17226_gb300 import cbfs, tune

    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist_

        dist_.init_process_group("nccl")
        pg = dist_

    def barrier():
        if pg:
            pg.barrier()

    n = off.size - 1
    # page-locked host buffers of the end-to-end measurement (cudaHostAlloc),
    # taken first, while the process's host memory is fresh
    e2e_host = None
    if args.e2e_steps > 0:
        off_pin = cbfs.pinned_empty(off.shape, torch.int64)
        off_pin.copy_(torch.from_numpy(off))
        adj_pin = cbfs.pinned_empty(adj.shape, torch.int32)
        adj_pin.copy_(torch.from_numpy(adj))
        # the 18 GB host-output variant only at N = 1 (N ranks on one node would pin N times that)
        outs = (cbfs.pinned_empty((C, n), torch.uint8), cbfs.pinned_empty((C, d, n), torch.int64)) if ws == 1 \
            else (None, None)
        e2e_host = (off_pin, adj_pin) + outs
    g = cbfs.Graph(off, adj, validate=True)
    if args.fixed_tune:
        parts = args.fixed_tune.split(",")
        tn = {"pull_alpha": float(parts[0]), "slots": int(parts[1]), "cached": None,
              "small_deg": int(parts[2]) if len(parts) > 2 else 0, "mid_deg": int(parts[3]) if len(parts) > 3 else 0}
    else:
        tn = tune.autotune(g, clusters, d, key_extra=f"rmat-s{args.scale}-{tune.signature(off)}")
    tset = {"pull_alpha": tn["pull_alpha"], "slots": tn["slots"], "small_deg": tn.get("small_deg", 0),
            "mid_deg": tn.get("mid_deg", 0), "fused_pull": tn.get("fused_pull", 0)}
    dist = torch.empty((C, n), dtype=torch.uint8, device=dev)
    masks = torch.empty((C, d, n), dtype=torch.int64, device=dev)
    L = cbfs.Labels(n, C, d)
    pairs_dev = torch.from_numpy(pairs).to(dev)
    answers = torch.empty(args.query_batch, dtype=torch.int16, device=dev)
    stream = torch.cuda.current_stream()

    src_cat = np.concatenate(clusters).astype(np.int32)
    coff = np.concatenate([[0], np.cumsum(ks)]).astype(np.int32)

    def step(ev=None):
        # stream-ordered: the step enqueues its work; errors are read once after the timed region
        g.run_batched(None, d, dist, masks, tune=tset, sources_concat=src_cat, cluster_off=coff, check=False)
        if ev is not None:
            ev.record(stream)
        L.reset()
        L.append(dist, masks, ks)
        L.query(pairs_dev, out=answers)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    g.profile(False)  # reset the counters; the timed steps run as CUDA graphs
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    marks = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t_start.record(stream)
        for k in range(args.steps):
            marks[k][0].record(stream)
            step(marks[k][1])
        t_end.record(stream)
        torch.cuda.synchronize()
    barrier()
    st_rc = cbfs.sync_status(stream)
    if st_rc != cbfs.OK:
        raise cbfs.CbfsError(st_rc, "timed steps")
    prof = g.profile(False)  # launch counts of the timed steps
    t_ms = t_start.elapsed_time(t_end)
    cbfs_ms = sum(a.elapsed_time(b) for a, b in marks)
    t_max = max_over_ranks(t_ms, pg, dev)

    st = g.output_stats(dist, masks, ks, d)
    V, A, R = int(st[:, 0].sum()), int(st[:, 1].sum()), st[:, 2]
    lockstep = lockstep_rounds(ks, st[:, 3], tset["slots"])
    src_edges = int(sum(int(k) * int(r) // 2 for k, r in zip(ks, R)))
    value = job_value(src_edges * args.steps, ws, t_max)
    alg_bytes_step = ARC_BYTES * A + VERTEX_BYTES * V + C * n * (1 + 8 * d)
    peak, peak_kind = measured_peak_hbm()
    # the dominant launch: one batched traversal (a CUDA graph holding every
    # traversal kernel of the call), timed by events around it in every step
    cbfs_step_ms = cbfs_ms / args.steps
    achieved = alg_bytes_step / (cbfs_step_ms / 1e3) / 1e9
    traffic = ncu_traffic("traversal", alg_bytes_step)
    roofline = {"kernel": f"cbfs_run_batched traversal graph (vertex + edge phases of all {C} clusters)",
                "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "peak_kind": peak_kind,
                "avg_launch_ms": round(cbfs_step_ms, 3), "alg_bytes_per_launch": int(alg_bytes_step),
                # Sigma A_c / t: arcs scanned in the push model (Theorem 1) per second, all clusters
                "arcs_per_s": round(A / (cbfs_step_ms / 1e3), 1)}
    if traffic:
        # the physical side: ncu DRAM bytes of the same launch over the same time
        roofline["physical_gbs"] = round(traffic / (cbfs_step_ms / 1e3) / 1e9, 1)
        roofline["physical_frac"] = round(traffic / (cbfs_step_ms / 1e3) / 1e9 / peak, 4)
    # per-kernel split from one extra, untimed traversal with event brackets (host-driven rounds)
    g.profile(True)
    g.run_batched(None, d, dist, masks, tune=dict(tset, host_loop=1), sources_concat=src_cat, cluster_off=coff)
    torch.cuda.synchronize()
    split = g.profile(False)
    e_ms, e_n = split["edge_phase"]["ms"], max(split["edge_phase"]["launches"], 1)
    roofline["edge_phase"] = {"kernel": "k_phase_b", "avg_launch_ms": round(e_ms / e_n, 4),
                              "alg_bytes_per_launch": int(ARC_BYTES * A / e_n),
                              "achieved": round(ARC_BYTES * A / (e_ms / 1e3) / 1e9, 1),
                              "share_of_traversal": round(e_ms / max(sum(split[k]["ms"] for k in
                                                                        ("setup", "vertex_phase", "edge_phase")), 1e-9), 3)}

    # the same 256 clusters as 256 separate one-cluster calls (cbfs_run) on the same GPU
    one = None
    if args.single_compare:
        d1 = torch.empty(n, dtype=torch.uint8, device=dev)
        m1 = torch.empty((d, n), dtype=torch.int64, device=dev)
        for S in clusters:  # warm: every cluster size's graph captured
            g.run(S, d, d1, m1)
        for S in clusters:
            g.run(S, d, d1, m1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for S in clusters:
            g.run(S, d, d1, m1)
        e1.record(stream)
        torch.cuda.synchronize()
        one_ms = e0.elapsed_time(e1)
        one = {"ms_for_all_clusters": round(one_ms, 3), "gteps": round(src_edges / (one_ms / 1e3) / 1e9, 3),
               "batched_speedup": round(one_ms / cbfs_step_ms, 3),
               "mode": "cbfs_run per cluster (its own waves of one slot), same clusters, same GPU"}
        del d1, m1

    # label-query latency: single requests of U{1..65536} pairs, H2D + kernel + D2H each
    lat = []
    rng = np.random.default_rng(rank_seed(rank) + 11)
    pin_pairs = cbfs.pinned_empty(pairs.shape, torch.int32)
    pin_pairs.copy_(torch.from_numpy(pairs))
    pin_ans = cbfs.pinned_empty(args.query_batch, torch.int16)
    qtot, t_q0 = 0, time.perf_counter()
    for _ in range(args.latency_requests):
        q = int(rng.integers(1, args.query_batch + 1))
        t0 = time.perf_counter()
        pairs_dev[:q].copy_(pin_pairs[:q], non_blocking=True)
        L.query(pairs_dev[:q], out=answers[:q])
        pin_ans[:q].copy_(answers[:q], non_blocking=True)
        torch.cuda.synchronize()
        lat.append((time.perf_counter() - t0) * 1e3)
        qtot += q
    q_wall = time.perf_counter() - t_q0
    query = {"p50_ms": round(float(np.percentile(lat, 50)), 4), "p99_ms": round(float(np.percentile(lat, 99)), 4),
             "qps": round(qtot / q_wall, 1), "requests": len(lat), "clusters": C,
             "mode": "one request at a time, sizes U{1..65536}, pinned H2D + kernel + D2H"}
    # the query kernel alone on a full batch: its algorithmic bytes are the
    # pairs, the answers and both label rows, q * (8 + 2 + 2 * C * (1 + 8 d))
    pairs_dev.copy_(pin_pairs)
    reps = 20
    L.query(pairs_dev, out=answers)
    torch.cuda.synchronize()
    qe0, qe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    qe0.record(stream)
    for _ in range(reps):
        L.query(pairs_dev, out=answers, stream=stream)
    qe1.record(stream)
    torch.cuda.synchronize()
    q_ms = qe0.elapsed_time(qe1) / reps
    q_alg = args.query_batch * (8 + 2 + 2 * C * (1 + 8 * d))
    query["kernel"] = {"pairs": args.query_batch, "avg_launch_ms": round(q_ms, 4),
                       "alg_bytes_per_launch": int(q_alg), "achieved_gbs": round(q_alg / (q_ms / 1e3) / 1e9, 1),
                       "peak_gbs": peak, "frac": round(q_alg / (q_ms / 1e3) / 1e9 / peak, 4),
                       "note": "random rows of 4.4 KB (256 clusters x 17 B): the label store (18 GB) exceeds L2"}

    # serving (continuous batching) over labels of 60 degree-ordered clusters of the same graph
    serving = None
    if args.serve_s > 0:
        from paper_2410_17226_gb300.serve import QueryServer, RequestPool, poisson_load

        lab_clusters, _ = I.degree_clusters(off, adj, 60)
        ld, lm = g.run_batched(lab_clusters, d, tune=tset)
        L60 = cbfs.Labels(n, len(lab_clusters), d)
        L60.append(ld, lm, [len(S) for S in lab_clusters])
        del ld, lm
        torch.cuda.synchronize()
        serve_batch = 4 * args.query_batch  # one launch may pack several requests
        sopt = {"pause_gc": True, "switch_interval_s": 1e-4}
        with QueryServer(L60, max_batch=serve_batch, slots=4, **sopt) as srv:
            # saturation: the same request mix (sizes uniform in 1..65536) offered as fast as possible
            rng = np.random.default_rng(rank_seed(rank) + 13)
            pool = RequestPool(n, args.query_batch, seed=rank_seed(rank) + 13, pinned=True)
            sizes = rng.integers(1, args.query_batch + 1, size=3000)
            starts = rng.integers(0, 3 * args.query_batch + 1, size=3000)
            for i in range(50):
                pool.submit(srv, int(starts[i]), int(sizes[i]))
            t0 = time.perf_counter()
            futs = [pool.submit(srv, int(starts[i]), int(sizes[i])) for i in range(50, 3000)]
            for f in futs:
                f.result()
            sat_qps = float(sizes[50:].sum()) / (time.perf_counter() - t0)
        loads = {}
        mean_req = (args.query_batch + 1) / 2.0
        for load in (0.5, 0.8):
            with QueryServer(L60, max_batch=serve_batch, slots=4, **sopt) as srv:
                futs, offered, elapsed = poisson_load(srv, n, rate_rps=load * sat_qps / mean_req,
                                                      duration_s=args.serve_s, max_pairs=args.query_batch,
                                                      seed=rank_seed(rank) + int(load * 100), pinned=True)
                st_ = srv.stats()
            loads[f"{load}x"] = {"p50_ms": round(st_["p50_ms"], 4), "p90_ms": round(st_["p90_ms"], 4),
                                 "p99_ms": round(st_["p99_ms"], 4), "max_ms": round(st_["max_ms"], 4),
                                 "qps": round(offered / elapsed, 1), "requests": st_["requests"],
                                 "batches": st_["batches"]}
        serving = {"labels": "60 degree-ordered clusters (Section 4.2 selection), d=2, 1020 B/vertex",
                   "server_options": sopt,
                   "arrivals": "Poisson, request sizes uniform in 1..65536 pairs, page-locked request and "
                               "answer buffers (copied by DMA)",
                   "saturation_qps": round(sat_qps, 1), "max_batch_pairs": serve_batch,
                   "offered": loads}
        del L60

    # single-source BFS comparison and the d sweep (the same resident graph)
    nxt = None
    if args.next_rows and rank == 0:
        nxt = {"bfs_comparison": bfs_comparison(g, off, adj, seed=rank_seed(rank) + 21,
                                                seq=cpu.get("seq_bfs") if cpu else None)}
        # centres of degree >= 63 so that even d = 2, 3 clusters have 64 vertices
        sweep = {f"rmat_s{args.scale}": d_sweep(cbfs, g, off, adj, seed=rank_seed(rank) + 22, min_deg=63)}
        goff, gadj = I.road_grid(1024, seed=I.MASTER_SEED + 2)
        with cbfs.Graph(goff, gadj) as gg:
            sweep["road_grid_1024"] = d_sweep(cbfs, gg, goff, gadj, seed=rank_seed(rank) + 23)
        nxt["d_sweep"] = sweep
        nxt["ll_quality"] = ll_quality(cbfs, g, off, adj, seed=rank_seed(rank) + 24)
        nxt["road_grid"] = road_grid_throughput(cbfs, seed=I.MASTER_SEED + 3)

    # End to end through the public API, the timed step's work: the CSR from
    # page-locked host memory (H2D inside graph create), the batched traversal
    # into device outputs, the label append, the query with its pairs H2D and
    # its answers D2H -- the answers are the step's result.  Two variants
    # beside it: the traversal writing the label store itself
    # (cbfs_run_batched_labels, no outputs kept; label calls keep one cluster
    # per slot word), and that plus all 18 GB of dist/masks streamed into
    # page-locked host memory during the traversal, whose rate depends on the
    # machine's host-memory bandwidth (shared with the other GPUs' tenants).
    e2e = None
    if args.e2e_steps > 0:
        off_pin, adj_pin, dist_h, masks_h = e2e_host
        bi = off.nbytes + adj.nbytes + src_cat.nbytes + coff.nbytes + pairs.nbytes

        def e2e_run(mode: str):
            times, parts = [], []
            for it in range(args.e2e_steps + 1):  # the first step is an untimed warm-up
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                g2 = cbfs.Graph(off_pin, adj_pin, validate=True)
                t1 = time.perf_counter()
                L.reset()
                if mode == "outputs":
                    g2.run_batched(None, d, dist, masks, tune=tset, sources_concat=src_cat, cluster_off=coff)
                    L.append(dist, masks, ks)
                else:
                    g2.run_batched_labels(None, d, L, dist=dist_h if mode == "host" else None,
                                          masks=masks_h if mode == "host" else None, tune=tset,
                                          sources_concat=src_cat, cluster_off=coff)
                torch.cuda.synchronize()  # the traversal's share of the step (the calls only enqueue)
                t2 = time.perf_counter()
                pairs_dev.copy_(pin_pairs, non_blocking=True)
                L.query(pairs_dev, out=answers)
                pin_ans.copy_(answers, non_blocking=True)
                torch.cuda.synchronize()
                t3 = time.perf_counter()
                if it > 0:
                    times.append(t3 - t0)
                    parts.append((t1 - t0, t2 - t1, t3 - t2))
                g2.close()
            t = max(statistics.median(times), 1e-9)
            return t, dict(zip(("graph_create", "traversal_labels", "query"),
                               [round(1e3 * statistics.median(p[i] for p in parts), 2) for i in range(3)]))

        e_t, e_parts = e2e_run("outputs")
        e2e = {"value": round(src_edges / e_t / 1e9 * ws, 4), "unit": "GTEPS", "h2d_bytes_per_step": int(bi),
               "d2h_bytes_per_step": int(args.query_batch * 2), "ms_per_step": round(e_t * 1e3, 3),
               "includes": "graph create + validate from the page-locked host CSR; batched C-BFS of all clusters "
                           "into device outputs (cbfs_run_batched) and the label append; query with pairs H2D "
                           "and answers D2H",
               "ms_parts": e_parts}
        l_t, l_parts = e2e_run("labels")
        e2e["labels_by_the_traversal"] = {
            "value": round(src_edges / l_t / 1e9 * ws, 4), "unit": "GTEPS", "ms_per_step": round(l_t * 1e3, 3),
            "ms_parts": l_parts,
            "includes": "the same with the traversal writing the label store itself (cbfs_run_batched_labels, "
                        "no outputs kept)"}
        del dist, masks
        torch.cuda.empty_cache()
        if dist_h is not None:
            h_t, h_parts = e2e_run("host")
            e2e["with_host_outputs"] = {
                "value": round(src_edges / h_t / 1e9 * ws, 4), "unit": "GTEPS", "ms_per_step": round(h_t * 1e3, 3),
                "d2h_bytes_per_step": int(dist_h.numel() + masks_h.numel() * 8 + args.query_batch * 2),
                "ms_parts": h_parts,
                "includes": "the same plus every cluster's dist/masks streamed into page-locked host memory "
                            "(copies overlap later waves)"}

    # the other two workloads, last: one small cluster, and label construction
    # at scale 24 (its 0.5 GB-CSR generation churns host memory, which slows
    # later page-locked copies, so it runs after the end-to-end measurement)
    configs = None
    if args.configs and rank == 0:
        configs = {"single_cluster_s14": single_cluster_config(cbfs),
                   "label_construction_s24": label_construction_config(cbfs)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": bench_config(args.scale, C, d, n, adj.size, int(ks.sum()), args.query_batch),
            "tune": dict(tset, cached=tn.get("cached")),
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(prof["total_launches"] + 2 * args.steps),
            "clocks": clocks.summary(),
            "phase_ms_per_step": {"cbfs": round(cbfs_ms / args.steps, 3),
                                  "labels_query": round((t_ms - cbfs_ms) / args.steps, 3)},
            "alg_gbs_step": round(alg_bytes_step * args.steps / (t_ms / 1e3) / 1e9, 1),
            "work_per_step": {"V": V, "A": A, "source_edges": src_edges, "alg_bytes": int(alg_bytes_step)},
            "lockstep": lockstep,
            "kernel_ms_one_untimed_step": {k: split[k] for k in ("setup", "vertex_phase", "edge_phase")},
            "query": query,
            "serving": serving,
            "one_cluster_per_launch": one,
            "next": nxt,
            "configs": configs,
        }
        # last, so that it stays inside the tail of the output a reader keeps
        line["summary"] = summary_of(line)
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def pack_words(ks, per_word: int = 31) -> list:
    """The library's slot words for a call with device outputs (cbfs_tune_t
    pack): clusters by size descending (ties in call order), each into the
    fullest word with room for it (the latest such word first), at most
    `per_word` to a word, 64 bits each; one cluster per word when that saves
    no words.  Reporting only: the library decides on its own."""
    ks = [int(k) for k in ks]
    order = sorted(range(len(ks)), key=lambda c: -ks[c])
    words, used, by_free = [], [], [[] for _ in range(65)]
    for c in order:
        k, ws = ks[c], -1
        for f in range(k, 65):
            lst = by_free[f]
            while lst and ws < 0:
                wi = lst.pop()
                if 64 - used[wi] == f and len(words[wi]) < per_word:
                    ws = wi
            if ws >= 0:
                break
        if ws < 0:
            ws = len(words)
            words.append([])
            used.append(0)
        words[ws].append(c)
        used[ws] += k
        if used[ws] < 64 and len(words[ws]) < per_word:
            by_free[64 - used[ws]].append(ws)
    if len(ks) < 2 or len(words) >= len(ks):
        return [[c] for c in order]
    return words


def lockstep_rounds(ks, rounds, slots: int) -> dict:
    """How long work waits in the lockstep waves: the library packs a call's
    clusters into 64-bit slot words (pack_words), `slots` words to a wave in
    that order, and a word runs as many rounds as its deepest cluster, a wave
    as many as its deepest word.  Returns the rounds the waves ran against
    the rounds their words needed (slot-rounds; 1 - ratio is the idle share)
    and the rounds the clusters needed."""
    rounds = np.asarray(rounds, dtype=np.int64)
    words = pack_words(ks)
    word_rounds = [int(rounds[w].max()) for w in words]
    P = max(1, int(slots))
    wave_rounds = [max(word_rounds[i:i + P]) for i in range(0, len(words), P)]
    used = sum(word_rounds)
    offered = sum(r * min(P, len(words) - i * P) for i, r in enumerate(wave_rounds))
    return {"waves": len(wave_rounds), "words": len(words), "wave_rounds": int(sum(wave_rounds)),
            "word_rounds": int(used), "cluster_rounds": int(rounds.sum()),
            "busy_slot_round_share": round(used / max(offered, 1), 4)}


def summary_of(line: dict) -> dict:
    """The figures of every workload in a few hundred bytes."""
    def get(*path):
        x = line
        for k in path:
            if not isinstance(x, dict) or k not in x:
                return None
            x = x[k]
        return x

    rf = line["roofline"]
    out = {"gteps": line["value"], "ms_per_step": line["ms_per_step"],
           "traversal_ms": rf["avg_launch_ms"], "alg_frac": rf["frac"],
           "physical_frac": rf.get("physical_frac"), "garcs_per_s": round(rf["arcs_per_s"] / 1e9, 1),
           "e2e_gteps": get("e2e", "value"),
           "batched_speedup_vs_one_cluster_per_launch": get("one_cluster_per_launch", "batched_speedup"),
           "query_kernel_frac": get("query", "kernel", "frac"),
           "query_single_p50_p99_ms": [get("query", "p50_ms"), get("query", "p99_ms")],
           "serving_saturation_qps": get("serving", "saturation_qps")}
    for load in ("0.5x", "0.8x"):
        out[f"serving_{load}_p50_p99_ms"] = [get("serving", "offered", load, "p50_ms"),
                                             get("serving", "offered", load, "p99_ms")]
    rg = get("next", "road_grid")
    if rg:
        out["road_grid_4096"] = {"gteps": rg["gteps"], "alg_frac": rg["alg_frac"], "ms": rg["ms_all_clusters"],
                                 "garcs_per_s": round(rg["arcs_per_s"] / 1e9, 1)}
    # share of slot-rounds in which a wave's cluster still had work (lockstep waves)
    out["lockstep_busy"] = [get("lockstep", "busy_slot_round_share"),
                            get("next", "road_grid", "lockstep", "busy_slot_round_share")]
    lc = get("configs", "label_construction_s24")
    if lc:
        out["labels_s24_1024"] = {"traversal_ms": lc["traversal_ms"], "alg_frac": lc["alg_frac"],
                                  "garcs_per_s": round(lc["arcs_per_s"] / 1e9, 1)}
    sc = get("configs", "single_cluster_s14")
    if sc:
        out["single_s14_ms"] = {k: sc[k]["ms_per_call_device"] for k in ("random_centres", "centres_deg_ge_63")}
    bc = get("next", "bfs_comparison")
    if bc:
        out["bit_level_gain"] = bc["bit_level_gain"]
    return out


def record_traffic(csv_paths: str, run_json: str, note: str):
    """Writes profiles/traffic.json from ncu CSVs and the runcli line of the
    captured run (see traffic_from_csv)."""
    with open(run_json) as f:
        run = json.loads([ln for ln in f.read().splitlines() if ln.startswith("{")][-1])
    out = traffic_from_csv(csv_paths.split(","), run, note)
    with open(os.path.join(ROOT, "profiles", "traffic.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))
    return 0


def memset_bytes_per_wave(n: int, P: int, rows: bool = True) -> int:
    """Bytes the per-wave state resets write: vis and acc (8 P bytes per
    vertex each), the claim stamps (4), the Delta rows (P; waves with round
    records have none), two frontier bitmaps and the round control blocks
    (288 x 56 bytes)."""
    bitmap_words = (n + 31) // 32 + 1
    return (16 * P + 4 + (P if rows else 0)) * n + 2 * 4 * bitmap_words + 288 * 56


def traffic_from_csv(csv_paths, run: dict, note: str) -> dict:
    """DRAM bytes of the traversal kernels of one host-driven `runcli` call
    (ncu dram__bytes_read.sum + dram__bytes_write.sum, one kernel and at most
    three launches per capture, the captures together covering every launch
    of the call), plus the per-wave memset bytes counted from their sizes,
    over that call's algorithmic bytes (13 A + 41 V + C n (1 + 8 d)).  The
    bench multiplies its own launch's algorithmic bytes by this ratio."""
    import csv as csv_

    kinds = ("k_seed", "k_phase_a", "k_phase_b", "k_emit", "k_flush", "k_check_sources", "k_map_seeds")
    per_kernel, launches = {}, {}
    for path in csv_paths:
        with open(path) as f:
            rows = [r for r in csv_.reader(f)]
        hdr = next((i for i, r in enumerate(rows) if r and r[0] == "ID"), None)
        if hdr is None:
            continue
        cols = rows[hdr]
        for r in rows[hdr + 1:]:
            if len(r) != len(cols):
                continue
            rec = dict(zip(cols, r))
            name = rec["Kernel Name"]
            if not rec["Metric Name"].startswith("dram__bytes") or not any(k in name for k in kinds):
                continue
            scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}[rec["Metric Unit"]]
            v = float(rec["Metric Value"].replace(",", "")) * scale
            key = name.split("(")[0].replace("void ", "")
            per_kernel[key] = per_kernel.get(key, 0.0) + v
            launches.setdefault(key, set()).add((path, rec["ID"]))
    n, d, C = int(run["n"]), int(run["d"]), int(run["clusters"])
    P = int(run["tune"]["slots"])
    # k_seed runs once per wave (packed waves hold more clusters than slots);
    # waves that write their outputs from round records (k_flush) have no rows
    seeds = [k for k in launches if "k_seed" in k]
    waves = len(launches[seeds[0]]) if seeds else (C + P - 1) // P
    rows = not any("k_flush" in k for k in per_kernel)
    kernel_bytes = sum(per_kernel.values())
    memsets = waves * memset_bytes_per_wave(n, P, rows)
    alg = ARC_BYTES * int(run["A"]) + VERTEX_BYTES * int(run["V"]) + C * n * (1 + 8 * d)
    return {"traversal": {"dram_bytes_per_alg_byte": (kernel_bytes + memsets) / alg,
                          "kernel_dram_bytes": int(kernel_bytes), "memset_bytes": int(memsets),
                          "alg_bytes": int(alg), "clusters": C, "slots": P, "waves": waves,
                          "per_kernel_bytes": {k: int(v) for k, v in sorted(per_kernel.items())},
                          "launches_captured": {k: len(v) for k, v in sorted(launches.items())},
                          "source_hash": kernel_source_hash(), "measured_on": note}}


def main():
    args = parse()
    if args.record_traffic:
        return record_traffic(args.record_traffic, args.traffic_run,
                              f"R-MAT scale {args.scale}, one host-driven runcli call; per-wave memsets counted "
                              "from their sizes; scaled to a launch by its algorithmic bytes")
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    return run_cbfs(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
