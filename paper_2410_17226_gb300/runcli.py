"""Command line: one batched C-BFS on a synthetic graph, with its work counters.

    python -m paper_2410_17226_gb300.runcli --graph rmat --scale 22 --clusters 16 --slots 8

Builds the seeded graph, picks the clusters (random stars for R-MAT, BFS
balls for the road grid), runs ``cbfs_run_batched`` once (``--repeat`` more
times to replay the cached CUDA graph) and prints the Theorem 1 counters
A (arcs scanned) and V (frontier appearances) and the wall time of the last
call.  Useful for profiling a single traversal in isolation.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import cbfs
from . import inputs as I


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--graph", choices=["rmat", "grid"], default="rmat")
    ap.add_argument("--scale", type=int, default=20, help="R-MAT scale, or the grid side for --graph grid")
    ap.add_argument("--clusters", type=int, default=16)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--pull-alpha", type=float, default=0.0, help="0: the library default")
    ap.add_argument("--small-deg", type=int, default=0, help="thread-per-vertex degree limit (0: default)")
    ap.add_argument("--mid-deg", type=int, default=0, help="warp-per-vertex degree limit (0: default)")
    ap.add_argument("--host-loop", action="store_true", help="host-driven rounds instead of a CUDA graph")
    ap.add_argument("--fused-pull", action="store_true", help="pull rounds do the next vertex phase (tune.fused_pull)")
    ap.add_argument("--repeat", type=int, default=0, help="extra calls after the first")
    args = ap.parse_args(argv)

    if args.graph == "rmat":
        off, adj = I.rmat(args.scale)
        clusters, d = I.star_clusters(off, adj, args.clusters, seed=I.MASTER_SEED + 1, size="uniform")
    else:
        off, adj = I.road_grid(args.scale)
        clusters, ds = I.ball_clusters(off, adj, args.clusters, 64, seed=I.MASTER_SEED + 3)
        d = max(ds)
    g = cbfs.Graph(off, adj, validate=False)
    C = len(clusters)
    dist = torch.empty((C, g.n), dtype=torch.uint8, device="cuda")
    masks = torch.empty((C, d, g.n), dtype=torch.int64, device="cuda")
    tune = {"slots": args.slots, "pull_alpha": args.pull_alpha, "host_loop": int(args.host_loop),
            "small_deg": args.small_deg, "mid_deg": args.mid_deg, "fused_pull": int(args.fused_pull)}
    ms = 0.0
    for _ in range(1 + args.repeat):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.run_batched(clusters, d, dist, masks, tune=tune)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
    st = g.output_stats(dist, masks, [len(S) for S in clusters], d)
    print(json.dumps({"n": g.n, "nnz": g.nnz, "clusters": C, "d": d, "A": int(st[:, 1].sum()),
                      "V": int(st[:, 0].sum()), "reached_arcs": int(st[:, 2].sum()),
                      "last_call_ms": round(ms, 3), "tune": tune}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
