"""Autotuner for the traversal: the push/pull switch factor, the number of
clusters in flight per wave, and the degree thresholds of the dense edge
phase (thread, warp or CTA per vertex).

The direction rule (Appendix A, Algorithm "EdgeMap") switches to the dense
(pull) edge phase when |F| + sum deg(F) exceeds a fraction of the arcs; the
best fraction for C-BFS differs from plain BFS because pull cannot stop at
the first frontier neighbour.  ``autotune`` times a sample of clusters on the
resident graph for every (switch factor, clusters per wave) pair, then for
every (thread, warp) degree threshold pair at the best of those, and keeps the
fastest.  Results are cached in ``tune_cache.json`` next to this file, keyed
by GPU name and graph shape.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import numpy as np
import torch

from . import cbfs

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json")
ALPHAS = (0.005, 0.01, 0.02, 0.04, 0.08, 0.2, 0.4, 0.6, -1.0)  # -1: push only
SLOTS = (1, 2, 4, 8)
SMALL_DEGS = (8, 16, 32)          # one thread per vertex up to this degree
MID_DEGS = (1024, 2048, 4096, 16384, 65536)  # one warp per vertex up to this degree, CTA pieces above


def graph_key(g: "cbfs.Graph", d: int, extra: str = "") -> str:
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "none"
    return f"{name}|n={g.n}|nnz={g.nnz}|d={d}|{extra}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(table):
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def autotune(g: "cbfs.Graph", clusters, d: int, sample: int = 32, alphas=ALPHAS, slots=SLOTS,
             small_degs=SMALL_DEGS, mid_degs=MID_DEGS, key_extra: str = "", use_cache: bool = True,
             write_cache: bool = True, stream=None) -> dict:
    """Returns ``{"pull_alpha": a, "slots": s, "small_deg": t, "mid_deg": m,
    "fused_pull": r, "ms": best, "table": {...}}``."""
    key = graph_key(g, d, key_extra)
    if use_cache:
        hit = _load().get(key)
        if hit:
            return dict(hit, cached=True)
    part = list(clusters[:sample])
    C = len(part)
    dist = torch.empty((C, g.n), dtype=torch.uint8, device="cuda")
    masks = torch.empty((C, max(d, 0), g.n), dtype=torch.int64, device="cuda")
    table = {}

    def timed(tune):
        g.run_batched(part, d, dist, masks, tune=tune, stream=stream)  # warm-up (and graph capture)
        g.run_batched(part, d, dist, masks, tune=tune, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.run_batched(part, d, dist, masks, tune=tune, stream=stream)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3

    best = None
    for s in slots:
        for a in alphas:
            ms = timed({"pull_alpha": a, "slots": s})
            table[f"a={a},s={s}"] = round(ms, 3)
            if best is None or ms < best["ms"]:
                best = {"pull_alpha": a, "slots": s, "small_deg": 0, "mid_deg": 0, "ms": ms}
    for t in small_degs:
        for m in mid_degs:
            if m < t:
                continue
            tune = {"pull_alpha": best["pull_alpha"], "slots": best["slots"], "small_deg": t, "mid_deg": m}
            ms = timed(tune)
            table[f"a={best['pull_alpha']},s={best['slots']},t={t},m={m}"] = round(ms, 3)
            if ms < best["ms"]:
                best = dict(tune, ms=ms)
    # plain or fused pull rounds (the vertex phase of the next round done by
    # the pull): graphs differ
    tune = {k: best[k] for k in ("pull_alpha", "slots", "small_deg", "mid_deg")}
    tune["fused_pull"] = 1
    ms = timed(tune)
    table[f"a={best['pull_alpha']},s={best['slots']},t={best['small_deg']},m={best['mid_deg']},fused_pull"] = round(ms, 3)
    best["fused_pull"] = 0
    if ms < best["ms"]:
        best = dict(tune, ms=ms)
    best["table"] = table
    best["sample"] = C
    if write_cache:
        t = _load()
        t[key] = best
        _store(t)
    return dict(best, cached=False)


def signature(off) -> str:
    """Short hash of a degree sequence (for cache keys of generated graphs)."""
    off = np.asarray(off)
    return hashlib.sha1(np.diff(off).astype(np.int64).tobytes()).hexdigest()[:12]
