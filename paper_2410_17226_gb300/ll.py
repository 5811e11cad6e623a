"""Approximate distance oracle by landmark labeling (Section 4.2) with
clustered landmarks, and its distortion.

Clusters are chosen by the paper's degree rule (the highest-degree unmarked
vertex plus its w-1 highest-degree unmarked neighbours, repeated), as many as
a memory budget of ``t`` bytes per vertex allows: a cluster of word size w and
diameter d costs 1 + d * w / 8 bytes per vertex (one distance byte and d
subset words), a plain landmark (k = 1, d = 0) one byte.  With t = 1024 that
is 60 clusters for w = 64, 341 for w = 8, 1024 plain landmarks.  The index is
the label store of those clusters, built on the GPU by one batched C-BFS
call that writes the rows as it goes.

Distortion (Section 4.2): for a pair with finite true distance delta(u, v) > 0
the answer q(u, v) >= delta(u, v) (one-sided), psi = q / delta, and the
reported error is epsilon = mean(psi) - 1.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs as I

NO_PATH = 0xFFFF


def cluster_count(budget_bytes_per_vertex: int, d: int, w: int) -> int:
    """Clusters that fit the budget: floor(t / (1 + d * w / 8))."""
    return int(budget_bytes_per_vertex // (1 + d * w // 8))


def select(off, adj, budget_bytes_per_vertex: int = 1024, w: int = 64, d: int = 2):
    """Landmark clusters for the budget.  ``w = 1`` selects plain landmarks
    (single vertices by degree, d = 0).  Returns ``(clusters, d)``."""
    if w == 1:
        deg = I.degrees(off)
        order = np.lexsort((np.arange(deg.size), -deg))
        picks = order[:min(int(budget_bytes_per_vertex), deg.size)]
        return [np.array([v], np.int32) for v in picks], 0
    if d != 2:
        raise ValueError("the degree rule draws a vertex and its neighbours: d = 2")
    clusters, d = I.degree_clusters(off, adj, cluster_count(budget_bytes_per_vertex, d, w), k=w)
    return clusters, d


def build(g, clusters, d: int, w: int, tune: dict | None = None, stream=None):
    """Label store of the clusters (``Labels`` of word size w; w = 64 for
    plain landmarks) filled by ``cbfs_run_batched_labels``.  Returns
    ``(labels, milliseconds)``."""
    import torch

    from . import cbfs

    L = cbfs.Labels(g.n, max(len(clusters), 1), d, w=max(w, 8) if d > 0 else 64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.run_batched_labels(clusters, d, L, tune=tune, stream=stream)
    torch.cuda.synchronize()
    return L, (time.perf_counter() - t0) * 1e3


def distortion(answers, exact) -> dict:
    """epsilon = mean(q / delta) - 1 over pairs with finite delta > 0 (answers
    uint16, exact int: hop counts, negative = unreachable).  Pairs the index
    cannot answer (no landmark reached from both ends) are counted apart."""
    q = np.asarray(answers).astype(np.int64)
    t = np.asarray(exact).astype(np.int64)
    ok = t > 0
    unanswered = ok & (q == NO_PATH)
    use = ok & ~unanswered
    if not use.any():
        return {"pairs": 0, "epsilon": None, "exact_share": None, "unanswered": int(unanswered.sum())}
    if (q[use] < t[use]).any():
        raise ValueError("an answer below the true distance: the index is not one-sided")
    psi = q[use] / t[use]
    return {"pairs": int(use.sum()), "epsilon": float(psi.mean() - 1.0),
            "exact_share": float((q[use] == t[use]).mean()), "unanswered": int(unanswered.sum())}
