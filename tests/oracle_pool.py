"""Many clusters checked against the oracle in parallel (test helper).

The oracle is plain C called through ctypes, and ctypes releases the GIL for
the duration of a foreign call, so a thread pool runs one oracle cluster per
host core with no process fork (a fork after CUDA has started in this process
could hang) and no copy of the graph.  Each cluster's CUDA outputs are copied
to the host in chunks of the pool's width and compared with Algorithm 1's
outputs element by element.
"""
from __future__ import annotations

import concurrent.futures as cf
import os

import numpy as np

import oracle as O


def host_cores() -> int:
    return max(1, len(os.sched_getaffinity(0)))


def _u64(t) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint64)


def oracle_outputs(off, adj, clusters, d, workers: int | None = None):
    """Algorithm 1 outputs of every cluster: (dist uint8 [C, n], masks uint64 [C, d, n])."""
    n = off.size - 1
    dist = np.empty((len(clusters), n), np.uint8)
    masks = np.empty((len(clusters), d, n), np.uint64)

    def one(c):
        dist[c], masks[c] = O.cbfs_alg1(off, adj, clusters[c], d)

    with cf.ThreadPoolExecutor(workers or host_cores()) as ex:
        list(ex.map(one, range(len(clusters))))
    return dist, masks


def assert_host_equal_oracle(off, adj, clusters, d, got, workers: int | None = None):
    """got: {cluster index: (dist uint8 [n], masks uint64 [d, n])} already on
    the host; every entry is compared with the oracle, one per worker thread.
    Returns the number of clusters compared."""
    def check(c):
        od, om = O.cbfs_alg1(off, adj, clusters[c], d)
        gd, gm = got[c]
        bad_d = np.flatnonzero(gd != od)
        bad_m = np.flatnonzero((gm != om).any(axis=0)) if d else np.zeros(0, np.int64)
        return c, bad_d[:5].tolist(), bad_m[:5].tolist()

    done = 0
    with cf.ThreadPoolExecutor(workers or host_cores()) as ex:
        for c, bd, bm in ex.map(check, sorted(got)):
            assert not bd, f"cluster {c}: dist differs from the oracle at vertices {bd}"
            assert not bm, f"cluster {c}: masks differ from the oracle at vertices {bm}"
            done += 1
    return done


def host_copy(dist_row, masks_rows):
    """One cluster's CUDA outputs as host arrays (dist uint8, masks uint64)."""
    return dist_row.cpu().numpy(), _u64(masks_rows)


def assert_equal_oracle(off, adj, clusters, d, dist_dev, masks_dev, which, workers: int | None = None):
    """dist_dev [C, n] / masks_dev [C, d, n] (torch, any device) hold the CUDA
    outputs of `clusters`; clusters `which` are compared with the oracle bit
    for bit.  Returns the number of clusters compared."""
    which = list(which)
    width = workers or host_cores()
    done = 0
    for i in range(0, len(which), width):
        got = {c: host_copy(dist_dev[c], masks_dev[c]) for c in which[i:i + width]}
        done += assert_host_equal_oracle(off, adj, clusters, d, got, workers=width)
        del got
    return done
