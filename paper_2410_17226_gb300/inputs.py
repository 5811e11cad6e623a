"""Seeded synthetic inputs: graphs in CSR form and source clusters.

This module feeds both the CUDA path and the oracle.  It holds none of the
C-BFS arithmetic: it only draws graphs and picks clusters.  Every generator is
deterministic given its seed.  Graphs come from a small C helper
(``gen/graph_gen.c``) driven by splitmix64 as a counter-based generator;
clusters and query pairs use the raw PCG64 bit stream
(``numpy.random.PCG64.random_raw``).  Both streams are fixed by their
published definitions, so the inputs are identical on every machine.

Graphs (all undirected, stored with both arc directions, no self loops, no
duplicate arcs, adjacency lists sorted, ``off`` int64[n+1], ``adj`` int32):

* ``rmat``: R-MAT(scale, edge factor, a, b, c) -- the power-law stand-in for
  the paper's social and web graphs (Section 5).  Each of the
  ``edge_factor * 2**scale`` draws picks a quadrant per bit level from a
  16-bit uniform field; vertex ids are then relabelled by a seeded
  Fisher-Yates permutation, self loops dropped, duplicates merged, arcs
  symmetrised.
* ``road_grid``: a ``side x side`` 4-neighbour grid with each edge deleted
  independently with probability ``p_delete`` and ``floor(shortcut_frac *
  grid_edges)`` uniform random shortcut edges added -- the high-diameter
  road-like stand-in.
* small exact families for tests: ``path``, ``cycle``, ``grid``,
  ``erdos_renyi``, ``from_edges``.

Clusters (each a list of distinct vertex ids; the diameter bound ``d`` is
returned beside it):

* ``star_clusters``: a random non-isolated centre plus random neighbours
  (d = 2), the workload of the paper's microbenchmarks (Section 5.1).
* ``degree_clusters``: the paper's landmark selection (Section 4.2): the
  highest-degree unmarked vertex plus its k-1 highest-degree unmarked
  neighbours, repeated (d = 2).
* ``ball_clusters``: a random centre plus the next k-1 vertices in BFS order
  from it; d = the exact diameter of that set (at most twice the BFS level
  of the last one taken).
* ``radius_cluster``: a cluster whose diameter is at most a given d, drawn
  from hop counts to a centre that the caller supplies (the d-sweep
  workload; the hop counts come from whichever BFS the caller trusts).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

MASTER_SEED = 2410172260

_GEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gen")
_GEN_SRC = os.path.join(_GEN_DIR, "graph_gen.c")
_GEN_LIB = os.path.join(_GEN_DIR, "libgraphgen.so")
_glib = None


def build_generator(force: bool = False) -> str:
    """Compile the C graph generator next to its source (gcc -O2)."""
    if force or not os.path.exists(_GEN_LIB) or os.path.getmtime(_GEN_LIB) < os.path.getmtime(_GEN_SRC):
        tmp = _GEN_LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _GEN_SRC]
        try:  # OpenMP only parallelises the draws; the output does not depend on it
            subprocess.check_call(base + ["-fopenmp"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _GEN_LIB)
    return _GEN_LIB


def _gl():
    global _glib
    if _glib is None:
        lib = ctypes.CDLL(build_generator())
        P, i64, u64, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32
        lib.gen_splitmix64.argtypes = [u64, u64]
        lib.gen_splitmix64.restype = u64
        lib.gen_rmat_edges.argtypes = [ctypes.c_int, i64, u32, u32, u32, u64, u64, P, P]
        lib.gen_rmat_edges.restype = ctypes.c_int
        lib.gen_road_grid_edges.argtypes = [i64, u32, i64, u64, P, P]
        lib.gen_road_grid_edges.restype = i64
        lib.gen_unique_edges.argtypes = [i64, i64, P, P, P]
        lib.gen_unique_edges.restype = i64
        lib.gen_csr_fill.argtypes = [i64, i64, P, P, P]
        lib.gen_csr_fill.restype = ctypes.c_int
        _glib = lib
    return _glib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _raw(gen: np.random.Generator, count: int) -> np.ndarray:
    return gen.bit_generator.random_raw(count).astype(np.uint64, copy=False)


def _gen(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _uniform_below(gen: np.random.Generator, count: int, bound: int) -> np.ndarray:
    """``count`` integers uniform in [0, bound) (64-bit draw reduced mod bound)."""
    if bound <= 0:
        raise ValueError("bound must be positive")
    return (_raw(gen, count) % np.uint64(bound)).astype(np.int64)


# --------------------------------------------------------------------------- CSR


def from_edges(n: int, src, dst):
    """CSR of the undirected simple graph with the given edge list.

    Self loops are dropped, both directions stored, duplicates merged,
    adjacency lists sorted.  Returns ``(off int64[n+1], adj int32[nnz])``.
    """
    src = np.ascontiguousarray(src, dtype=np.int64).ravel()
    dst = np.ascontiguousarray(dst, dtype=np.int64).ravel()
    if src.size != dst.size:
        raise ValueError("src and dst differ in length")
    if n < 0 or n > 0x7FFFFFFF:
        raise ValueError("vertex count out of range")
    m = src.size
    keys = np.empty(max(m, 1), dtype=np.uint64)
    u = _gl().gen_unique_edges(n, m, _ptr(src), _ptr(dst), _ptr(keys))
    if u < 0:
        raise ValueError("edge endpoint out of range" if u == -1 else f"generator error {u}")
    off = np.empty(n + 1, dtype=np.int64)
    adj = np.empty(max(2 * u, 1), dtype=np.int32)
    rc = _gl().gen_csr_fill(n, u, _ptr(keys), _ptr(off), _ptr(adj))
    if rc:
        raise MemoryError("gen_csr_fill")
    return off, adj[:2 * u]


def path(n: int):
    v = np.arange(max(n - 1, 0))
    return from_edges(n, v, v + 1)


def cycle(n: int):
    v = np.arange(n)
    return from_edges(n, v, (v + 1) % n)


def grid(w: int, h: int):
    """w x h 4-neighbour grid, vertex (x, y) has id y*w + x."""
    ids = np.arange(w * h).reshape(h, w)
    src = np.concatenate([ids[:, :-1].ravel(), ids[:-1, :].ravel()])
    dst = np.concatenate([ids[:, 1:].ravel(), ids[1:, :].ravel()])
    return from_edges(w * h, src, dst)


def erdos_renyi(n: int, m: int, seed: int):
    """n vertices, m uniform random edge draws (before dedup / self-loop removal)."""
    g = _gen(seed)
    if n <= 0:
        return from_edges(max(n, 0), [], [])
    return from_edges(n, _uniform_below(g, m, n), _uniform_below(g, m, n))


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = MASTER_SEED, permute: bool = True):
    """Undirected R-MAT graph with ``2**scale`` vertices (see module docstring)."""
    n = 1 << scale
    m = edge_factor * n
    src = np.empty(m, dtype=np.int64)
    dst = np.empty(m, dtype=np.int64)
    ta, tab, tabc = (int(round(x * 65536)) for x in (a, a + b, a + b + c))
    perm_seed = (seed ^ 0x5EED5EED5EED5EED) & 0xFFFFFFFFFFFFFFFF if permute else 0
    rc = _gl().gen_rmat_edges(scale, edge_factor, ta, tab, tabc, seed, perm_seed, _ptr(src), _ptr(dst))
    if rc:
        raise ValueError(f"gen_rmat_edges failed ({rc})")
    return from_edges(n, src, dst)


def road_grid(side: int, p_delete: float = 0.10, shortcut_frac: float = 0.01, seed: int = MASTER_SEED + 2):
    """Grid with random edge deletions and random long-range shortcuts."""
    n = side * side
    e_grid = 2 * side * (side - 1)
    n_short = int(shortcut_frac * e_grid)
    src = np.empty(max(e_grid + n_short, 1), dtype=np.int64)
    dst = np.empty(max(e_grid + n_short, 1), dtype=np.int64)
    thr = min(int(round(p_delete * 2.0 ** 32)), 0xFFFFFFFF)
    cnt = _gl().gen_road_grid_edges(side, thr, n_short, seed, _ptr(src), _ptr(dst))
    if cnt < 0:
        raise ValueError("gen_road_grid_edges failed")
    return from_edges(n, src[:cnt], dst[:cnt])


# ----------------------------------------------------------------------- clusters


def degrees(off) -> np.ndarray:
    off = np.asarray(off, dtype=np.int64)
    return off[1:] - off[:-1]


def star_clusters(off, adj, count: int, seed: int, size: str = "max", kmax: int = 64, min_deg: int = 1):
    """``count`` star clusters: a uniform random centre of degree >= min_deg
    (default: any non-isolated vertex) plus a uniform random subset of its
    neighbours, drawn without replacement.

    ``size="max"``: as many neighbours as fit (k = min(kmax, 1 + deg)).
    ``size="uniform"``: k uniform in 1..kmax, capped at 1 + deg.
    Returns ``(list of int32 arrays, d)`` with d = 2 (1 for k = 1 ... still 2
    is a valid bound; callers may pass it as is).
    """
    deg = degrees(off)
    cand = np.flatnonzero(deg >= max(min_deg, 1))
    if cand.size == 0:
        raise ValueError("graph has no edges")
    g = _gen(seed)
    out = []
    for _ in range(count):
        ctr = int(cand[int(_uniform_below(g, 1, cand.size)[0])])
        nb = np.asarray(adj[off[ctr]:off[ctr + 1]], dtype=np.int64)
        if size == "uniform":
            k = 1 + int(_uniform_below(g, 1, kmax)[0])
        else:
            k = kmax
        k = min(k, 1 + nb.size)
        order = np.argsort(_raw(g, nb.size), kind="stable")
        members = np.concatenate([[ctr], nb[order[:k - 1]]]).astype(np.int32)
        out.append(members)
    return out, 2


def degree_clusters(off, adj, count: int, k: int = 64):
    """The paper's landmark-cluster selection for d = 2 (Section 4.2).

    Repeatedly take the highest-degree unmarked vertex and up to k-1 of its
    unmarked neighbours with the highest degrees (ties go to the smaller id),
    then mark them all.  Stops early when no unmarked vertex is left.
    """
    deg = degrees(off)
    n = deg.size
    order = np.lexsort((np.arange(n), -deg))
    marked = np.zeros(n, dtype=bool)
    out = []
    p = 0
    while len(out) < count:
        while p < n and marked[order[p]]:
            p += 1
        if p >= n:
            break
        ctr = int(order[p])
        nb = np.asarray(adj[off[ctr]:off[ctr + 1]], dtype=np.int64)
        nb = nb[~marked[nb]]
        nb = nb[np.lexsort((nb, -deg[nb]))][:k - 1]
        members = np.concatenate([[ctr], nb]).astype(np.int32)
        marked[members] = True
        out.append(members)
    return out, 2


def _bounded_bfs(off, adj, src: int, limit: int) -> dict:
    """Hop counts from src to every vertex within `limit` hops."""
    level = {src: 0}
    frontier = [src]
    for h in range(1, limit + 1):
        nxt = []
        for u in frontier:
            for v in adj[off[u]:off[u + 1]]:
                v = int(v)
                if v not in level:
                    level[v] = h
                    nxt.append(v)
        frontier = nxt
        if not frontier:
            break
    return level


def ball_clusters(off, adj, count: int, k: int, seed: int, dmax: int = 15, max_tries: int = 1000):
    """Clusters of a random centre plus the next k-1 vertices in BFS order
    (neighbours taken in adjacency order, i.e. smaller id first).

    Returns ``(list of int32 arrays, list of d)`` where d is the exact
    diameter of the cluster (largest pairwise hop count, found by BFSs bounded
    at twice the ball radius).  Centres whose component holds fewer than k
    vertices, or whose cluster diameter exceeds ``dmax``, are redrawn.
    """
    off = np.asarray(off, dtype=np.int64)
    n = off.size - 1
    g = _gen(seed)
    clusters, ds = [], []
    tries = 0
    while len(clusters) < count:
        tries += 1
        if tries > max_tries * max(count, 1):
            raise ValueError("could not find enough clusters")
        ctr = int(_uniform_below(g, 1, n)[0])
        taken = [ctr]
        level = {ctr: 0}
        head = 0
        while head < len(taken) and len(taken) < k:
            u = taken[head]
            head += 1
            for v in adj[off[u]:off[u + 1]]:
                v = int(v)
                if v not in level:
                    level[v] = level[u] + 1
                    taken.append(v)
                    if len(taken) == k:
                        break
        if len(taken) < k:
            continue
        radius = level[taken[-1]]
        members = set(taken)
        diam = 0
        for s in taken:
            lv = _bounded_bfs(off, adj, s, 2 * radius)
            diam = max(diam, max(lv[t] for t in members))
        if diam > dmax:
            continue
        clusters.append(np.asarray(taken, dtype=np.int32))
        ds.append(int(diam))
    return clusters, ds


def radius_cluster(hops, centre: int, d: int, k: int = 64, seed: int = 0) -> np.ndarray:
    """k distinct vertices (the centre first) whose pairwise hop counts are at
    most d by construction, given ``hops`` = hop counts from ``centre`` (any
    negative value = unreachable).

    With r = d // 2, members lie within r hops of the centre, so any two are
    at most 2r apart; half of them (when there are enough) are drawn at
    exactly r hops to spread the set.  For odd d one more member is taken at
    r + 1 hops, at most r + (r + 1) = d from every other.  Fewer than k
    vertices come back when the ball is smaller.
    """
    hops = np.asarray(hops)
    g = _gen(seed)
    r = d // 2
    inner = np.flatnonzero((hops >= 1) & (hops < r))
    rim = np.flatnonzero(hops == r) if r >= 1 else np.zeros(0, np.int64)
    want = k - 1 - (d % 2)

    def draw(pool, m):
        m = int(min(m, pool.size))
        if m <= 0:
            return np.zeros(0, np.int64)
        keys = _raw(g, pool.size)
        return np.sort(pool[np.argsort(keys, kind="stable")[:m]])

    from_rim = draw(rim, max(want // 2, want - inner.size))
    from_inner = draw(inner, want - from_rim.size)
    out = [np.array([centre], np.int64), from_rim, from_inner]
    if d % 2 == 1:
        out.append(draw(np.flatnonzero(hops == r + 1), 1))
    return np.concatenate(out).astype(np.int32)


def random_pairs(n: int, q: int, seed: int) -> np.ndarray:
    """``q`` uniform random vertex pairs, int32[q, 2]."""
    g = _gen(seed)
    return _uniform_below(g, 2 * q, n).astype(np.int32).reshape(q, 2)


def concat_clusters(clusters):
    """(sources_concat int32, cluster_off int32[C+1]) for the batched call."""
    sizes = np.array([len(c) for c in clusters], dtype=np.int64)
    coff = np.zeros(len(clusters) + 1, dtype=np.int32)
    np.cumsum(sizes, out=coff[1:])
    src = np.concatenate(clusters).astype(np.int32) if clusters else np.zeros(0, np.int32)
    return src, coff
