"""Pins for the oracle: checks against facts fixed by the paper and by
mathematics, never against the oracle itself.

* the paper's worked example (Section 3.1, Figure 2 text) -> golden file;
* closed forms: paths, cycles, grids (|i - j|, min(|i-j|, n-|i-j|),
  Manhattan distance);
* textbook BFS from SciPy / NetworkX (k = 1, d = 0 reduces C-BFS to BFS);
* brute force: all-pairs distances from SciPy decoded into the definition of
  the cluster distance vector (Section 3.1) on thousands of tiny graphs;
* Corollary 1 invariants on R-MAT graphs;
* Theorem 1 counters against their definition;
* the landmark-labeling query (Section 4.2) against min over landmarks of
  APSP sums.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

import oracle as O
from paper_2410_17226_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ helpers


def apsp(off, adj):
    n = off.size - 1
    rows = np.repeat(np.arange(n), np.diff(off))
    A = sp.csr_matrix((np.ones(adj.size), (rows, adj)), shape=(n, n))
    D = shortest_path(A, method="D", unweighted=True, directed=False)
    D[np.isinf(D)] = -1
    return D.astype(np.int64)


def expected_from_distances(dist_sv, d):
    """Definition of the cluster distance vector (Section 3.1) from a
    [k, n] table of exact distances (-1 = unreachable)."""
    k, n = dist_sv.shape
    dist = np.full(n, 0xFF, dtype=np.uint8)
    masks = np.zeros((d, n), dtype=np.uint64)
    for v in range(n):
        col = dist_sv[:, v]
        if (col < 0).all():
            continue
        lo = col[col >= 0].min()
        dist[v] = lo
        for j in range(k):
            i = col[j] - lo
            if i < d:
                masks[i, v] |= np.uint64(1) << np.uint64(j)
    return dist, masks


def all_mask(k):
    return (1 << 64) - 1 if k == 64 else (1 << k) - 1


# ------------------------------------------------------------ worked example


def load_worked_example():
    names, edges, sources, d, expect = None, [], None, None, {}
    with open(os.path.join(GOLDEN, "worked_example.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "vertices":
                names = tok[1:]
            elif tok[0] == "edges":
                edges = [e.split("-") for e in tok[1:]]
            elif tok[0] == "sources":
                sources = tok[1:]
            elif tok[0] == "d":
                d = int(tok[1])
            elif tok[0] == "expect":
                expect[tok[1]] = (int(tok[2]), tok[3:])
    return names, edges, sources, d, expect


def test_worked_example_figure2():
    names, edges, sources, d, expect = load_worked_example()
    idx = {nm: i for i, nm in enumerate(names)}
    off, adj = I.from_edges(len(names), [idx[a] for a, b in edges], [idx[b] for a, b in edges])
    S = np.array([idx[s] for s in sources], dtype=np.int32)
    bit = {s: 1 << j for j, s in enumerate(sources)}

    def setbits(txt):
        return 0 if txt == "-" else sum(bit[x] for x in txt.split(","))

    for fn in (O.cbfs_definition, O.cbfs_alg1):
        dist, masks = fn(off, adj, S, d)
        for nm, (dd, subsets) in expect.items():
            v = idx[nm]
            assert dist[v] == dd, (fn.__name__, nm)
            stored = [setbits(t) for t in subsets]
            for i in range(d):
                assert int(masks[i, v]) == stored[i], (fn.__name__, nm, i)
            implied = all_mask(len(sources)) & ~int(np.bitwise_or.reduce(masks[:, v]))
            assert implied == stored[d], (fn.__name__, nm)
    # the sentence of Section 3.1: S_F[1] = {A, C}, so A and C are at distance 2 from F
    dist, masks = O.cbfs_alg1(off, adj, S, d)
    assert int(masks[1, idx["F"]]) == bit["A"] | bit["C"]
    assert dist[idx["F"]] + 1 == 2


# -------------------------------------------------------------- closed forms


@pytest.mark.parametrize("fn", [O.cbfs_definition, O.cbfs_alg1])
def test_path_closed_form(fn):
    n = 50
    off, adj = I.path(n)
    for start, k in [(0, 1), (10, 3), (20, 7), (47, 3), (0, 16), (30, 16)]:
        S = np.arange(start, start + k, dtype=np.int32)
        d = k - 1
        table = np.abs(S[:, None].astype(np.int64) - np.arange(n)[None, :])
        ed, em = expected_from_distances(table, d)
        dist, masks = fn(off, adj, S, d)
        assert (dist == ed).all() and (masks == em).all()


@pytest.mark.parametrize("fn", [O.cbfs_definition, O.cbfs_alg1])
def test_cycle_closed_form(fn):
    n = 37
    off, adj = I.cycle(n)
    S = np.array([5, 6, 4, 7], dtype=np.int32)  # arc 4..7: pairwise distance <= 3
    d = 3
    a = np.arange(n)
    table = np.stack([np.minimum(np.abs(a - s), n - np.abs(a - s)) for s in S])
    ed, em = expected_from_distances(table, d)
    dist, masks = fn(off, adj, S, d)
    assert (dist == ed).all() and (masks == em).all()


@pytest.mark.parametrize("fn", [O.cbfs_definition, O.cbfs_alg1])
def test_grid_manhattan_closed_form(fn):
    w, h = 23, 17
    off, adj = I.grid(w, h)
    cx, cy = 8, 9
    pts = [(cx, cy), (cx + 1, cy), (cx - 1, cy), (cx, cy + 1), (cx, cy - 1), (cx + 1, cy + 1)]
    S = np.array([y * w + x for x, y in pts], dtype=np.int32)
    d = 3  # max pairwise Manhattan distance among pts is 3
    xs, ys = np.arange(w * h) % w, np.arange(w * h) // w
    table = np.stack([np.abs(xs - x) + np.abs(ys - y) for x, y in pts])
    ed, em = expected_from_distances(table, d)
    dist, masks = fn(off, adj, S, d)
    assert (dist == ed).all() and (masks == em).all()


# ---------------------------------------------------------------- textbook BFS


def test_bfs_matches_scipy_and_networkx():
    nx = pytest.importorskip("networkx")
    for seed in range(20):
        off, adj = I.erdos_renyi(200, 260, seed)
        D = apsp(off, adj)
        G = nx.Graph()
        G.add_nodes_from(range(200))
        rows = np.repeat(np.arange(200), np.diff(off))
        G.add_edges_from(zip(rows.tolist(), adj.tolist()))
        for src in (0, 17, 199):
            bd = O.bfs(off, adj, src)
            assert (bd == D[src]).all()
            ref = nx.single_source_shortest_path_length(G, src)
            assert all(bd[v] == ref.get(v, -1) for v in range(200))


@pytest.mark.parametrize("fn", [O.cbfs_definition, O.cbfs_alg1])
def test_single_source_is_textbook_bfs(fn):
    off, adj = I.rmat(10, seed=11)
    D = apsp(off, adj)
    for src in (0, 5, 1000):
        dist, masks = fn(off, adj, np.array([src], np.int32), 0)
        assert masks.shape == (0, off.size - 1)
        want = np.where(D[src] < 0, 0xFF, D[src]).astype(np.uint8)
        assert (dist == want).all()


# ------------------------------------------------------ brute force, tiny graphs


def random_cluster(D, rng, kmax=64):
    """A valid cluster from a random centre's neighbourhood, with its exact
    diameter as d (or a larger bound)."""
    n = D.shape[0]
    c = int(rng.integers(n))
    reach = np.flatnonzero((D[c] >= 0) & (D[c] <= int(rng.integers(1, 4))))
    k = int(min(reach.size, rng.integers(1, kmax + 1)))
    S = rng.choice(reach, size=k, replace=False).astype(np.int32)
    sub = D[np.ix_(S, S)]
    d = int(sub.max()) + int(rng.integers(0, 2))
    return S, min(d, 15)


def test_definition_and_alg1_match_brute_force_tiny():
    rng = np.random.default_rng(20241017)
    cases = 0
    for t in range(1500):
        n = int(rng.integers(1, 48))
        m = int(rng.integers(0, 3 * n + 1))
        off, adj = I.erdos_renyi(n, m, seed=1000 + t)
        D = apsp(off, adj)
        S, d = random_cluster(D, rng)
        table = D[S]
        ed, em = expected_from_distances(table, d)
        for fn in (O.cbfs_definition, O.cbfs_alg1):
            dist, masks = fn(off, adj, S, d)
            assert (dist == ed).all(), (t, fn.__name__)
            assert (masks == em).all(), (t, fn.__name__)
        cases += 1
    assert cases == 1500


def test_counters_match_definition():
    """Theorem 1's work measures: V = sum_i |F_i| = number of (v, i) with
    S_v[i] non-empty; A = the same weighted by deg(v)."""
    rng = np.random.default_rng(7)
    for t in range(200):
        n = int(rng.integers(2, 60))
        off, adj = I.erdos_renyi(n, int(rng.integers(n, 4 * n)), seed=5000 + t)
        D = apsp(off, adj)
        S, d = random_cluster(D, rng)
        _, _, cnt = O.cbfs_alg1(off, adj, S, d, with_counters=True)
        deg = np.diff(off)
        table = D[S]
        V = A = reached = 0
        for v in range(n):
            col = table[:, v]
            if (col < 0).all():
                continue
            distinct = np.unique(col)
            V += distinct.size
            A += distinct.size * deg[v]
            reached += deg[v]
        assert cnt["V"] == V and cnt["A"] == A and cnt["reached_arcs"] == reached
        assert cnt["rounds"] == table.max() + 1


# ------------------------------------------------------------- invariants


@pytest.mark.parametrize("seed", [1, 2])
def test_corollary1_invariants_rmat(seed):
    off, adj = I.rmat(12, seed=seed)
    clusters, d = I.star_clusters(off, adj, 4, seed=seed, size="uniform")
    n = off.size - 1
    rows = np.repeat(np.arange(n), np.diff(off))
    for S in clusters:
        k = S.size
        dist, masks = O.cbfs_alg1(off, adj, S, d)
        reach = dist != 0xFF
        # |Delta_u - Delta_v| <= 1 along every edge, reachability closed under edges
        du, dv = dist[rows].astype(int), dist[adj].astype(int)
        both = reach[rows] & reach[adj]
        assert (np.abs(du - dv)[both] <= 1).all()
        assert (reach[rows] == reach[adj]).all()
        # subsets disjoint, union = ALL, S_v[0] non-empty; unreachable -> empty
        union = np.bitwise_or.reduce(masks, axis=0)
        assert (masks[0][reach] != 0).all()
        assert (union[~reach] == 0).all()
        assert ((masks[0] & masks[1]) == 0).all()
        assert (union & ~np.uint64(all_mask(k)) == 0).all()
        # every source at offset 0 of itself
        for j, s in enumerate(S):
            assert dist[s] == 0 and (int(masks[0, s]) >> j) & 1
        assert O.certify(off, adj, S, d, dist, masks) == -1


# -------------------------------------------------------------- certificate


def test_certificate_accepts_exact_and_rejects_corruption():
    rng = np.random.default_rng(3)
    off, adj = I.rmat(10, seed=4)
    clusters, d = I.star_clusters(off, adj, 6, seed=9)
    for S in clusters:
        dist, masks = O.cbfs_definition(off, adj, S, d)
        assert O.certify(off, adj, S, d, dist, masks) == -1
        reach = np.flatnonzero(dist != 0xFF)
        for _ in range(20):
            dd, mm = dist.copy(), masks.copy()
            v = int(rng.choice(reach))
            kind = int(rng.integers(3))
            if kind == 0:
                dd[v] = (int(dd[v]) + 1) % 255
            elif kind == 1:
                j = int(rng.integers(S.size))
                i = int(rng.integers(d))
                mm[i, v] ^= np.uint64(1) << np.uint64(j)
            else:
                mm[[0, 1], v] = mm[[1, 0], v]
                if mm[0, v] == masks[0, v]:
                    continue
            assert O.certify(off, adj, S, d, dd, mm) != -1


# --------------------------------------------------------------- error paths


def test_error_codes():
    off, adj = I.path(10)
    with pytest.raises(O.OracleError) as e:
        O.cbfs_definition(off, adj, np.array([0, 5], np.int32), 2)  # distance 5 > d
    assert e.value.code == O.DIAMETER
    for bad in ([], list(range(65)), [1, 1], [-1], [10]):
        for fn in (O.cbfs_definition, O.cbfs_alg1):
            with pytest.raises(O.OracleError) as e:
                fn(off, adj, np.array(bad, np.int32), 2)
            assert e.value.code == O.INVALID
    off, adj = I.path(300)
    for fn in (O.cbfs_definition, O.cbfs_alg1):
        with pytest.raises(O.OracleError) as e:
            fn(off, adj, np.array([0], np.int32), 0)
        assert e.value.code == O.DEPTH
    off, adj = I.path(255)
    dist, _ = O.cbfs_alg1(off, adj, np.array([0], np.int32), 0)
    assert dist[254] == 254


# ---------------------------------------------------------------- the query


def brute_query(D, landmarks, pairs):
    out = []
    for u, v in pairs:
        if u == v:
            out.append(0)
            continue
        best = None
        for s in landmarks:
            if D[s, u] >= 0 and D[s, v] >= 0:
                t = D[s, u] + D[s, v]
                best = t if best is None else min(best, t)
        out.append(0xFFFF if best is None else best)
    return np.array(out, dtype=np.uint16)


def test_query_matches_landmark_definition():
    rng = np.random.default_rng(5)
    for t in range(40):
        n = int(rng.integers(5, 80))
        off, adj = I.erdos_renyi(n, int(rng.integers(n // 2, 3 * n)), seed=9000 + t)
        D = apsp(off, adj)
        C = int(rng.integers(1, 5))
        clusters, ds = [], []
        for _ in range(C):
            S, d = random_cluster(D, rng)
            clusters.append(S)
            ds.append(d)
        d = max(ds)
        dist = np.zeros((C, n), np.uint8)
        masks = np.zeros((C, d, n), np.uint64)
        for c, S in enumerate(clusters):
            dist[c], masks[c] = O.cbfs_alg1(off, adj, S, d)
        pairs = rng.integers(0, n, size=(60, 2)).astype(np.int32)
        pairs[:5, 1] = pairs[:5, 0]
        got = O.query(dist, masks, [len(S) for S in clusters], pairs)
        want = brute_query(D, np.concatenate(clusters), pairs)
        assert (got == want).all(), t
        # one-sided and exact when an endpoint is a landmark
        fin = (got != 0xFFFF)
        assert (got[fin] >= D[pairs[fin, 0], pairs[fin, 1]]).all()
        L = np.concatenate(clusters)
        for u in L[:5]:
            vs = rng.integers(0, n, size=10)
            q = O.query(dist, masks, [len(S) for S in clusters], np.stack([np.full(10, u), vs], 1))
            exact = np.where(D[u, vs] < 0, 0xFFFF, D[u, vs])
            assert (q == exact).all()


def test_label_rows_layout():
    C, n, d = 3, 4, 2
    rng = np.random.default_rng(1)
    dist = rng.integers(0, 255, size=(C, n)).astype(np.uint8)
    masks = rng.integers(0, 2 ** 63, size=(C, d, n)).astype(np.uint64)
    rows = O.label_rows(dist, masks)
    P = 8
    assert rows.shape == (n, P + 8 * d * C)
    for v in range(n):
        assert (rows[v, :C] == dist[:, v]).all() and (rows[v, C:P] == 0).all()
        blk = rows[v, P:].view(np.uint64).reshape(d, C)
        assert (blk == masks[:, :, v].T).all()


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6])
def test_radius_cluster_diameter_bound(d):
    """The d-sweep clusters: every pair of members within d hops (checked by
    BFS from each member), centre first, distinct, and for odd d one member
    at (d + 1) / 2 hops from the centre."""
    off, adj = I.rmat(10, seed=3)
    deg = np.diff(off)
    cand = np.flatnonzero(deg > 0)
    rng = np.random.default_rng(d)
    for _ in range(4):
        ctr = int(cand[rng.integers(0, cand.size)])
        hops = O.bfs(off, adj, ctr)
        S = I.radius_cluster(hops, ctr, d, k=64, seed=5)
        assert S[0] == ctr and len(set(S.tolist())) == S.size <= 64
        for v in S:
            hv = O.bfs(off, adj, int(v))
            assert (hv[S] >= 0).all() and hv[S].max() <= d
        if d % 2 and (hops == d // 2 + 1).any():
            assert (hops[S] == d // 2 + 1).sum() == 1


def _path_ball(u, n, tau):
    """Whole BFS levels around u on a path of n vertices, at most tau vertices."""
    ball = {u}
    h = 0
    while True:
        h += 1
        nxt = {x for x in (u - h, u + h) if 0 <= x < n}
        if not nxt or len(ball) + len(nxt) > tau:
            return ball
        ball |= nxt


@pytest.mark.parametrize("tau", [1, 2, 3, 4, 7])
def test_local_search_closed_form_on_a_path(tau):
    """Appendix B's bounded bidirectional search on a path of 12 vertices:
    the answer is |u - v| when the two whole-level balls meet, else none."""
    n = 12
    off, adj = I.path(n)
    pairs = np.array([(u, v) for u in range(n) for v in range(n)], np.int32)
    got = O.local_search(off, adj, pairs, tau)
    for (u, v), a in zip(pairs, got):
        if u == v:
            assert a == 0
        elif _path_ball(u, n, tau) & _path_ball(v, n, tau):
            assert a == abs(u - v), (u, v, tau)
        else:
            assert a == 0xFFFF, (u, v, tau)


def test_local_search_whole_levels_on_a_star():
    # centre 0, leaves 1..9; tau = 5: a leaf's ball is {leaf, 0} (the next
    # level, 8 leaves, would overflow and is dropped as a whole)
    src = np.zeros(9, np.int64)
    dst = np.arange(1, 10)
    off, adj = I.from_edges(10, src, dst)
    got = O.local_search(off, adj, np.array([[1, 2], [0, 5], [3, 3]], np.int32), 5)
    assert got.tolist() == [2, 1, 0]
    # the centre's ball is {0} alone (its first level has 9 vertices)
    assert O.local_search(off, adj, np.array([[0, 1]], np.int32), 9).tolist() == [1]
    assert O.local_search(off, adj, np.array([[0, 1]], np.int32), 1).tolist() == [0xFFFF]


def test_local_search_unbounded_is_exact():
    """tau >= n: the balls are whole components, so the answer is the BFS
    distance (SciPy), 0xFFFF between components."""
    off, adj = I.erdos_renyi(300, 330, seed=4)
    n = off.size - 1
    rng = np.random.default_rng(0)
    pairs = rng.integers(0, n, size=(400, 2)).astype(np.int32)
    A = sp.csr_matrix((np.ones(adj.size), adj, off), shape=(n, n))
    D = shortest_path(A, unweighted=True)
    got = O.local_search(off, adj, pairs, n)
    for (u, v), a in zip(pairs, got):
        exp = 0xFFFF if np.isinf(D[u, v]) else int(D[u, v])
        assert a == exp
