"""GPU parity: the CUDA path (through the C ABI) against the oracle, bit for
bit.  C-BFS is exact integer/bitwise work, so every byte of dist and every
bit of every subset word must match.
"""
import numpy as np
import pytest

import oracle as O
from paper_2410_17226_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PUSH_ONLY = {"pull_alpha": -1.0}
PULL_EAGER = {"pull_alpha": 1e-9}


@pytest.fixture(scope="module")
def cb():
    import __graft_entry__ as ge

    ge.build()
    from paper_2410_17226_gb300 import cbfs

    return cbfs


def check_one(cb, g, off, adj, S, d, tune=None, oracle_fn=O.cbfs_alg1):
    od, om = oracle_fn(off, adj, S, d)
    if tune is None:
        dist, masks = g.run(S, d)
    else:
        dist, masks = g.run_batched([S], d, tune=tune)
        dist, masks = dist[0], masks[0]
    gd = dist.cpu().numpy()
    gm = cb.as_numpy_u64(masks)
    bad = np.flatnonzero(gd != od)
    assert bad.size == 0, f"dist differs at {bad[:5]}: gpu {gd[bad[:5]]} oracle {od[bad[:5]]}"
    bad = np.argwhere(gm != om)
    assert bad.size == 0, f"masks differ at {bad[:5].tolist()}"


def random_cluster(off, adj, rng, kmax=64, hops=2):
    """Sources within `hops` of a random centre; d = 2 * hops bounds them."""
    n = off.size - 1
    c = int(rng.integers(n))
    dist = O.bfs(off, adj, c)
    reach = np.flatnonzero((dist >= 0) & (dist <= hops))
    k = int(min(reach.size, rng.integers(1, kmax + 1)))
    S = rng.choice(reach, size=k, replace=False).astype(np.int32)
    return S, min(2 * hops, 15)


def test_tiny_random_graphs_all_modes(cb):
    rng = np.random.default_rng(2410)
    for t in range(150):
        n = int(rng.integers(1, 300))
        off, adj = I.erdos_renyi(n, int(rng.integers(0, 4 * n + 1)), seed=77 + t)
        g = cb.Graph(off, adj)
        S, d = random_cluster(off, adj, rng, hops=int(rng.integers(0, 3)))
        if S.size > 1 and d == 0:
            d = 2
        for tune in (None, PUSH_ONLY, PULL_EAGER):
            check_one(cb, g, off, adj, S, d, tune, oracle_fn=O.cbfs_definition)
        g.close()


def test_config1_rmat_scale14_star_clusters(cb):
    """R-MAT scale 14, edge factor 16, a random vertex plus up to 63 neighbours, d = 2."""
    off, adj = I.rmat(14)
    g = cb.Graph(off, adj)
    clusters, d = I.star_clusters(off, adj, 6, seed=I.MASTER_SEED + 1)
    for S in clusters:
        for tune in (None, PUSH_ONLY, PULL_EAGER):
            check_one(cb, g, off, adj, S, d, tune)


def test_general_d_and_ball_clusters(cb):
    off, adj = I.road_grid(96, seed=5)
    g = cb.Graph(off, adj)
    clusters, ds = I.ball_clusters(off, adj, 4, 64, seed=9)
    for S, d in zip(clusters, ds):
        for tune in (None, PUSH_ONLY):
            check_one(cb, g, off, adj, S, d, tune)
    # larger d on a power-law graph
    off, adj = I.rmat(12, seed=3)
    g = cb.Graph(off, adj)
    rng = np.random.default_rng(1)
    for hops in (1, 2, 3):
        S, d = random_cluster(off, adj, rng, hops=hops)
        check_one(cb, g, off, adj, S, d)


def test_batched_equals_single_and_oracle(cb):
    off, adj = I.rmat(12, seed=21)
    g = cb.Graph(off, adj)
    clusters, d = I.star_clusters(off, adj, 19, seed=4, size="uniform")
    single = [g.run(S, d) for S in clusters]
    for tune in (None, {"slots": 1}, {"slots": 3}, {"slots": 16}, dict(PUSH_ONLY, slots=4),
                 dict(PULL_EAGER, slots=5), {"slots": 8, "host_loop": 1}, {"slots": 2, "dense_div": -1},
                 {"slots": 4, "dense_div": 1}, dict(PUSH_ONLY, slots=8, host_loop=1),
                 dict(PULL_EAGER, slots=4, fused_pull=1), {"slots": 8, "fused_pull": 1, "host_loop": 1}):
        # the first call of a shape runs host-driven, a repeat replays a CUDA graph
        for rep in range(2):
            bd, bm = g.run_batched(clusters, d, tune=tune)
            for c, (sd, sm) in enumerate(single):
                assert torch.equal(bd[c], sd), (tune, rep, c)
                assert torch.equal(bm[c], sm), (tune, rep, c)
    for c, S in enumerate(clusters):
        od, om = O.cbfs_alg1(off, adj, S, d)
        assert (single[c][0].cpu().numpy() == od).all()
        assert (cb.as_numpy_u64(single[c][1]) == om).all()


@pytest.mark.parametrize("stage_rounds", [-1, 1, 2, 5, 0])
def test_fused_round_records_at_every_cap(cb, stage_rounds):
    """Waves with fused pulls record each round's new sources and write the
    outputs from the records after the wave; a wave with more rounds than
    recorded writes them from the records at the cap and directly after it;
    stage_rounds = -1 writes directly from the start (outputs cleared first).
    Replayed graphs, host-driven rounds (bounded waves that may run again)
    and eager pulls all equal the oracle on a road grid (tens of rounds) and
    on R-MAT."""
    for graph in ("grid", "rmat"):
        if graph == "grid":
            off, adj = I.road_grid(48, seed=I.MASTER_SEED + 2)
            clusters, ds = I.ball_clusters(off, adj, 6, 16, seed=5)
            d = max(ds)
        else:
            off, adj = I.rmat(12, seed=29)
            clusters, d = I.star_clusters(off, adj, 6, seed=9, size="uniform")
        g = cb.Graph(off, adj)
        want = [O.cbfs_alg1(off, adj, S, d) for S in clusters]
        for tune in ({"slots": 4}, {"slots": 2, "host_loop": 1}, dict(PULL_EAGER, slots=4)):
            t = dict(tune, fused_pull=1, stage_rounds=stage_rounds)
            for rep in range(2):
                bd, bm = g.run_batched(clusters, d, tune=t)
                for c, (od, om) in enumerate(want):
                    assert (bd[c].cpu().numpy() == od).all(), (graph, t, rep, c)
                    assert (cb.as_numpy_u64(bm[c]) == om).all(), (graph, t, rep, c)


@pytest.mark.parametrize("tune", [{"slots": 4}, {"slots": 2, "host_loop": 1}, {"slots": 4, "stage_rounds": 2},
                                  {"slots": 4, "fused_pull": 1}, dict(PULL_EAGER, slots=8),
                                  {"slots": 1, "stage_rounds": 3, "host_loop": 1}])
def test_packed_waves_equal_oracle(cb, tune):
    """Clusters that fill only part of a 64-bit word share words (packed
    waves): 70 clusters of 1..64 sources (many small, some sharing source
    vertices), each compared with the oracle; the same call without packing
    gives the same outputs.  stage_rounds 2 / 3: the words' outputs come from
    two or three rounds of records and directly, member by member, after."""
    off, adj = I.rmat(12, seed=31)
    g = cb.Graph(off, adj)
    stars, d = I.star_clusters(off, adj, 60, seed=12, size="uniform")
    clusters = list(stars) + [stars[3][: max(1, len(stars[3]) // 2)], stars[5], stars[7][:1]] * 3
    clusters.append(np.array([int(np.argmax(np.diff(off)))], np.int32))
    want = [O.cbfs_alg1(off, adj, S, d) for S in clusters]
    for rep in range(2):
        bd, bm = g.run_batched(clusters, d, tune=tune)
        for c, (od, om) in enumerate(want):
            assert (bd[c].cpu().numpy() == od).all(), (tune, rep, c)
            assert (cb.as_numpy_u64(bm[c]) == om).all(), (tune, rep, c)
    ud, um = g.run_batched(clusters, d, tune=dict(tune, pack=-1))
    assert torch.equal(ud, bd) and torch.equal(um, bm)


def test_packed_single_sources_and_errors(cb):
    """64 single-source clusters at d = 0 (31 to a word), then 0-diameter
    clusters packed with one whose sources are 4 apart at d = 2: the call
    reports CBFS_E_DIAMETER, and the handle's next call is exact."""
    off, adj = I.rmat(11, seed=33)
    g = cb.Graph(off, adj)
    deg = np.diff(off)
    singles = [np.array([v], np.int32) for v in np.flatnonzero(deg > 0)[:64]]
    bd, bm = g.run_batched(singles, 0, tune={"slots": 2})
    for c, S in enumerate(singles):
        od, _ = O.cbfs_alg1(off, adj, S, 0)
        assert (bd[c].cpu().numpy() == od).all(), c
    poff, padj = I.path(60)
    gp = cb.Graph(poff, padj)
    bad = [np.array([v], np.int32) for v in range(10)] + [np.array([20, 24], np.int32)]
    with pytest.raises(cb.CbfsError) as e:
        gp.run_batched(bad, 2, tune={"slots": 2})
    assert e.value.code == cb.E_DIAMETER
    ok = [np.array([v], np.int32) for v in range(10)] + [np.array([20, 22], np.int32)]
    bd, bm = gp.run_batched(ok, 2, tune={"slots": 2})
    for c, S in enumerate(ok):
        od, om = O.cbfs_alg1(poff, padj, S, 2)
        assert (bd[c].cpu().numpy() == od).all() and (cb.as_numpy_u64(bm[c]) == om).all(), c


def test_waves_grouped_by_size_or_in_call_order(cb):
    """Clusters of mixed sizes: the default groups them into waves by size,
    wave_order = 1 keeps the call order; both, host-driven and replayed,
    equal the oracle cluster by cluster (outputs stay at the call's
    positions whatever wave a cluster ran in)."""
    off, adj = I.rmat(12, seed=23)
    g = cb.Graph(off, adj)
    stars, d = I.star_clusters(off, adj, 11, seed=8, size="max", min_deg=63)
    sizes = [1, 64, 2, 33, 5, 64, 1, 7, 3, 40, 2]
    clusters = [S[:k] for S, k in zip(stars, sizes)]
    want = [O.cbfs_alg1(off, adj, S, d) for S in clusters]
    for tune in ({"slots": 4}, {"slots": 4, "wave_order": 1}, {"slots": 8, "host_loop": 1},
                 {"slots": 2, "wave_order": 1, "host_loop": 1}):
        for rep in range(2):
            bd, bm = g.run_batched(clusters, d, tune=tune)
            for c, (od, om) in enumerate(want):
                assert (bd[c].cpu().numpy() == od).all() and (cb.as_numpy_u64(bm[c]) == om).all(), (tune, rep, c)


def test_graph_replay_with_new_sources_each_call(cb):
    """A cached graph replays a call shape; the sources of every call are
    uploaded before the replay, so different clusters of the same shape give
    their own results."""
    off, adj = I.rmat(12, seed=5)
    g = cb.Graph(off, adj)
    for seed in range(4):
        clusters, d = I.star_clusters(off, adj, 6, seed=100 + seed, size="max")
        clusters = [c[:5] if len(c) >= 5 else c for c in clusters]
        if any(len(c) != 5 for c in clusters):
            continue
        bd, bm = g.run_batched(clusters, d, tune={"slots": 2})
        for c, S in enumerate(clusters):
            od, om = O.cbfs_alg1(off, adj, S, d)
            assert (bd[c].cpu().numpy() == od).all() and (cb.as_numpy_u64(bm[c]) == om).all(), (seed, c)


def test_host_loop_reruns_waves_deeper_than_the_first(cb):
    """Host-driven rounds: waves after the first enqueue about as many rounds
    as the first needed; a deeper wave is detected and traversed again."""
    off, adj = I.path(240)
    g = cb.Graph(off, adj)
    clusters = [np.array([120, 121], np.int32), np.array([0, 1], np.int32), np.array([60], np.int32),
                np.array([239, 238], np.int32)]
    for tune in ({"slots": 1, "host_loop": 1}, {"slots": 2, "host_loop": 1}):
        bd, bm = g.run_batched(clusters, 2, tune=tune)
        for c, S in enumerate(clusters):
            od, om = O.cbfs_alg1(off, adj, S, 2)
            assert (bd[c].cpu().numpy() == od).all() and (cb.as_numpy_u64(bm[c]) == om).all(), (tune, c)


def test_hubs_and_big_lists(cb):
    # a star with 10000 leaves plus a path hanging off it: hub lists go
    # through the big-list pieces in push and the CTA-per-vertex pull
    leaves = 10000
    src = np.concatenate([np.zeros(leaves, np.int64), np.arange(leaves, leaves + 40)])
    dst = np.concatenate([np.arange(1, leaves + 1), np.arange(leaves + 1, leaves + 41)])
    n = leaves + 41
    off, adj = I.from_edges(n, src, dst)
    g = cb.Graph(off, adj)
    for S, d in (([0] + list(range(1, 64)), 2), ([5, 0, 7], 2), ([leaves + 20, leaves + 21], 1), ([3], 0)):
        S = np.array(S, np.int32)
        for tune in (None, PUSH_ONLY, PULL_EAGER):
            check_one(cb, g, off, adj, S, d, tune, oracle_fn=O.cbfs_definition)


def test_edge_cases(cb):
    # single vertex, no edges
    off, adj = I.from_edges(1, [], [])
    g = cb.Graph(off, adj)
    check_one(cb, g, off, adj, np.array([0], np.int32), 0)
    check_one(cb, g, off, adj, np.array([0], np.int32), 3)
    # isolated source among others, unreachable components
    off, adj = I.from_edges(10, [1, 2, 5], [2, 3, 6])
    g = cb.Graph(off, adj)
    check_one(cb, g, off, adj, np.array([0], np.int32), 0)
    check_one(cb, g, off, adj, np.array([2, 1, 3], np.int32), 2)
    # k = 64 exactly (all bits), d = 1 clique
    src, dst = np.triu_indices(70, 1)
    off, adj = I.from_edges(70, src, dst)
    g = cb.Graph(off, adj)
    check_one(cb, g, off, adj, np.arange(64, dtype=np.int32), 1)
    # deepest representable distance: 254 on a path
    off, adj = I.path(255)
    g = cb.Graph(off, adj)
    check_one(cb, g, off, adj, np.array([0], np.int32), 0)
    check_one(cb, g, off, adj, np.array([0, 1, 2], np.int32), 2)


@pytest.mark.parametrize("stage", [0, 2, 200, -1])
def test_fused_waves_report_depth_and_diameter(cb, stage):
    """Fused waves with round records: a first visit past distance 254 and a
    source pair farther apart than d are reported whether the outputs come
    from the records (stage 0 = default, 200), from two rounds of records and
    then directly (2), or directly (-1); the deepest representable distance,
    254, still works, and a call after an error on the same handle is exact
    (an error a call returns is not reported again by the next one)."""
    off, adj = I.path(300)
    g = cb.Graph(off, adj)
    for host_loop, alpha in ((0, 0.0), (1, 0.0), (0, 1e-9), (1, 1e-9)):  # pushes on a path, or pulls
        tune = {"slots": 1, "fused_pull": 1, "stage_rounds": stage, "host_loop": host_loop, "pull_alpha": alpha}
        with pytest.raises(cb.CbfsError) as e:
            g.run_batched([np.array([0], np.int32)], 0, tune=tune)
        assert e.value.code == cb.E_DEPTH
        with pytest.raises(cb.CbfsError) as e:
            g.run_batched([np.array([10, 14], np.int32)], 2, tune=tune)
        assert e.value.code == cb.E_DIAMETER
        check_one(cb, g, off, adj, np.array([45, 46, 47], np.int32), 2, tune)
    off, adj = I.path(255)
    g = cb.Graph(off, adj)
    check_one(cb, g, off, adj, np.array([0, 1, 2], np.int32), 2,
              {"slots": 2, "fused_pull": 1, "stage_rounds": stage, "pull_alpha": 1e-9})


def test_error_paths(cb):
    off, adj = I.path(300)
    g = cb.Graph(off, adj)
    with pytest.raises(cb.CbfsError) as e:
        g.run([0], 0)  # distance 299 does not fit one byte
    assert e.value.code == cb.E_DEPTH
    offs, adjs = I.path(50)
    gs = cb.Graph(offs, adjs)
    with pytest.raises(cb.CbfsError) as e:
        gs.run([10, 14], 2)  # pairwise distance 4 > d
    assert e.value.code == cb.E_DIAMETER
    for bad_S, bad_d in (([], 2), (list(range(65)), 2), ([1, 1], 2), ([-1], 2), ([300], 2), ([1], 16), ([1], -1)):
        with pytest.raises(cb.CbfsError) as e:
            g.run(bad_S, bad_d)
        assert e.value.code == cb.E_INVALID
    # sources in two components: not a cluster of diameter d
    off2, adj2 = I.from_edges(6, [0, 1, 3, 4], [1, 2, 4, 5])
    g2 = cb.Graph(off2, adj2)
    with pytest.raises(cb.CbfsError) as e:
        g2.run([0, 3], 5)
    assert e.value.code == cb.E_DIAMETER
    # graph validation
    bad_off = np.array([0, 1, 1], np.int64)
    bad_adj = np.array([1], np.int32)  # arc 0->1 without 1->0
    with pytest.raises(cb.CbfsError) as e:
        cb.Graph(bad_off, bad_adj, validate=True)
    assert e.value.code == cb.E_GRAPH
    with pytest.raises(cb.CbfsError) as e:
        cb.Graph(np.array([0, 2], np.int64), np.array([0, 0], np.int32), validate=True)
    assert e.value.code == cb.E_GRAPH
    # the handles stay usable after errors
    check_one(cb, gs, offs, adjs, np.array([10, 11, 12], np.int32), 2)


def test_device_inputs_and_int32_offsets(cb):
    off, adj = I.rmat(11, seed=8)
    S = I.star_clusters(off, adj, 1, seed=3)[0][0]
    g1 = cb.Graph(torch.from_numpy(off).cuda(), torch.from_numpy(adj).cuda())
    g2 = cb.Graph(off.astype(np.int32), adj)
    for g in (g1, g2):
        check_one(cb, g, off, adj, S, 2)


def test_output_stats_match_oracle_counters(cb):
    off, adj = I.rmat(12, seed=13)
    g = cb.Graph(off, adj)
    clusters, d = I.star_clusters(off, adj, 5, seed=6, size="uniform")
    bd, bm = g.run_batched(clusters, d)
    st = g.output_stats(bd, bm, [len(S) for S in clusters], d)
    for c, S in enumerate(clusters):
        _, _, cnt = O.cbfs_alg1(off, adj, S, d, with_counters=True)
        assert st[c].tolist() == [cnt["V"], cnt["A"], cnt["reached_arcs"], cnt["rounds"]]


def test_graph_replay_after_the_seed_buffer_grows(cb):
    """Cached CUDA graphs hold the seed buffer's address: a larger call that
    reallocates it must retire them, and later calls of an old shape with
    new sources must still be exact."""
    off, adj = I.rmat(12, seed=8)
    g = cb.Graph(off, adj)
    deg = np.diff(off)
    order = np.argsort(-deg, kind="stable")
    small = [np.array([int(order[i])] + [int(x) for x in adj[off[order[i]]:off[order[i]] + 4]], np.int32)
             for i in (10, 20, 30)]
    big = [np.array([int(order[0])] + [int(x) for x in adj[off[order[0]]:off[order[0]] + 40]], np.int32)]
    for S in (small[0], small[0], small[0]):  # first sighting, capture, replay
        dd, dm = g.run_batched([S], 2)
    g.run_batched(big * 3, 2)  # more seeds than ever: the buffer moves
    for S in (small[1], small[1], small[2]):
        dd, dm = g.run_batched([S], 2)
        od, om = O.cbfs_alg1(off, adj, S, 2)
        assert (dd[0].cpu().numpy() == od).all() and (cb.as_numpy_u64(dm[0]) == om).all()


@pytest.mark.parametrize("small,mid", [(1, 1), (8, 64), (32, 32), (16, 4096), (32, 2048), (4, 300), (32, 65536)])
def test_pull_degree_classes_equal_oracle(cb, small, mid):
    """Runtime degree classes of the dense edge phase (thread per vertex up to
    `small`, warp up to `mid`, CTA pieces above): bit-exact for every pair,
    including the degenerate ones, on a power-law graph, a hub graph and a
    grid, switching classes between calls on one handle."""
    leaves = 10000
    src = np.concatenate([np.zeros(leaves, np.int64), np.arange(leaves, leaves + 40)])
    dst = np.concatenate([np.arange(1, leaves + 1), np.arange(leaves + 1, leaves + 41)])
    cases = [("rmat", I.rmat(14, seed=13)), ("hub", I.from_edges(leaves + 41, src, dst)), ("grid", I.road_grid(80, seed=3))]
    for name, (off, adj) in cases:
        g = cb.Graph(off, adj)
        if name == "grid":
            clusters, ds = I.ball_clusters(off, adj, 5, 12, seed=5)
            d = max(ds)
        else:
            clusters, d = I.star_clusters(off, adj, 6, seed=small + mid, size="uniform")
        for slots in (1, 4, 8):
            for tune in ({"slots": slots, "pull_alpha": 1e-9, "small_deg": small, "mid_deg": mid},
                         {"slots": slots, "small_deg": small, "mid_deg": mid, "host_loop": 1},
                         {"slots": slots, "pull_alpha": 1e-9, "small_deg": small, "mid_deg": mid,
                          "sparse_mid_deg": -1},  # the same classes in every pull round
                         {"slots": slots, "pull_alpha": 1e-9, "small_deg": small, "mid_deg": mid,
                          "sparse_mid_deg": max(small, 40)},  # other classes in sparse rounds
                         {"slots": slots, "pull_alpha": 1e-9, "small_deg": small, "mid_deg": mid,
                          "fused_pull": 1},  # the last hub piece does the hub's vertex phase
                         {"slots": slots, "pull_alpha": 1e-9}):  # back to the defaults
                for _ in range(2):
                    dist, masks = g.run_batched(clusters, d, tune=tune)
                for c, S in enumerate(clusters):
                    od, om = O.cbfs_alg1(off, adj, S, d)
                    assert (dist[c].cpu().numpy() == od).all() and (cb.as_numpy_u64(masks[c]) == om).all(), \
                        (name, small, mid, tune, c)


def test_pull_degree_classes_reject_bad_thresholds(cb):
    off, adj = I.rmat(10, seed=1)
    g = cb.Graph(off, adj)
    clusters, d = I.star_clusters(off, adj, 2, seed=1)
    for small, mid in ((33, 64), (8, 4), (8, 65537), (-1, 64)):
        with pytest.raises(cb.CbfsError) as e:
            g.run_batched(clusters, d, tune={"small_deg": small, "mid_deg": mid})
        assert e.value.code == cb.E_INVALID


def test_empty_graph_and_empty_calls(cb):
    """n = 0: the graph builds, every source is out of range, zero clusters
    and zero pairs are no-ops; on a small graph, zero clusters write nothing."""
    off = np.zeros(1, np.int64)
    adj = np.zeros(0, np.int32)
    g = cb.Graph(off, adj)
    assert g.n == 0 and g.nnz == 0
    with pytest.raises(cb.CbfsError) as e:
        g.run([0], 2)
    assert e.value.code == cb.E_INVALID
    dist, masks = g.run_batched([], 2)
    assert dist.shape == (0, 0) and masks.shape == (0, 2, 0)
    L = cb.Labels(0, 1, 2)
    out = L.query(torch.zeros((0, 2), dtype=torch.int32, device="cuda"))
    assert out.numel() == 0 and L.status() == cb.OK
    off2, adj2 = I.path(20)
    g2 = cb.Graph(off2, adj2)
    d2 = torch.full((1, 20), 7, dtype=torch.uint8, device="cuda")
    m2 = torch.full((1, 2, 20), 7, dtype=torch.int64, device="cuda")
    g2.run_batched([], 2, d2, m2)
    assert int(d2.min()) == 7 and int(m2.min()) == 7  # untouched


@pytest.mark.parametrize("slots,fused_pull", [(1, 0), (4, 0), (4, 1)])
def test_largest_diameter_bound(cb, slots, fused_pull):
    """d = 15, the largest bound: sources 15 apart on a path and a grid
    ball of diameter up to 15; every offset 0..15 occurs."""
    off, adj = I.path(60)
    g = cb.Graph(off, adj)
    clusters = [np.array([10, 25], np.int32), np.array([0, 5, 15], np.int32), np.array([40, 55, 47], np.int32)]
    dist, masks = g.run_batched(clusters, 15, tune={"slots": slots, "fused_pull": fused_pull})
    for c, S in enumerate(clusters):
        od, om = O.cbfs_alg1(off, adj, S, 15)
        assert (dist[c].cpu().numpy() == od).all() and (cb.as_numpy_u64(masks[c]) == om).all()
    goff, gadj = I.grid(20, 20)
    gg = cb.Graph(goff, gadj)
    S = np.array([0, 7, 8 * 20], np.int32)  # (0,0), (7,0), (0,8): 7, 8 and 15 apart
    gd, gm = gg.run_batched([S], 15, tune={"slots": slots, "fused_pull": fused_pull})
    od, om = O.cbfs_alg1(goff, gadj, S, 15)
    assert (gd[0].cpu().numpy() == od).all() and (cb.as_numpy_u64(gm[0]) == om).all()
