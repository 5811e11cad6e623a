"""Parity at the full sizes of the benchmark workloads.

Each test runs the CUDA path in the launch configuration the benchmark uses
and compares clusters bit for bit with the oracle (Algorithm 1 in C, one
cluster per host core through tests/oracle_pool.py):
  * config 2 (R-MAT scale 22, 256 clusters, autotuned launch): every cluster,
    so every slot position of every wave;
  * config 3 (road grid 4096^2, 64 ball clusters): every cluster;
  * config 4 (R-MAT scale 24, 1024 clusters in launches of 32): a seeded
    sample of two clusters per launch (64), covering every slot position;
  * config 5: the served answers against the oracle's query over the
    oracle's own outputs of the same 60 clusters.
Invariants that hold for every cluster are checked on the device as well:
  * every source S[j] has Delta = 0 and bit j in S[0];
  * a vertex is unreached exactly when all its stored subsets are empty;
  * the stored subsets are disjoint and inside ALL.
"""
import numpy as np
import pytest

import oracle as O
from oracle_pool import assert_equal_oracle, assert_host_equal_oracle, host_copy, host_cores, oracle_outputs
from paper_2410_17226_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def cb():
    import __graft_entry__ as ge

    ge.build()
    from paper_2410_17226_gb300 import cbfs

    return cbfs


def assert_invariants(dist, masks, clusters):
    """dist uint8 [C, n], masks int64 [C, d, n] on the device."""
    d = masks.shape[1]
    for c, S in enumerate(clusters):
        k = len(S)
        all_ = -1 if k == 64 else (1 << k) - 1
        src = torch.as_tensor(np.asarray(S, np.int64), device=dist.device)
        assert bool((dist[c, src] == 0).all())
        bits = torch.as_tensor([1 << j if j < 63 else -(1 << 63) for j in range(k)], device=dist.device)
        if d > 0:
            assert bool(((masks[c, 0, src] & bits) == bits).all())
            union = masks[c, 0].clone()
            for i in range(1, d):
                assert bool(((union & masks[c, i]) == 0).all())
                union |= masks[c, i]
            assert bool(((union & ~torch.tensor(all_, device=dist.device)) == 0).all())
            assert bool(((dist[c] == 255) == (union == 0)).all())


def test_config2_scale22_256_clusters_batched(cb):
    """Undirected R-MAT scale 22, 256 star clusters of 1..64 sources, d = 2,
    batched with the autotuned parameters the benchmark uses (clusters packed
    several to a slot word, the default for device outputs): all 256 clusters
    equal the oracle."""
    from paper_2410_17226_gb300 import tune

    off, adj = I.rmat(22)
    clusters, d = I.star_clusters(off, adj, 256, seed=I.MASTER_SEED + 1, size="uniform")
    g = cb.Graph(off, adj)
    tn = tune.autotune(g, clusters, d, key_extra=f"rmat-s22-{tune.signature(off)}")
    tset = {"pull_alpha": tn["pull_alpha"], "slots": tn["slots"], "small_deg": tn.get("small_deg", 0),
            "mid_deg": tn.get("mid_deg", 0), "fused_pull": tn.get("fused_pull", 0)}
    dist, masks = g.run_batched(clusters, d, tune=tset)
    assert_invariants(dist, masks, clusters)
    assert assert_equal_oracle(off, adj, clusters, d, dist, masks, range(256)) == 256
    for c in (1, 77):
        sd, sm = g.run(clusters[c], d)
        assert torch.equal(sd, dist[c]) and torch.equal(sm, masks[c])


def test_config3_road_grid_4096_ball_clusters(cb):
    """4096 x 4096 grid, 10 % of edges deleted, 1 % shortcuts, 64 clusters of
    64 sources (BFS balls, d = their largest exact diameter), in launches of
    16 clusters with the benchmark's autotuned settings: all 64 clusters equal
    the oracle; two of them also with the other pull variant."""
    from paper_2410_17226_gb300 import tune

    off, adj = I.road_grid(4096)
    clusters, ds = I.ball_clusters(off, adj, 64, 64, seed=I.MASTER_SEED + 3)
    d = max(ds)
    g = cb.Graph(off, adj)
    # the benchmark's autotuned settings (the fused pull on this graph)
    tn = tune.autotune(g, clusters, d, sample=16, key_extra=f"grid-4096-{tune.signature(off)}")
    tset = {k: tn.get(k, 0) for k in ("pull_alpha", "slots", "small_deg", "mid_deg", "fused_pull")}
    checked = 0
    for b in range(0, 64, 16):
        part = clusters[b:b + 16]
        dist, masks = g.run_batched(part, d, tune=tset)
        assert_invariants(dist, masks, part)
        # at d = 12 one cluster's outputs are 1.6 GB: at most 16 on the host at once
        checked += assert_equal_oracle(off, adj, part, d, dist, masks, range(len(part)), workers=min(16, host_cores()))
        del dist, masks
    assert checked == 64
    other = dict(tset, fused_pull=0 if tset.get("fused_pull") else 1)
    dist, masks = g.run_batched(clusters[:2], d, tune=other)
    assert assert_equal_oracle(off, adj, clusters[:2], d, dist, masks, range(2)) == 2


def test_config4_scale24_1024_degree_clusters_labels(cb):
    """R-MAT scale 24 (int64 offsets), 1024 degree-ordered clusters of 64
    (Section 4.2 selection), 32 clusters per launch, labels kept on the device
    within a 1024 B/vertex budget (60 clusters of 17 B).  Two seeded clusters
    of every launch (64 in all, every slot position among them) equal the
    oracle."""
    off, adj = I.rmat(24)
    assert off.dtype == np.int64
    clusters, d = I.degree_clusters(off, adj, 1024)
    assert len(clusters) == 1024
    g = cb.Graph(off, adj)
    n = g.n
    budget = 1024 * n
    cap = budget // (n * (1 + 8 * d)) if n else 0
    L = cb.Labels(n, int(cap), d, budget_bytes=budget)
    rng = np.random.default_rng(I.MASTER_SEED + 4)
    kept, positions, got = 0, set(), {}
    for b in range(0, 1024, 32):
        part = clusters[b:b + 32]
        dist, masks = g.run_batched(part, d)
        # one position from each half of the launch, so every slot of a wave appears
        pick = [int(rng.integers(0, 16)), 16 + int(rng.integers(0, 16))]
        if b < 256:  # the first eight launches walk the positions 0..7 mod 8 in turn
            pick[0] = (b // 32) % 8
        positions.update(p % 8 for p in pick)
        for p in pick:  # compared below, all 64 at once over the host cores
            got[b + p] = host_copy(dist[p], masks[p])
        if b in (0, 992):
            assert_invariants(dist, masks, part)
        take = min(len(part), int(cap) - kept)
        if take > 0:
            L.append(dist[:take], masks[:take], [len(S) for S in part[:take]])
            kept += take
        del dist, masks
    assert len(got) == 64 and positions == set(range(8))
    assert assert_host_equal_oracle(off, adj, clusters, d, got) == 64
    del got
    assert kept == cap == L.count == 60
    pairs = I.random_pairs(n, 1000, seed=1)
    ans = cb.as_numpy_u16(L.query(torch.from_numpy(pairs).cuda()))
    assert L.status() == cb.OK
    # finite exactly when both ends lie in the landmarks' component, and never
    # below the true distance (one-sided error, Section 4.2)
    comp = O.bfs(off, adj, int(clusters[0][0])) >= 0
    both = comp[pairs[:, 0]] & comp[pairs[:, 1]]
    assert ((ans != 0xFFFF) == (both | (pairs[:, 0] == pairs[:, 1]))).all()
    for u, v in pairs[both][:3]:
        du = O.bfs(off, adj, int(u))
        a = ans[np.flatnonzero((pairs[:, 0] == u) & (pairs[:, 1] == v))[0]]
        assert a >= du[v]


def test_config5_serving_scale22_labels(cb):
    """Distance-query serving over the scale-22 graph's device-resident labels
    (60 degree-ordered clusters): Poisson arrivals of 1..65536-pair requests;
    4096 sampled pairs answered alone and in a mix of other requests equal
    the oracle's query over the oracle's outputs of the same 60 clusters."""
    from paper_2410_17226_gb300.serve import QueryServer, poisson_load

    off, adj = I.rmat(22)
    clusters, d = I.degree_clusters(off, adj, 60)
    g = cb.Graph(off, adj)
    dist, masks = g.run_batched(clusters, d)
    L = cb.Labels(g.n, 60, d)
    L.append(dist, masks, [len(S) for S in clusters])
    del dist, masks
    with QueryServer(L, max_batch=65536, slots=4) as srv:
        futs, offered, elapsed = poisson_load(srv, g.n, rate_rps=300.0, duration_s=1.0, max_pairs=65536, seed=7)
        st = srv.stats()
    assert st["requests"] == len(futs) and st["pairs"] == offered
    rng = np.random.default_rng(11)
    sample = rng.integers(0, g.n, size=(4096, 2)).astype(np.int32)
    with QueryServer(L, max_batch=65536, slots=2) as srv:
        alone = srv.submit(sample).result()
    mixed_srv = QueryServer(L, max_batch=8192, slots=4)
    noise = [mixed_srv.submit(rng.integers(0, g.n, size=(int(rng.integers(1, 20000)), 2)).astype(np.int32))
             for _ in range(8)]
    mixed = mixed_srv.submit(sample)
    for f in noise:
        f.result()
    mixed = mixed.result()
    mixed_srv.close()
    assert (alone == mixed).all()
    # the served store against the oracle: its outputs of the 60 clusters, its query
    od, om = oracle_outputs(off, adj, clusters, d)
    want = O.query(od, om, [len(S) for S in clusters], sample)
    assert (np.asarray(alone).view(np.uint16) == want).all()


def test_config2_host_outputs_and_labels_at_full_size(cb):
    """Scale-22 R-MAT: 40 clusters (a full label group of 32 and a ragged one)
    written to pinned host memory and to a label store by one
    cbfs_run_batched_labels call; sampled clusters equal the oracle and the
    label rows hold the same bytes as the host outputs."""
    off, adj = I.rmat(22)
    clusters, d = I.star_clusters(off, adj, 40, seed=I.MASTER_SEED + 5, size="uniform")
    g = cb.Graph(off, adj)
    n, C = g.n, len(clusters)
    hd = torch.empty((C, n), dtype=torch.uint8).pin_memory()
    hm = torch.empty((C, d, n), dtype=torch.int64).pin_memory()
    L = cb.Labels(n, C, d)
    g.run_batched_labels(clusters, d, L, dist=hd, masks=hm, tune={"slots": 4})
    for c in (0, 31, 39):
        od, om = O.cbfs_alg1(off, adj, clusters[c], d)
        assert (hd[c].numpy() == od).all() and (hm[c].numpy().view(np.uint64) == om).all()
    ptr, stride = L.rows()
    rng = np.random.default_rng(1)
    vs = rng.integers(0, n, 2000)

    class _Rows:
        __cuda_array_interface__ = {"shape": (n, stride), "typestr": "|u1", "data": (ptr, False), "version": 3}

    rows = torch.as_tensor(_Rows(), device="cuda")[torch.from_numpy(vs).cuda()].cpu().numpy()
    P = (C + 7) // 8 * 8
    assert (rows[:, :C] == hd.numpy()[:, vs].T).all()
    for s in range(d):
        words = rows[:, P + 8 * s * C:P + 8 * (s + 1) * C].copy().view(np.uint64)
        assert (words == hm.numpy()[:, s, vs].T.view(np.uint64)).all()
