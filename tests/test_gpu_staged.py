"""Batched C-BFS with outputs in host memory, and label rows written by the
traversal itself (cbfs_run_batched_labels): the same bits as device outputs
and as cbfs_labels_append, checked against the oracle on sample clusters.
Also the device-side graph set-up (offset checks, degree order)."""
import numpy as np
import pytest

import oracle as O
from paper_2410_17226_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cb():
    import __graft_entry__ as ge

    ge.build()
    from paper_2410_17226_gb300 import cbfs

    return cbfs


def rows_of(L, n):
    """Host copy of a label store's rows (uint8 [n, stride])."""
    ptr, stride = L.rows()

    class _Rows:
        __cuda_array_interface__ = {"shape": (n, stride), "typestr": "|u1", "data": (ptr, False), "version": 3}

    return torch.as_tensor(_Rows(), device="cuda").cpu().numpy()


def valid_columns(rows, count, cap, d):
    """The bytes of the first `count` clusters in every row: the distance
    bytes and each subset block (layout [dist cap | pad to 8 | d x cap u64])."""
    P = (cap + 7) // 8 * 8
    parts = [rows[:, :count]]
    for s in range(d):
        a = P + 8 * s * cap
        parts.append(rows[:, a:a + 8 * count])
    return np.concatenate(parts, axis=1)


@pytest.mark.parametrize("slots,host_loop,fused,stage", [(1, 0, 0, 0), (2, 1, 0, 0), (4, 0, 0, 0), (8, 0, 0, 0),
                                                        (4, 0, 1, 0), (2, 1, 1, 0), (4, 1, 1, 2), (4, 0, 1, -1)])
def test_host_outputs_equal_device_outputs(cb, slots, host_loop, fused, stage):
    """fused: fused pulls, whose waves write their outputs (into the staging
    ring for host outputs) from their round records after the wave, or with
    stage = 2 from two rounds of records and directly after them, or with
    stage = -1 directly as they arise, instead of emitting internal rows."""
    off, adj = I.rmat(12, seed=5)
    clusters, d = I.star_clusters(off, adj, 19, seed=3, size="uniform")
    g = cb.Graph(off, adj)
    tune = {"slots": slots, "host_loop": host_loop, "fused_pull": fused, "stage_rounds": stage}
    dd, dm = g.run_batched(clusters, d, tune=tune)
    C, n = len(clusters), g.n
    ref_d, ref_m = dd.cpu(), dm.cpu()
    pin_d = torch.empty((C, n), dtype=torch.uint8).pin_memory()
    pin_m = torch.empty((C, d, n), dtype=torch.int64).pin_memory()
    for _ in range(2):  # twice in a row: the two staging buffers are reused
        pin_d.fill_(7)
        pin_m.fill_(7)
        g.run_batched(clusters, d, pin_d, pin_m, tune=tune)
        assert torch.equal(pin_d, ref_d) and torch.equal(pin_m, ref_m)
    # page-locked buffers from the library's own allocator
    lib_d = cb.pinned_empty((C, n), torch.uint8)
    lib_m = cb.pinned_empty((C, d, n), torch.int64)
    g.run_batched(clusters, d, lib_d, lib_m, tune=tune)
    assert torch.equal(lib_d, ref_d) and torch.equal(lib_m, ref_m)
    del lib_d, lib_m
    page_d = torch.full((C, n), 7, dtype=torch.uint8)
    page_m = torch.full((C, d, n), 7, dtype=torch.int64)
    g.run_batched(clusters, d, page_d, page_m, tune=tune)
    assert torch.equal(page_d, ref_d) and torch.equal(page_m, ref_m)
    od, om = O.cbfs_alg1(off, adj, clusters[C - 1], d)
    assert (pin_d[C - 1].numpy() == od).all() and (pin_m[C - 1].numpy().view(np.uint64) == om).all()


def test_single_run_into_host_memory(cb):
    off, adj = I.rmat(11, seed=4)
    clusters, d = I.star_clusters(off, adj, 2, seed=9, size="max")
    g = cb.Graph(off, adj)
    hd = torch.empty(g.n, dtype=torch.uint8).pin_memory()
    hm = torch.empty((d, g.n), dtype=torch.int64).pin_memory()
    g.run(clusters[1], d, hd, hm)
    od, om = O.cbfs_alg1(off, adj, clusters[1], d)
    assert (hd.numpy() == od).all() and (hm.numpy().view(np.uint64) == om).all()


def test_labels_fed_by_the_traversal_equal_append(cb):
    off, adj = I.rmat(11, seed=2)
    clusters, d = I.degree_clusters(off, adj, 37)
    ks = [len(S) for S in clusters]
    C = len(clusters)
    g = cb.Graph(off, adj)
    n = g.n
    L1 = cb.Labels(n, 40, d)
    dd, dm = g.run_batched(clusters, d)
    L1.append(dd, dm, ks)
    L2 = cb.Labels(n, 40, d)
    g.run_batched_labels(clusters[:10], d, L2, tune={"slots": 4})  # labels only
    hd = torch.empty((C - 10, n), dtype=torch.uint8).pin_memory()
    hm = torch.empty((C - 10, d, n), dtype=torch.int64).pin_memory()
    g.run_batched_labels(clusters[10:], d, L2, dist=hd, masks=hm, tune={"slots": 8})
    assert L2.count == C
    assert torch.equal(hd, dd[10:].cpu()) and torch.equal(hm, dm[10:].cpu())
    L3 = cb.Labels(n, 40, d)
    dev_d = torch.empty((C, n), dtype=torch.uint8, device="cuda")
    dev_m = torch.empty((C, d, n), dtype=torch.int64, device="cuda")
    g.run_batched_labels(clusters, d, L3, dist=dev_d, masks=dev_m, tune={"slots": 2, "host_loop": 1})
    assert torch.equal(dev_d, dd) and torch.equal(dev_m, dm)
    r1 = valid_columns(rows_of(L1, n), C, 40, d)
    assert (valid_columns(rows_of(L2, n), C, 40, d) == r1).all()
    assert (valid_columns(rows_of(L3, n), C, 40, d) == r1).all()
    pairs = I.random_pairs(n, 5000, seed=3)
    pt = torch.from_numpy(pairs).cuda()
    a1 = cb.as_numpy_u16(L1.query(pt))
    assert (cb.as_numpy_u16(L2.query(pt)) == a1).all()
    # and the answers against the oracle's query over the same clusters
    od = np.zeros((C, n), np.uint8)
    om = np.zeros((C, d, n), np.uint64)
    for i, S in enumerate(clusters):
        od[i], om[i] = O.cbfs_alg1(off, adj, S, d)
    assert (a1 == O.query(od, om, ks, pairs)).all()


def test_labels_errors_leave_the_store_unchanged(cb):
    off, adj = I.rmat(10, seed=6)
    clusters, d = I.degree_clusters(off, adj, 8)
    g = cb.Graph(off, adj)
    small = cb.Labels(g.n, 5, d)
    with pytest.raises(cb.CbfsError) as e:
        g.run_batched_labels(clusters[:6], d, small)
    assert e.value.code == cb.E_NOMEM and small.count == 0
    g.run_batched_labels(clusters[:5], d, small)
    assert small.count == 5
    wrong_d = cb.Labels(g.n, 8, d + 1)
    with pytest.raises(cb.CbfsError) as e:
        g.run_batched_labels(clusters, d, wrong_d)
    assert e.value.code == cb.E_INVALID and wrong_d.count == 0
    # a star of three or more sources needs d = 2: with d = 1 the call fails
    # after the traversal and the reservation is undone
    star = [S for S in clusters if len(S) >= 3][:1]
    L1 = cb.Labels(g.n, 4, 1)
    with pytest.raises(cb.CbfsError) as e:
        g.run_batched_labels(star, 1, L1)
    assert e.value.code == cb.E_DIAMETER and L1.count == 0


def test_offsets_are_checked_on_the_device(cb):
    adj = np.array([1, 0, 2, 1], np.int32)  # path 0 - 1 - 2
    good = np.array([0, 1, 3, 4], np.int64)
    cb.Graph(good, adj, validate=False).close()
    for bad in ([0, 3, 1, 4], [1, 1, 3, 4], [0, 1, 3, 3]):
        for dtype in (np.int64, np.int32):
            with pytest.raises(cb.CbfsError) as e:
                cb.Graph(np.array(bad, dtype), adj, validate=False)
            assert e.value.code == cb.E_GRAPH
            with pytest.raises(cb.CbfsError) as e:
                cb.Graph(torch.tensor(bad, dtype=torch.int64 if dtype == np.int64 else torch.int32).cuda(),
                         torch.from_numpy(adj).cuda(), validate=False)
            assert e.value.code == cb.E_GRAPH


@pytest.mark.parametrize("shape", ["ties", "hubs", "isolated"])
def test_degree_order_on_skewed_graphs(cb, shape):
    """Degree orders that take one radix pass with every degree tied (cycle),
    three passes (a hub of degree 70,000 and one of 300), and many isolated
    vertices: outputs equal the oracle's (Section 3.1 definition)."""
    if shape == "ties":
        off, adj = I.cycle(401)
    elif shape == "hubs":
        n = 70300
        src = np.concatenate([np.zeros(70000, np.int64), np.ones(298, np.int64), np.arange(2, n - 1)])
        dst = np.concatenate([np.arange(2, 70002), np.arange(70002, n), np.arange(3, n)])
        off, adj = I.from_edges(n, src, dst)
        assert np.diff(off).max() >= 70000
    else:
        off, adj = I.erdos_renyi(20000, 12000, seed=5)
        assert (np.diff(off) == 0).sum() > 5000
    g = cb.Graph(off, adj)
    clusters, ds = I.ball_clusters(off, adj, 3, 8, seed=11)
    d = max(ds)
    dist, masks = g.run_batched(clusters, d, tune={"slots": 2})
    for c, S in enumerate(clusters):
        od, om = O.cbfs_definition(off, adj, S, d)
        assert (dist[c].cpu().numpy() == od).all() and (cb.as_numpy_u64(masks[c]) == om).all()


@pytest.mark.parametrize("slots,fused,stage", [(1, 0, 0), (2, 0, 0), (2, 1, 0), (2, 1, 3)])
def test_labels_and_host_outputs_with_rerun_waves(cb, slots, fused, stage):
    """Waves deeper than the first are traversed again at the end of the call
    (host-driven rounds); their host copies and label rows are rewritten.
    With one cluster per wave the label groups span many waves.  fused: the
    waves write their outputs into the staging ring from their round records
    (96 rounds by default, 3 with stage = 3: waves of up to 239 rounds are
    flushed at the last recorded round and write directly after it)."""
    off, adj = I.path(240)
    g = cb.Graph(off, adj)
    base = [np.array([120, 121], np.int32), np.array([0, 1], np.int32), np.array([60], np.int32),
            np.array([239, 238], np.int32)]
    clusters = base * 10  # 40 clusters: groups of 32 / slots waves, a ragged last group
    C, n, d = len(clusters), g.n, 2
    L = cb.Labels(n, C, d)
    hd = torch.empty((C, n), dtype=torch.uint8).pin_memory()
    hm = torch.empty((C, d, n), dtype=torch.int64).pin_memory()
    tune = {"slots": slots, "fused_pull": fused, "stage_rounds": stage}
    g.run_batched_labels(clusters, d, L, dist=hd, masks=hm, tune=tune)
    od = np.zeros((C, n), np.uint8)
    om = np.zeros((C, d, n), np.uint64)
    for c, S in enumerate(clusters):
        od[c], om[c] = O.cbfs_alg1(off, adj, S, d)
    assert (hd.numpy() == od).all() and (hm.numpy().view(np.uint64) == om).all()
    L2 = cb.Labels(n, C, d)
    g.run_batched_labels(clusters, d, L2, tune=tune)  # labels only (wave ring)
    L3 = cb.Labels(n, C, d)
    L3.append(torch.from_numpy(od).cuda(), torch.from_numpy(om.view(np.int64)).cuda(), [len(S) for S in clusters])
    ref = valid_columns(rows_of(L3, n), C, C, d)
    assert (valid_columns(rows_of(L, n), C, C, d) == ref).all()
    assert (valid_columns(rows_of(L2, n), C, C, d) == ref).all()


def _csr(n, arcs):
    arcs = sorted(arcs)
    off = np.zeros(n + 1, np.int64)
    for a, _ in arcs:
        off[a + 1] += 1
    return np.cumsum(off), np.array([b for _, b in arcs], np.int32)


def test_graph_check_by_counting(cb):
    """Symmetry is checked by searching the reverse of every arc that points
    to a later vertex of the degree order and by counting those arcs: a
    missing reverse on either side must fail, symmetric graphs must pass."""
    star = [(0, v) for v in range(1, 6)] + [(v, 0) for v in range(1, 6)]
    off, adj = _csr(7, star)
    cb.Graph(off, adj, validate=True).close()
    # hub -> isolated vertex without its reverse: found missing by the search
    off, adj = _csr(7, star + [(0, 6)])
    with pytest.raises(cb.CbfsError) as e:
        cb.Graph(off, adj, validate=True)
    assert e.value.code == cb.E_GRAPH
    # low-degree vertex -> hub without its reverse: only the count sees it
    off, adj = _csr(7, star + [(6, 0)])
    with pytest.raises(cb.CbfsError) as e:
        cb.Graph(off, adj, validate=True)
    assert e.value.code == cb.E_GRAPH
    # two equal-degree vertices joined one way only (ties broken by id, both directions)
    for a, b in ((3, 4), (4, 3)):
        off, adj = _csr(7, star + [(a, b)])
        with pytest.raises(cb.CbfsError) as e:
            cb.Graph(off, adj, validate=True)
        assert e.value.code == cb.E_GRAPH
    # an extra symmetric edge keeps it valid; random symmetric graphs pass
    off, adj = _csr(7, star + [(3, 4), (4, 3)])
    cb.Graph(off, adj, validate=True).close()
    for seed in range(3):
        off, adj = I.erdos_renyi(500, 1500, seed=seed)
        cb.Graph(off, adj, validate=True).close()
    # an arc swapped for another endpoint keeps every degree but breaks symmetry
    off, adj = I.rmat(10, seed=1)
    adj2 = adj.copy()
    v = int(np.argmax(np.diff(off) == 1))  # a vertex of degree 1
    u = int(adj2[off[v]])
    w = next(x for x in range(off.size - 1) if x not in (v, u) and x not in set(adj[off[v]:off[v + 1]]))
    adj2[off[v]] = w
    with pytest.raises(cb.CbfsError) as e:
        cb.Graph(off, adj2, validate=True)
    assert e.value.code == cb.E_GRAPH
