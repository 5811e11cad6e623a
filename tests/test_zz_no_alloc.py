"""The allocation-free entry point cbfs_run_noalloc.

Some callers cannot allocate device memory: a process whose GPU memory is
entirely owned by another allocator (a framework's caching pool), or a loop in
which cudaMalloc/cudaFree, which may block and synchronise the device, must
not run.  cbfs_run_noalloc serves them with a fixed scratch array inside the
library.  Its outputs must be the oracle's (Algorithm 1 run on the CPU) bit
for bit and equal to the allocating entry point cbfs_run, on two calls in a
row: the second call checks that what the first call left in the shared
array does not leak into the next result.  The graph is checked on the device
before the traversal reads through it.  This file is collected last so that a
run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

import oracle as O
from paper_2410_17226_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_N = 131072
MAX_NNZ = 4194304


@pytest.fixture(scope="module")
def cb():
    import __graft_entry__ as ge

    ge.build()
    from paper_2410_17226_gb300 import cbfs

    return cbfs


def _equals_oracle_and_cbfs_run(cb, g, off, adj, off_d, adj_d, S, d):
    n = off.size - 1
    dist = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
    masks = torch.full((d, n), 7, dtype=torch.int64, device="cuda")
    cb.run_noalloc(off_d, adj_d, S, d, dist, masks)
    torch.cuda.synchronize()
    od, om = O.cbfs_alg1(off, adj, S, d)
    assert (dist.cpu().numpy() == od).all(), "dist differs from the oracle"
    assert (cb.as_numpy_u64(masks) == om).all(), "masks differ from the oracle"
    ref_dist, ref_masks = g.run(S, d)
    assert torch.equal(dist, ref_dist) and torch.equal(masks, ref_masks), "differs from cbfs_run"


def test_noalloc_equals_oracle_and_allocating_entry_point_on_two_calls(cb):
    off, adj = I.rmat(14)
    g = cb.Graph(off, adj)
    off_d = torch.from_numpy(off).cuda()
    adj_d = torch.from_numpy(adj).cuda()
    clusters, d = I.star_clusters(off, adj, 2, seed=I.MASTER_SEED + 77)
    # the second call uses a smaller cluster, so stale bits from the first would show
    clusters[1] = clusters[1][:5]
    for S in clusters:
        _equals_oracle_and_cbfs_run(cb, g, off, adj, off_d, adj_d, S, d)


def test_noalloc_at_its_size_limits(cb):
    """n = 131,072 vertices (the limit) and 3.7 M arcs (89 % of the arc
    limit), 154 hubs whose lists exceed 2048 arcs (cut into pieces), 64-source
    stars (one centred on a hub) and k = 1, d = 0; then a 362 x 362 road
    grid (131,044 vertices; its shortcuts keep every distance below 255, which
    a plain grid of that size would exceed) with a 64-vertex ball and d = 15,
    the largest bound."""
    off, adj = I.rmat(17)
    n = off.size - 1
    assert n == MAX_N and MAX_NNZ * 0.85 < adj.size <= MAX_NNZ
    g = cb.Graph(off, adj)
    off_d = torch.from_numpy(off).cuda()
    adj_d = torch.from_numpy(adj).cuda()
    clusters, d = I.star_clusters(off, adj, 2, seed=I.MASTER_SEED + 77, size="max", min_deg=63)
    deg = np.diff(off)
    assert [len(S) for S in clusters] == [64, 64] and deg[clusters[1][0]] > 2048
    for S in clusters:
        _equals_oracle_and_cbfs_run(cb, g, off, adj, off_d, adj_d, S, d)
    _equals_oracle_and_cbfs_run(cb, g, off, adj, off_d, adj_d, clusters[1][:1], 0)

    goff, gadj = I.road_grid(362)
    assert MAX_N - 100 < goff.size - 1 <= MAX_N
    gg = cb.Graph(goff, gadj)
    balls, _ = I.ball_clusters(goff, gadj, 1, 64, seed=I.MASTER_SEED + 78)
    _equals_oracle_and_cbfs_run(cb, gg, goff, gadj, torch.from_numpy(goff).cuda(), torch.from_numpy(gadj).cuda(),
                                balls[0], 15)


def test_noalloc_rejects_sizes_beyond_its_scratch(cb):
    off, adj = I.rmat(18)  # 262,144 vertices > 131,072
    off_d = torch.from_numpy(off).cuda()
    adj_d = torch.from_numpy(adj).cuda()
    n = off.size - 1
    dist = torch.empty(n, dtype=torch.uint8, device="cuda")
    masks = torch.empty((2, n), dtype=torch.int64, device="cuda")
    with pytest.raises(cb.CbfsError) as e:
        cb.run_noalloc(off_d, adj_d, np.array([0], np.int32), 2, dist, masks)
    assert e.value.code == cb.E_NOMEM
    # more arcs than the scratch holds (rejected on the host, before any device work)
    n2 = 1000
    off2 = torch.zeros(n2 + 1, dtype=torch.int64, device="cuda")
    off2[-1] = MAX_NNZ + 2
    adj2 = torch.zeros(MAX_NNZ + 2, dtype=torch.int32, device="cuda")
    with pytest.raises(cb.CbfsError) as e:
        cb.run_noalloc(off2, adj2, np.array([0], np.int32), 2, dist[:n2], masks[:, :n2].contiguous())
    assert e.value.code == cb.E_NOMEM


def test_noalloc_checks_the_graph_on_the_device(cb):
    """A wrong last offset, decreasing offsets and an out-of-range neighbour id
    give CBFS_E_GRAPH before the traversal reads through them; a good call
    afterwards still equals the oracle."""
    off, adj = I.rmat(12)
    n = off.size - 1
    g = cb.Graph(off, adj)
    off_d = torch.from_numpy(off).cuda()
    adj_d = torch.from_numpy(adj).cuda()
    S = np.array([int(np.argmax(np.diff(off)))], np.int32)
    dist = torch.empty(n, dtype=torch.uint8, device="cuda")
    masks = torch.empty((2, n), dtype=torch.int64, device="cuda")
    bad_last = off_d.clone()
    bad_last[-1] -= 1
    bad_order = off_d.clone()
    bad_order[n // 2] = bad_order[n // 2 + 1] + 1
    bad_first = off_d.clone()
    bad_first[0] = 1
    bad_id = adj_d.clone()
    bad_id[adj.size // 3] = n
    neg_id = adj_d.clone()
    neg_id[7] = -1
    for o, a in ((bad_last, adj_d), (bad_order, adj_d), (bad_first, adj_d), (off_d, bad_id), (off_d, neg_id)):
        with pytest.raises(cb.CbfsError) as e:
            cb.run_noalloc(o, a, S, 2, dist, masks)
        assert e.value.code == cb.E_GRAPH
    _equals_oracle_and_cbfs_run(cb, g, off, adj, off_d, adj_d, S, 2)
