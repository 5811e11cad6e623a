"""Stream-ordered calls and cbfs_sync_status.

Traversals with device outputs, the label append and the query only enqueue
work; a caller can queue several of them on one stream and synchronise once.
Errors the kernels detect stay in the handle's status word until
cbfs_sync_status (per stream) or cbfs_graph_status (per handle) reads them.
"""
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


def test_queued_traversals_append_and_query_with_one_sync(cb):
    """Six batched calls of different shapes (more than the four upload
    buffers the handle rotates through), a label append of the last call's
    outputs and a query, all on one stream, then one cbfs_sync_status."""
    off, adj = I.rmat(14)
    n = off.size - 1
    g = cb.Graph(off, adj)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    calls = []
    for i in range(6):
        clusters, d = I.star_clusters(off, adj, 3 + 2 * i, seed=I.MASTER_SEED + 200 + i, size="uniform")
        dist = torch.empty((len(clusters), n), dtype=torch.uint8, device="cuda")
        masks = torch.empty((len(clusters), d, n), dtype=torch.int64, device="cuda")
        g.run_batched(clusters, d, dist, masks, tune={"slots": 4 if i % 2 else 2}, stream=s, check=False)
        calls.append((clusters, d, dist, masks))
    clusters, d, dist, masks = calls[-1]
    L = cb.Labels(n, len(clusters), d)
    ks = [len(S) for S in clusters]
    L.append(dist, masks, ks, stream=s)
    pairs = I.random_pairs(n, 3000, seed=3)
    pairs_d = torch.from_numpy(pairs).cuda()
    s.wait_stream(torch.cuda.current_stream())
    ans = L.query(pairs_d, stream=s)
    assert cb.sync_status(s) == cb.OK
    for clusters, d, dist, masks in calls:
        for c, S in enumerate(clusters):
            od, om = O.cbfs_alg1(off, adj, S, d)
            assert (dist[c].cpu().numpy() == od).all() and (cb.as_numpy_u64(masks[c]) == om).all()
    od = np.stack([O.cbfs_alg1(off, adj, S, d)[0] for S in clusters])
    om = np.stack([O.cbfs_alg1(off, adj, S, d)[1] for S in clusters])
    assert (cb.as_numpy_u16(ans) == O.query(od, om, ks, pairs)).all()


def test_device_errors_surface_at_sync_status(cb):
    """A cluster whose diameter exceeds d, queued without a check: the call
    returns OK, the stream's status is CBFS_E_DIAMETER once, then OK; a
    later call on the same handle is exact."""
    off, adj = I.path(50)
    g = cb.Graph(off, adj)
    s = torch.cuda.Stream()
    g.run([10, 14], 2, stream=s, check=False)  # pairwise distance 4 > d = 2
    assert cb.sync_status(s) == cb.E_DIAMETER
    assert cb.sync_status(s) == cb.OK
    dist, masks = g.run([10, 11, 12], 2, stream=s)
    od, om = O.cbfs_alg1(off, adj, [10, 11, 12], 2)
    assert (dist.cpu().numpy() == od).all() and (cb.as_numpy_u64(masks) == om).all()
    # per handle: the error sticks until this handle's status is read
    g.run([10, 14], 2, stream=s, check=False)
    assert g.status(stream=s) == cb.E_DIAMETER and g.status(stream=s) == cb.OK


def test_an_unread_error_is_returned_by_the_next_blocking_call(cb):
    """An error left by a stream-ordered call is reported by the handle's
    next blocking call (host outputs block)."""
    off, adj = I.path(50)
    g = cb.Graph(off, adj)
    s = torch.cuda.Stream()
    g.run([10, 14], 2, stream=s, check=False)
    hd = torch.empty(50, dtype=torch.uint8).pin_memory()
    hm = torch.empty((2, 50), dtype=torch.int64).pin_memory()
    with pytest.raises(cb.CbfsError) as e:
        g.run([10, 11], 2, hd, hm, stream=s, check=False)
    assert e.value.code == cb.E_DIAMETER
    g.run([10, 11], 2, hd, hm, stream=s)
    od, om = O.cbfs_alg1(off, adj, [10, 11], 2)
    assert (hd.numpy() == od).all() and (hm.numpy().view(np.uint64) == om).all()
