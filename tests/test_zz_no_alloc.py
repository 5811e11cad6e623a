"""The allocation-free entry point cbfs_run_noalloc.

It serves callers that cannot allocate device memory (a process whose GPU
memory is owned by another allocator, or a loop where cudaMalloc/cudaFree
must not run): its scratch is a fixed array inside the library.  Its outputs
must equal those of the allocating entry point cbfs_run bit for bit, on two
calls in a row -- the second call checks that what the first call left in the
shared array does not leak into the next result.  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_2410_17226_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    import __graft_entry__ as ge

    ge.build()
    from paper_2410_17226_gb300 import cbfs

    off, adj = I.rmat(14)
    n = off.size - 1
    g = cbfs.Graph(off, adj)
    off_d = torch.from_numpy(off).cuda()
    adj_d = torch.from_numpy(adj).cuda()
    clusters, d = I.star_clusters(off, adj, 2, seed=I.MASTER_SEED + 77)
    # the second call uses a smaller cluster, so stale bits from the first would show
    clusters[1] = clusters[1][:5]
    for S in clusters:
        ref_dist, ref_masks = g.run(S, d)
        dist = torch.empty(n, dtype=torch.uint8, device="cuda")
        masks = torch.empty((d, n), dtype=torch.int64, device="cuda")
        cbfs.run_noalloc(off_d, adj_d, S, d, dist, masks)
        torch.cuda.synchronize()
        assert torch.equal(dist, ref_dist)
        assert torch.equal(masks, ref_masks)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import __graft_entry__ as ge

    ge.build()
    from paper_2410_17226_gb300 import cbfs

    off, adj = I.rmat(18)  # 262,144 vertices > 131,072
    off_d = torch.from_numpy(off).cuda()
    adj_d = torch.from_numpy(adj).cuda()
    n = off.size - 1
    dist = torch.empty(n, dtype=torch.uint8, device="cuda")
    masks = torch.empty((2, n), dtype=torch.int64, device="cuda")
    with pytest.raises(cbfs.CbfsError) as e:
        cbfs.run_noalloc(off_d, adj_d, np.array([0], np.int32), 2, dist, masks)
    assert e.value.code == cbfs.E_NOMEM
