"""GPU parity of the label layout (vertex-major rows) and of the landmark
query against the oracle: exact, including u == v, unreachable pairs and
out-of-range ids."""
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


def build_labels(cb, off, adj, clusters, d, capacity=None, chunks=1):
    g = cb.Graph(off, adj)
    L = cb.Labels(g.n, capacity or len(clusters), d)
    dists, masks = [], []
    per = (len(clusters) + chunks - 1) // chunks
    for i in range(0, len(clusters), per):
        part = clusters[i:i + per]
        bd, bm = g.run_batched(part, d)
        L.append(bd, bm, [len(S) for S in part])
        dists.append(bd.cpu().numpy())
        masks.append(cb.as_numpy_u64(bm))
    return g, L, np.concatenate(dists), np.concatenate(masks)


@pytest.mark.parametrize("chunks", [1, 3])
def test_label_rows_match_oracle_layout(cb, chunks):
    off, adj = I.rmat(11, seed=2)
    clusters, d = I.degree_clusters(off, adj, 37)
    g, L, dist, masks = build_labels(cb, off, adj, clusters, d, capacity=40, chunks=chunks)
    ptr, stride = L.rows()
    n = g.n

    class _Rows:  # wraps the device row store for torch, no copy
        __cuda_array_interface__ = {"shape": (n, stride), "typestr": "|u1", "data": (ptr, False), "version": 3}

    rows = torch.as_tensor(_Rows(), device="cuda").cpu().numpy()
    # oracle layout for capacity 40: pad the cluster axis to the capacity
    C = len(clusters)
    dpad = np.full((40, n), 0, np.uint8)
    dpad[:C] = dist
    mpad = np.zeros((40, d, n), np.uint64)
    mpad[:C] = masks
    want = O.label_rows(dpad, mpad)
    assert rows.shape == want.shape
    assert (rows == want).all()


def test_query_matches_oracle(cb):
    off, adj = I.rmat(12, seed=31)
    clusters, d = I.degree_clusters(off, adj, 20)
    g, L, dist, masks = build_labels(cb, off, adj, clusters, d)
    pairs = I.random_pairs(g.n, 5000, seed=3)
    pairs[:50, 1] = pairs[:50, 0]
    got = cb.as_numpy_u16(L.query(torch.from_numpy(pairs).cuda()))
    want = O.query(dist, masks, [len(S) for S in clusters], pairs)
    assert (got == want).all()
    assert L.status() == cb.OK


def test_query_general_d_and_star_mix(cb):
    off, adj = I.road_grid(64, seed=1)
    clusters, ds = I.ball_clusters(off, adj, 6, 40, seed=2)
    d = max(ds)
    g, L, dist, masks = build_labels(cb, off, adj, clusters, d)
    pairs = I.random_pairs(g.n, 3000, seed=4)
    got = cb.as_numpy_u16(L.query(torch.from_numpy(pairs).cuda()))
    want = O.query(dist, masks, [len(S) for S in clusters], pairs)
    assert (got == want).all()
    for dd in (1, 0):
        off1, adj1 = I.rmat(10, seed=5)
        if dd == 0:
            cl = [np.array([v], np.int32) for v in (3, 77, 500)]
        else:  # an edge (or a single vertex) has diameter <= 1
            cl = I.star_clusters(off1, adj1, 3, seed=1, kmax=2)[0]
        g1, L1, d1, m1 = build_labels(cb, off1, adj1, cl, dd)
        pr = I.random_pairs(g1.n, 2000, seed=6)
        got = cb.as_numpy_u16(L1.query(torch.from_numpy(pr).cuda()))
        want = O.query(d1, m1 if dd else np.zeros((len(cl), 0, g1.n), np.uint64), [len(S) for S in cl], pr)
        assert (got == want).all()


def test_query_edge_cases(cb):
    off, adj = I.from_edges(8, [0, 1, 4], [1, 2, 5])
    clusters = [np.array([0, 1], np.int32)]
    g, L, dist, masks = build_labels(cb, off, adj, clusters, 2)
    pairs = np.array([[0, 2], [2, 0], [3, 3], [4, 5], [0, 4], [7, 6]], np.int32)
    got = cb.as_numpy_u16(L.query(torch.from_numpy(pairs).cuda()))
    assert got.tolist() == [2, 2, 0, 0xFFFF, 0xFFFF, 0xFFFF]
    assert L.status() == cb.OK
    bad = torch.tensor([[0, 8], [-1, 2]], dtype=torch.int32, device="cuda")
    got = cb.as_numpy_u16(L.query(bad))
    assert got.tolist() == [0xFFFF, 0xFFFF]
    assert L.status() == cb.E_INVALID
    assert L.status() == cb.OK  # cleared
    empty = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    assert L.query(empty).numel() == 0
    with pytest.raises(cb.CbfsError):
        L.append(torch.zeros((1, 8), dtype=torch.uint8, device="cuda"),
                 torch.zeros((1, 2, 8), dtype=torch.int64, device="cuda"), [1])  # over capacity
    with pytest.raises(cb.CbfsError) as e:
        cb.Labels(1000, 10, 2, budget_bytes=100)
    assert e.value.code == cb.E_NOMEM
