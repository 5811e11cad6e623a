"""The landmark-labeling index on the GPU: label stores of word size
w = 8, 16, 32 (and 64) answer exactly what the oracle's query definition
gives on the same clusters, and the index is one-sided and exact through its
landmarks (Section 4.2)."""
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


@pytest.mark.parametrize("w", [1, 8, 16, 32, 64])
def test_ll_index_equals_oracle_query(cb, w):
    from paper_2410_17226_gb300 import ll

    off, adj = I.rmat(12, seed=3)
    g = cb.Graph(off, adj)
    clusters, d = ll.select(off, adj, 64, w=w)
    L, _ = ll.build(g, clusters, d, w)
    assert L.count == len(clusters)
    pairs = I.random_pairs(g.n, 4000, seed=w)
    landmark = np.concatenate(clusters)
    pairs[:200, 0] = landmark[np.arange(200) % landmark.size]  # some pairs through a landmark
    got = cb.as_numpy_u16(L.query(torch.from_numpy(pairs).cuda()))
    od = np.zeros((len(clusters), g.n), np.uint8)
    om = np.zeros((len(clusters), d, g.n), np.uint64)
    for c, S in enumerate(clusters):
        od[c], om[c] = O.cbfs_alg1(off, adj, S, d)
    ks = [len(S) for S in clusters]
    assert (got == O.query(od, om, ks, pairs)).all()
    # one-sided, and exact when u is a landmark
    for i in list(range(0, 200, 37)) + list(range(200, 4000, 397)):
        u, v = pairs[i]
        du = O.bfs(off, adj, int(u))
        if du[v] < 0:
            continue
        assert got[i] >= du[v]
        if i < 200:
            assert got[i] == du[v]


@pytest.mark.parametrize("w", [8, 16, 32])
def test_narrow_words_reject_wider_clusters(cb, w):
    off, adj = I.rmat(10, seed=2)
    g = cb.Graph(off, adj)
    clusters, d = I.degree_clusters(off, adj, 2, k=w + 1)
    assert max(len(S) for S in clusters) == w + 1
    L = cb.Labels(g.n, 4, d, w=w)
    with pytest.raises(cb.CbfsError) as e:
        g.run_batched_labels(clusters, d, L)
    assert e.value.code == cb.E_INVALID and L.count == 0
    dist, masks = g.run_batched(clusters, d)
    with pytest.raises(cb.CbfsError):
        L.append(dist, masks, [len(S) for S in clusters])
