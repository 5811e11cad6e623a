"""The bounded bidirectional search fused into the query (Appendix B):
bit-exact against the oracle alone (no labels) and fused with label stores
(answer = min of the two), on graphs that stress deep balls (paths), dropped
levels (stars, hubs) and ordinary sparse graphs."""
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


def graphs():
    yield "path", I.path(3000)
    src = np.concatenate([np.zeros(500, np.int64), np.arange(1, 500)])
    dst = np.concatenate([np.arange(1, 501), np.arange(501, 1000)])
    yield "star_with_tails", I.from_edges(1001, src, dst)
    yield "rmat12", I.rmat(12, seed=9)
    yield "grid", I.road_grid(64, seed=3)


@pytest.mark.parametrize("tau", [1, 3, 64, 512, 2048])
def test_local_search_alone_equals_oracle(cb, tau):
    for name, (off, adj) in graphs():
        g = cb.Graph(off, adj)
        n = g.n
        rng = np.random.default_rng(tau)
        pairs = rng.integers(0, n, size=(1500, 2)).astype(np.int32)
        pairs[:100, 1] = pairs[:100, 0]  # u == v
        nb = adj[np.minimum(off[pairs[100:300, 0]], adj.size - 1)]  # some adjacent pairs
        has = np.diff(off)[pairs[100:300, 0]] > 0
        pairs[100:300, 1] = np.where(has, nb, pairs[100:300, 1])
        got = cb.as_numpy_u16(g.query_local(torch.from_numpy(pairs).cuda(), tau))
        exp = O.local_search(off, adj, pairs, tau)
        assert (got == exp).all(), (name, tau, np.flatnonzero(got != exp)[:5])


@pytest.mark.parametrize("w", [8, 64])
@pytest.mark.parametrize("tau", [16, 256])
def test_local_search_fused_with_labels(cb, w, tau):
    from paper_2410_17226_gb300 import ll

    off, adj = I.rmat(12, seed=3)
    g = cb.Graph(off, adj)
    clusters, d = ll.select(off, adj, 40, w=w)
    L, _ = ll.build(g, clusters, d, w)
    pairs = I.random_pairs(g.n, 3000, seed=tau + w)
    got = cb.as_numpy_u16(g.query_local(torch.from_numpy(pairs).cuda(), tau, labels=L))
    od = np.zeros((len(clusters), g.n), np.uint8)
    om = np.zeros((len(clusters), d, g.n), np.uint64)
    for c, S in enumerate(clusters):
        od[c], om[c] = O.cbfs_alg1(off, adj, S, d)
    lab = O.query(od, om, [len(S) for S in clusters], pairs)
    loc = O.local_search(off, adj, pairs, tau)
    assert (got == np.minimum(lab, loc)).all()
    assert (got <= cb.as_numpy_u16(L.query(torch.from_numpy(pairs).cuda()))).all()


def test_local_search_arguments(cb):
    off, adj = I.path(50)
    g = cb.Graph(off, adj)
    p = torch.tensor([[0, 3], [1, 60]], dtype=torch.int32, device="cuda")
    for tau in (0, 2049):
        with pytest.raises(cb.CbfsError) as e:
            g.query_local(p, tau)
        assert e.value.code == cb.E_INVALID
    L = cb.Labels(g.n, 2, 2)
    got = cb.as_numpy_u16(g.query_local(p, 8, labels=L))
    assert got.tolist() == [3, 0xFFFF]
    assert L.status() == cb.E_INVALID and L.status() == cb.OK
    other = cb.Labels(g.n + 1, 2, 2)
    with pytest.raises(cb.CbfsError):
        g.query_local(p, 8, labels=other)
