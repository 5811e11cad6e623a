"""The rows after the core path: plain single-source BFS through the C-BFS
kernels (k = 1, d = 0, Algorithm "EdgeMap" direction optimisation) and the
d sweep (clusters of diameter up to d = 2..6), bit-exact against the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2410_17226_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PUSH_ONLY = {"pull_alpha": -1.0}
PULL_EAGER = {"pull_alpha": 1e-6}


@pytest.fixture(scope="module")
def cb():
    import __graft_entry__ as ge

    ge.build()
    from paper_2410_17226_gb300 import cbfs

    return cbfs


@pytest.mark.parametrize("graph", ["rmat14", "grid"])
@pytest.mark.parametrize("mode", [None, PUSH_ONLY, PULL_EAGER])
@pytest.mark.parametrize("slots", [1, 8])
def test_single_source_bfs_equals_oracle(cb, graph, mode, slots):
    if graph == "rmat14":
        off, adj = I.rmat(14)
    else:
        off, adj = I.road_grid(96, seed=5)
    g = cb.Graph(off, adj)
    deg = np.diff(off)
    rng = np.random.default_rng(3)
    srcs = rng.choice(np.flatnonzero(deg > 0), size=20, replace=False).astype(np.int32)
    tune = dict(mode or {}, slots=slots)
    dist, masks = g.run_batched([np.array([s], np.int32) for s in srcs], 0, tune=tune)
    assert masks.shape[1] == 0
    got = dist.cpu().numpy()
    for i, s in enumerate(srcs):
        ref = O.bfs(off, adj, int(s))
        exp = np.where(ref < 0, 255, ref).astype(np.uint8)
        assert (got[i] == exp).all(), (graph, i)


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6])
def test_d_sweep_clusters_equal_oracle(cb, d):
    off, adj = I.rmat(14, seed=7)
    g = cb.Graph(off, adj)
    deg = np.diff(off)
    cand = np.flatnonzero(deg > 0)
    rng = np.random.default_rng(100 + d)
    clusters = []
    while len(clusters) < 5:
        ctr = int(cand[rng.integers(0, cand.size)])
        S = I.radius_cluster(O.bfs(off, adj, ctr), ctr, d, k=64, seed=int(rng.integers(1 << 30)))
        if S.size >= 2:
            clusters.append(S)
    for slots in (1, 4):
        dist, masks = g.run_batched(clusters, d, tune={"slots": slots})
        for c, S in enumerate(clusters):
            od, om = O.cbfs_alg1(off, adj, S, d)
            assert (dist[c].cpu().numpy() == od).all() and (cb.as_numpy_u64(masks[c]) == om).all(), (d, slots, c)
