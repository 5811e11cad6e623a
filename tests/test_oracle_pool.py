"""The parallel oracle comparison used by the full-size parity tests.

Its inputs here are the definition oracle's outputs (k textbook BFSs, O1) held
in CPU tensors, standing in for CUDA outputs: equal outputs pass, and a single
flipped bit or distance anywhere in any cluster is reported.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle_pool import assert_equal_oracle, oracle_outputs
from paper_2410_17226_gb300 import inputs as I


@pytest.fixture(scope="module")
def case():
    off, adj = I.rmat(11)
    clusters, d = I.star_clusters(off, adj, 6, seed=I.MASTER_SEED + 9, size="uniform")
    n = off.size - 1
    dist = np.empty((len(clusters), n), np.uint8)
    masks = np.empty((len(clusters), d, n), np.uint64)
    for c, S in enumerate(clusters):
        dist[c], masks[c] = O.cbfs_definition(off, adj, S, d)
    return off, adj, clusters, d, dist, masks


def test_equal_outputs_pass(case):
    off, adj, clusters, d, dist, masks = case
    n_done = assert_equal_oracle(off, adj, clusters, d, torch.from_numpy(dist), torch.from_numpy(masks.view(np.int64)),
                                 range(len(clusters)), workers=3)
    assert n_done == len(clusters)
    od, om = oracle_outputs(off, adj, clusters, d, workers=2)
    assert (od == dist).all() and (om == masks).all()


@pytest.mark.parametrize("what", ["dist", "mask"])
def test_a_single_difference_is_reported(case, what):
    off, adj, clusters, d, dist, masks = case
    dist, masks = dist.copy(), masks.copy()
    rng = np.random.default_rng(3)
    c = int(rng.integers(0, len(clusters)))
    v = int(np.flatnonzero(dist[c] != 255)[rng.integers(0, (dist[c] != 255).sum())])
    if what == "dist":
        dist[c, v] ^= 1
    else:
        masks[c, 1, v] ^= np.uint64(1)
    with pytest.raises(AssertionError, match=f"cluster {c}"):
        assert_equal_oracle(off, adj, clusters, d, torch.from_numpy(dist), torch.from_numpy(masks.view(np.int64)),
                            range(len(clusters)), workers=4)
