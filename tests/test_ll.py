"""Host logic of the landmark-labeling index (no GPU): the budget rule of
Section 5.3 and the distortion measure of Section 4.2."""
import numpy as np
import pytest

from paper_2410_17226_gb300 import inputs as I
from paper_2410_17226_gb300 import ll


def test_cluster_count_matches_the_papers_budget_arithmetic():
    # 1024 bytes per vertex: 60 clusters of w = 64 (17 B each), 341 of w = 8 (3 B each)
    assert ll.cluster_count(1024, 2, 64) == 60
    assert ll.cluster_count(1024, 2, 8) == 341
    assert ll.cluster_count(1024, 2, 16) == 204
    assert ll.cluster_count(1024, 2, 32) == 113


def test_select_plain_landmarks_by_degree():
    off, adj = I.rmat(10, seed=4)
    deg = np.diff(off)
    clusters, d = ll.select(off, adj, 50, w=1)
    assert d == 0 and len(clusters) == 50 and all(len(S) == 1 for S in clusters)
    picked = np.array([S[0] for S in clusters])
    assert (np.diff(deg[picked]) <= 0).all()  # non-increasing degrees
    assert deg[picked].min() >= np.sort(deg)[::-1][49]


def test_select_clusters_fit_the_word():
    off, adj = I.rmat(10, seed=4)
    for w in (8, 16, 32, 64):
        clusters, d = ll.select(off, adj, 128, w=w)
        assert d == 2 and len(clusters) == ll.cluster_count(128, 2, w)
        assert all(1 <= len(S) <= w for S in clusters)
        seen = np.concatenate(clusters)
        assert np.unique(seen).size == seen.size  # marked vertices are not reused


def test_distortion_definition():
    exact = np.array([1, 2, 4, 0, -1, 3])
    answers = np.array([1, 3, 4, 0, 0xFFFF, 0xFFFF])
    r = ll.distortion(answers, exact)
    # pairs with delta > 0 and an answer: (1,1), (3,2), (4,4): psi = 1, 1.5, 1
    assert r["pairs"] == 3 and r["unanswered"] == 1
    assert r["epsilon"] == pytest.approx((1 + 1.5 + 1) / 3 - 1)
    assert r["exact_share"] == pytest.approx(2 / 3)
    with pytest.raises(ValueError):
        ll.distortion(np.array([1]), np.array([2]))  # below the true distance
