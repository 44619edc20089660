"""Pins for the graph-builder oracle: scipy's KD-tree for the kNN lists, a
hand trace on five points of a line (tests/golden/prune_line5.json) for the
detour counts and the pruned rows, and structural invariants on random
data."""
import json
import os

import numpy as np
from scipy.spatial import cKDTree

from oracle import INVALID
from oracle import graph as OG


def test_knn_lists_match_kdtree():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((400, 7)).astype(np.float32)
    got = OG.knn_lists(X, 12)
    _, want = cKDTree(X.astype(np.float64)).query(X.astype(np.float64), k=13)
    assert np.array_equal(got, want[:, 1:].astype(np.uint32))


def test_line_hand_trace(golden_dir):
    fx = json.load(open(os.path.join(golden_dir, "prune_line5.json")))
    X = np.array(fx["x"], np.float32)[:, None]
    knn = OG.knn_lists(X, fx["K"])
    assert knn.tolist() == fx["knn"]
    assert OG.detour_counts(knn).tolist() == fx["det"]
    assert OG.prune(knn, fx["degree"]).tolist() == fx["graph"]


def test_pruned_rows_are_valid_and_keep_the_least_detoured_half():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((300, 6)).astype(np.float32)
    knn = OG.knn_lists(X, 16)
    G = OG.prune(knn, 8)
    det = OG.detour_counts(knn)
    for u in range(len(X)):
        row = [int(v) for v in G[u] if v != INVALID]
        assert u not in row and len(set(row)) == len(row) == 8
        # the first half are the 4 least-detoured kNN entries, in (det, rank) order
        order = sorted(range(16), key=lambda r: (int(det[u, r]), r))
        assert row[:4] == [int(knn[u, r]) for r in order[:4]]
        assert set(row) <= set(knn[u].tolist()) | {w for w in range(len(X)) if u in G[w, :4].tolist()}
