"""Pins for the oracle's search and ground truth.

- ground truth vs scipy's exact KD-tree and vs planted duplicates (ties by id);
- a hand-traced search on 8 points (tests/golden/line8_trace.json);
- the search degenerates to brute force when the queue can hold every node
  (itopk >= n) on a connected graph, with and without DGS re-expansion, and
  for the ghost stage when the ghost set is the whole graph;
- DGS with discard 0 or cool-down 1.0 is the plain search, bit for bit;
- DGS by a similarity threshold: a hand-built star whose neighbours agree
  with the query in 8, 7, ..., 1 of 8 dimensions keeps exactly the ones at
  or above ceil(f * d), and a threshold every neighbour meets is the plain
  search.
"""
import json
import os

import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle as O


def _ring_graph(n, deg, rng):
    """Random out-neighbours plus a ring edge, so every node is reachable."""
    G = np.empty((n, deg), dtype=np.uint32)
    for i in range(n):
        others = rng.choice(np.delete(np.arange(n), [i, (i + 1) % n]), size=deg - 1, replace=False)
        G[i] = np.concatenate([[(i + 1) % n], others])
    return G


def test_knn_f64_matches_kdtree():
    rng = np.random.default_rng(10)
    X = rng.standard_normal((3000, 12)).astype(np.float32)
    Q = rng.standard_normal((40, 12)).astype(np.float32)
    ids, d = O.knn_f64(X, Q, 10)
    kd, ki = cKDTree(X.astype(np.float64)).query(Q.astype(np.float64), k=10)
    assert np.array_equal(ids, ki.astype(np.uint32))
    np.testing.assert_allclose(d, kd ** 2, rtol=1e-12)


def test_knn_f64_ties_by_smaller_id():
    X = np.zeros((6, 3), np.float32)
    X[:, 0] = [5, 1, 3, 1, 1, 9]          # ids 1, 3, 4 are all at distance 1 from q
    Q = np.zeros((1, 3), np.float32)
    ids, d = O.knn_f64(X, Q, 4)
    assert ids[0].tolist() == [1, 3, 4, 2]
    assert d[0].tolist() == [1.0, 1.0, 1.0, 9.0]


def test_line8_hand_trace(golden_dir):
    fx = json.load(open(os.path.join(golden_dir, "line8_trace.json")))
    X = np.array(fx["x"], np.float32)[:, None]
    G = np.array(fx["graph"], np.uint32)
    Q = np.array([[fx["q"]]], np.float32)
    ix = O.OracleIndex(X, G)
    assert O.splitmix64(O.splitmix64(fx["seed"])) % 8 == 0
    for case in fx["cases"]:
        ids, dists, cnt = O.search(ix, Q, seed=fx["seed"], **case["params"])
        assert ids[0].tolist() == case["ids"], case
        for f in ("iters", "parents", "dgs_parents", "vec_rows"):
            assert int(cnt[f][0]) == case[f], (f, case)
        qf = float(np.float32(fx["q"]))
        np.testing.assert_allclose(dists[0], (np.array(case["ids"]) - qf) ** 2, rtol=1e-6)


@pytest.fixture(scope="module")
def int_data():
    # integer coordinates: FP32 sums are exact (< 2^24), so FP32 and FP64
    # distances coincide and ties are exact on both sides
    rng = np.random.default_rng(11)
    n, d = 300, 16
    X = rng.integers(0, 20, size=(n, d)).astype(np.float32)
    Q = rng.integers(0, 20, size=(25, d)).astype(np.float32)
    G = _ring_graph(n, 8, rng)
    gt, gd = O.knn_f64(X, Q, 10)
    return X, Q, G, gt, gd


@pytest.mark.parametrize("kw", [
    dict(),
    dict(search_width=4),
    dict(dgs_discard=0.5, dgs_reexpand=1),
    dict(dgs_discard=0.75, dgs_reexpand=1, search_width=2),
    dict(dgs_min_match=0.6, dgs_reexpand=1),
])
def test_full_queue_equals_brute_force(int_data, kw):
    X, Q, G, gt, gd = int_data
    ix = O.OracleIndex(X, G)
    ids, dists, cnt = O.search(ix, Q, k=10, itopk=512, max_iters=2000, seed=3, **kw)
    assert np.array_equal(ids, gt)
    assert np.array_equal(dists.astype(np.float64), gd)
    assert (cnt["vec_rows"] == X.shape[0]).all()      # every node evaluated exactly once


def test_complete_graph_equals_brute_force():
    rng = np.random.default_rng(12)
    n = 40
    X = rng.integers(-5, 6, size=(n, 5)).astype(np.float32)
    Q = rng.integers(-5, 6, size=(10, 5)).astype(np.float32)
    G = np.array([[j for j in range(n) if j != i] for i in range(n)], np.uint32)
    ix = O.OracleIndex(X, G)
    ids, dists, _ = O.search(ix, Q, k=5, itopk=64, max_iters=64, seed=1)
    gt, gd = O.knn_f64(X, Q, 5)
    assert np.array_equal(ids, gt) and np.array_equal(dists.astype(np.float64), gd)


def test_dgs_discard_zero_and_full_cooldown_are_plain():
    rng = np.random.default_rng(13)
    X = rng.standard_normal((2000, 40)).astype(np.float32)
    Q = rng.standard_normal((50, 40)).astype(np.float32)
    G = _ring_graph(2000, 16, rng)
    ix = O.OracleIndex(X, G)
    base = O.search(ix, Q, k=10, itopk=32, max_iters=80, seed=9)
    for kw in (dict(dgs_discard=0.0), dict(dgs_discard=0.5, dgs_cooldown=1.0)):
        got = O.search(ix, Q, k=10, itopk=32, max_iters=80, seed=9, **kw)
        assert np.array_equal(got[0], base[0]) and np.array_equal(got[1], base[1])
        assert np.array_equal(got[2], base[2])
    # with discarding on, fewer rows are evaluated
    dgs = O.search(ix, Q, k=10, itopk=32, max_iters=80, seed=9, dgs_discard=0.5)
    assert dgs[2]["vec_rows"].sum() < base[2]["vec_rows"].sum()
    assert (dgs[2]["dgs_parents"] > 0).all()


def test_ghost_stage_over_whole_graph_is_brute_force(int_data):
    X, Q, G, gt, gd = int_data
    n = X.shape[0]
    S = np.arange(n, dtype=np.uint32)
    ix = O.OracleIndex(X, G, S=S, Gg=G)
    # ghost queue holds all n: after the ghost stage the top g are exact, and
    # a base search with a full queue stays exact
    ids, dists, cnt = O.search(ix, Q, k=10, itopk=512, max_iters=2000, entry=1, ghost_itopk=512,
                               ghost_max_iters=2000, seed=5)
    assert np.array_equal(ids, gt)
    assert (cnt["ghost_vec_rows"] == n).all()
    # with T = 0 base iterations the answer is the ghost stage's own top-k
    ids0, _, cnt0 = O.search(ix, Q, k=10, itopk=512, max_iters=0, entry=1, ghost_itopk=512,
                             ghost_max_iters=2000, seed=5)
    assert np.array_equal(ids0, gt) and (cnt0["iters"] == 0).all()
    # a ghost stage with several parents per iteration reaches the same exact
    # answer in fewer iterations
    ids3, _, cnt3 = O.search(ix, Q, k=10, itopk=512, max_iters=0, entry=1, ghost_itopk=512,
                             ghost_max_iters=2000, seed=5, ghost_search_width=3)
    assert np.array_equal(ids3, gt) and (cnt3["ghost_vec_rows"] == n).all()
    assert (cnt3["ghost_iters"] < cnt0["ghost_iters"]).all()
    assert (cnt3["ghost_parents"] <= 3 * cnt3["ghost_iters"]).all()


def test_given_ghost_seeds_and_fallback(int_data):
    X, Q, G, gt, gd = int_data
    n = X.shape[0]
    S = np.arange(0, n, 3, dtype=np.uint32)
    rng = np.random.default_rng(14)
    Gg = _ring_graph(len(S), 6, rng)
    ix = O.OracleIndex(X, G, S=S, Gg=Gg)
    seeds = rng.integers(0, len(S), size=(Q.shape[0], 4)).astype(np.uint32)
    seeds[::2, 0] = O.INVALID   # every other query falls back to random ghost seeds
    a = O.search(ix, Q, given_ghost_seeds=seeds, entry=2, k=10, itopk=32, max_iters=40, seed=2)
    b = O.search(ix, Q, entry=1, k=10, itopk=32, max_iters=40, seed=2)
    assert np.array_equal(a[0][::2], b[0][::2])          # fallback rows = plain ghost staging
    assert (a[2]["ghost_iters"][1::2] <= 4).all()        # given seeds run the short ghost stage


def test_ghost_judge_continues_exactly_the_far_queries(int_data):
    """The judge of given ghost seeds: with a distance every query's ghost
    result beats it changes nothing; with one none beats it every query runs
    the whole ghost budget, exactly as given seeds with ghost_max_iters_given
    = ghost_max_iters (continuing from the state reached is the same search);
    in between, each query takes one of the two results according to its
    own ghost result after the short stage."""
    X, Q, G, gt, gd = int_data
    n = X.shape[0]
    S = np.arange(0, n, 3, dtype=np.uint32)
    rng = np.random.default_rng(15)
    Gg = _ring_graph(len(S), 6, rng)
    ix = O.OracleIndex(X, G, S=S, Gg=Gg)
    seeds = rng.integers(0, len(S), size=(Q.shape[0], 2)).astype(np.uint32)
    common = dict(given_ghost_seeds=seeds, entry=2, k=10, itopk=32, max_iters=40, seed=3, ghost_itopk=16,
                  ghost_max_iters=12, ghost_max_iters_given=1)
    short = O.search(ix, Q, **common)
    full = O.search(ix, Q, **dict(common, ghost_max_iters_given=12))
    assert (short[2]["ghost_iters"] <= 1).all() and (full[2]["ghost_iters"] > 1).any()
    never = O.search(ix, Q, **common, ghost_judge=1e30)
    always = O.search(ix, Q, **common, ghost_judge=1e-30)
    for a, b in ((never, short), (always, full)):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert np.array_equal(a[2]["ghost_iters"], b[2]["ghost_iters"])
    # the ghost stage's own best distance after the short stage decides
    best = O.search(ix, Q, **dict(common, k=1, itopk=16, max_iters=0))[1][:, 0]
    judge = float(np.median(best))
    mid = O.search(ix, Q, **common, ghost_judge=judge)
    far = best > np.float32(judge)
    assert far.any() and (~far).any()
    assert np.array_equal(mid[0][far], full[0][far]) and np.array_equal(mid[0][~far], short[0][~far])
    assert np.array_equal(mid[2]["ghost_iters"][far], full[2]["ghost_iters"][far])
    with pytest.raises(ValueError):
        O.search(ix, Q, **common, ghost_judge=float("inf"))


def test_rerank_uses_fp32_originals():
    rng = np.random.default_rng(15)
    X = rng.standard_normal((500, 32)).astype(np.float32) * 3
    Q = rng.standard_normal((20, 32)).astype(np.float32) * 3
    G = _ring_graph(500, 12, rng)
    ix = O.OracleIndex(X, G, storage=O.E4M3)
    ids, dists, cnt = O.search(ix, Q, k=10, itopk=512, max_iters=3000, rerank=1, seed=4)
    gt, gd = O.knn_f64(X, Q, 10)
    # a full queue holds every node, so the FP32 rerank of it is exact kNN
    assert np.array_equal(ids, gt)
    np.testing.assert_allclose(dists, gd, rtol=1e-5)
    assert (cnt["rerank_rows"] == 500).all()


def test_recall_tie_aware():
    X = np.array([[0.0], [1.0], [-1.0], [2.0]], np.float32)
    Q = np.array([[0.0]], np.float32)
    gt, gd = O.knn_f64(X, Q, 2)          # [0, 1] with the tie 1/2 going to id 1
    assert gt[0].tolist() == [0, 1]
    tie_aware, strict = O.recall_at_k(np.array([[0, 2]]), gt, gd, X, Q, 2)
    assert tie_aware == 1.0 and strict == 0.5
    tie_aware, strict = O.recall_at_k(np.array([[0, 3]]), gt, gd, X, Q, 2)
    assert tie_aware == 0.5 and strict == 0.5


def test_rejects_bad_arguments():
    X = np.zeros((10, 4), np.float32)
    G = np.zeros((10, 2), np.uint32)
    ix = O.OracleIndex(X, G)
    with pytest.raises(ValueError):
        O.search(ix, X[:1], k=8, itopk=4)


def _star_case():
    """Node 0 at the origin with neighbours 1..8; neighbour j has 9 - j
    coordinates +1 and the rest -1, so with q = (3, ..., 3) its direction
    from node 0 agrees with the query's in exactly 9 - j of the 8
    dimensions. Nodes 1..8 link back to node 0 only."""
    d = 8
    X = np.zeros((9, d), np.float32)
    for j in range(1, 9):
        X[j] = -1.0
        X[j, :9 - j] = 1.0
    G = np.zeros((9, 8), np.uint32)
    G[0] = np.arange(1, 9)
    Q = np.full((1, d), 3.0, np.float32)
    # the seed that makes node 0 the single random seed of query 0
    seed = next(s for s in range(1000) if O.splitmix64(O.splitmix64(s)) % 9 == 0)
    return X, G, Q, seed


@pytest.mark.parametrize("f,kept", [(1.0, [1]), (0.75, [1, 2, 3]), (0.5, [1, 2, 3, 4, 5]), (0.01, list(range(1, 9)))])
def test_min_match_star_keeps_the_neighbours_at_or_above_the_threshold(f, kept):
    X, G, Q, seed = _star_case()
    ix = O.OracleIndex(X, G)
    ids, dists, cnt = O.search(ix, Q, k=9, itopk=16, max_iters=1, num_seeds=1, seed=seed,
                               dgs_min_match=f, dgs_cooldown=0.0)
    # distance to q = (3, ..., 3): node 0: 72; neighbour j: 4 (9 - j) + 16 (j - 1)
    expect = sorted([0] + kept, key=lambda j: 72 if j == 0 else 4 * (9 - j) + 16 * (j - 1))
    got = [int(i) for i in ids[0] if i != O.INVALID]
    assert got == expect
    assert int(cnt["vec_rows"][0]) == 1 + len(kept) and int(cnt["dgs_parents"][0]) == 1
    # the fixed top-n rule at discard 0.5 keeps four whatever their agreement
    ids, _, cnt = O.search(ix, Q, k=9, itopk=16, max_iters=1, num_seeds=1, seed=seed,
                           dgs_discard=0.5, dgs_cooldown=0.0)
    assert int(cnt["vec_rows"][0]) == 1 + 4


def test_min_match_met_by_every_neighbour_is_plain():
    rng = np.random.default_rng(14)
    n, d = 2000, 40
    X = rng.standard_normal((n, d)).astype(np.float32)
    Q = rng.standard_normal((50, d)).astype(np.float32)
    G = _ring_graph(n, 16, rng)
    # f = 0.01 asks for one agreeing dimension of 40; check on the data that
    # no (query, parent, neighbour) agrees in none, so every neighbour passes
    qbits = Q[:, None, :] > X[None, :, :]                  # query vs each parent
    nbits = X[G] > X[:, None, :]                           # neighbour vs its parent
    agree = (qbits[:, :, None, :] == nbits[None]).sum(-1)  # 50 x n x 16
    assert agree.min() >= 1
    base = O.search(ix := O.OracleIndex(X, G), Q, k=10, itopk=32, max_iters=80, seed=9)
    got = O.search(ix, Q, k=10, itopk=32, max_iters=80, seed=9, dgs_min_match=0.01)
    assert np.array_equal(got[0], base[0]) and np.array_equal(got[1], base[1])
    assert np.array_equal(got[2]["vec_rows"], base[2]["vec_rows"])
    assert (got[2]["dgs_parents"] > 0).all()


def test_min_match_arguments():
    X, G, Q, seed = _star_case()
    ix = O.OracleIndex(X, G)
    for kw in (dict(dgs_min_match=1.5), dict(dgs_min_match=-0.1), dict(dgs_min_match=0.5, dgs_discard=0.5)):
        with pytest.raises(ValueError):
            O.search(ix, Q, k=1, itopk=4, **kw)
