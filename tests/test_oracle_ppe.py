"""Pins for the path-extension oracle (Section 3.1.2, Eq. 3, Section 4):
one shard is the plain search; links built by a search whose queue holds the
whole next shard are Eq. 3's exact nearest nodes; with full queues every
stage is brute force over its shard, so the reduced result is the exact kNN
of the whole dataset; forwarded seeds are the linked nodes of each local
result; and on clustered data the forwarded start needs fewer iterations."""
import numpy as np
import pytest

import oracle as O
from oracle import ppe


def ring_graph(n, deg, rng):
    G = np.empty((n, deg), dtype=np.uint32)
    for i in range(n):
        others = rng.choice(np.delete(np.arange(n), [i, (i + 1) % n]), size=deg - 1, replace=False)
        G[i] = np.concatenate([[(i + 1) % n], others])
    return G


@pytest.fixture(scope="module")
def sharded():
    """Integer data (exact FP32 distances, exact ties) in 3 shards of uneven
    size, each with a ring graph."""
    from workloads import shard_split
    rng = np.random.default_rng(21)
    n, d, N = 301, 12, 3
    X = rng.integers(0, 16, size=(n, d)).astype(np.float32)
    Q = rng.integers(0, 16, size=(20, d)).astype(np.float32)
    parts = shard_split(n, N, 5)
    idx = [O.OracleIndex(X[p], ring_graph(len(p), 6, rng)) for p in parts]
    return X, Q, parts, idx


def test_split_is_a_partition():
    from workloads import shard_split
    parts = shard_split(1003, 4, 9)
    allids = np.concatenate(parts)
    assert np.array_equal(np.sort(allids), np.arange(1003)) and {len(p) for p in parts} == {250, 251}
    assert all((np.diff(p) > 0).all() for p in parts)


def test_chunks_cover_the_queries():
    for nq, N in ((10, 3), (3, 4), (101, 4), (0, 2)):
        b = ppe.chunk_bounds(nq, N)
        assert b[0][0] == 0 and b[-1][1] == nq and all(b[i][1] == b[i + 1][0] for i in range(N - 1))


def test_one_shard_is_the_plain_search(sharded):
    X, Q, parts, idx = sharded
    ix = O.OracleIndex(X, ring_graph(len(X), 6, np.random.default_rng(3)))
    ids = np.arange(len(X), dtype=np.uint32)
    for kw in (dict(itopk=16, max_iters=12), dict(itopk=32, max_iters=40, dgs_discard=0.5)):
        want = O.search(ix, Q, k=5, seed=4, **kw)
        for fwd, links in ((0, None), (1, [np.arange(len(X), dtype=np.uint32)])):
            got = ppe.ppe_search([ix], [ids], links, Q, n_forward=fwd, k=5, seed=4, **kw)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_links_by_full_search_are_eq3(sharded):
    X, Q, parts, idx = sharded
    for s in range(3):
        nxt = (s + 1) % 3
        exact = ppe.link_exact(X[parts[s]], X[parts[nxt]])
        got = ppe.link_by_search(idx[nxt], X[parts[s]], itopk=256, max_iters=2000, seed=1)
        # Eq. 3 picks a nearest node; the search breaks distance ties by
        # (distance, local index) as the exact one does
        assert np.array_equal(got, exact)
        # and a plausible mistake, linking into the shard itself, differs
        assert not np.array_equal(ppe.link_exact(X[parts[s]], X[parts[s]]), exact)


@pytest.mark.parametrize("fwd", [0, 1, 3])
def test_full_queues_give_the_exact_knn(sharded, fwd):
    X, Q, parts, idx = sharded
    links = [ppe.link_exact(X[parts[s]], X[parts[(s + 1) % 3]]) for s in range(3)]
    ids, d, cnt = ppe.ppe_search(idx, parts, links if fwd else None, Q, n_forward=fwd, k=10, itopk=128,
                                 max_iters=2000, seed=2)
    gt, gd = O.knn_f64(X, Q, 10)
    assert np.array_equal(ids, gt) and np.array_equal(d.astype(np.float64), gd)
    assert cnt.shape == (3, len(Q))


def test_forwarded_seed_is_the_link_of_the_local_top1(sharded):
    """With one iteration per stage, stage t > 0 evaluates exactly the linked
    node I(z) of the previous stage's best node z (as its single seed) and
    its neighbours."""
    X, Q, parts, idx = sharded
    links = [ppe.link_exact(X[parts[s]], X[parts[(s + 1) % 3]]) for s in range(3)]
    _, _, cnt = ppe.ppe_search(idx, parts, links, Q, n_forward=1, k=4, itopk=8, max_iters=1, seed=2)
    assert (cnt["vec_rows"][1:] <= 1 + 6).all() and (cnt["iters"][1:] == 1).all()
    _, _, cnt0 = ppe.ppe_search(idx, parts, None, Q, n_forward=0, k=4, itopk=8, max_iters=1, seed=2)
    assert (cnt0["vec_rows"][1:] >= 6).any()    # random seeds: search_width x degree of them


def test_forwarding_needs_fewer_iterations_on_clusters():
    """The paper's claim (Section 5.6.1, Fig. 12) as a sanity check on small
    clustered data: at a tight iteration cap, starting the later shards from
    the linked node of the previous result gives higher recall than starting
    each shard from random nodes."""
    from workloads import WORKLOADS, build_shards
    s = WORKLOADS[1].scaled(6000, nq=120, n_clusters=30)
    X, _ = s.mixture().sample(s.n, s.seeds["base"])
    from workloads import make_queries
    Q = make_queries(s)
    sh = build_shards(X, 3, 16, 32, "exact", 0.02, 8, seed=3, device="cpu")
    idx = [O.OracleIndex(t.X, t.G) for t in sh]
    gids = [t.ids for t in sh]
    links = [ppe.link_by_search(idx[(i + 1) % 3], sh[i].X, itopk=32, max_iters=64, seed=1) for i in range(3)]
    gt, gd = O.knn_f64(X, Q, 10)
    rec = {}
    for fwd in (0, 1):
        ids, _, _ = ppe.ppe_search(idx, gids, links if fwd else None, Q, n_forward=fwd, k=10, itopk=32, max_iters=6,
                                   seed=5)
        rec[fwd] = O.recall_at_k(ids, gt, gd, X, Q, 10)[0]
    assert rec[1] > rec[0], rec
