"""Path extension on simulated shards (Section 3.1.2, Eq. 3, Section 4) on the
GPU against the oracle: the links the library builds by search equal the
oracle's, and the sharded search (baseline sharding and forwarding of one or
several nodes) returns the oracle's ids, distances and per-stage counters,
with ghost staging or random entry and a query count that splits into
uneven chunks."""
import functools

import numpy as np
import pytest

import oracle as O
from oracle import ppe

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2507_17094_gb300 as A
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    A.build()


@functools.lru_cache(maxsize=None)
def ring(n_shards=4, storage=O.F32):
    """Workload 1's recipe (10,000 x 128, 50 clusters) in n_shards shards,
    each with its graph (degree 32) and a 2% ghost sample; 101 queries."""
    import paper_2507_17094_gb300 as A
    from workloads import WORKLOADS, build_shards, make_queries
    s = WORKLOADS[1]
    X, _ = s.mixture().sample(s.n, s.seeds["base"])
    Q = make_queries(s, nq=101)
    sh = build_shards(X, n_shards, 32, 64, "exact", 0.02, 8, seed=11)
    gidx = [A.Index(t.X, t.G, storage=storage, ghost_ids=t.S, ghost_graph=t.Gg) for t in sh]
    oidx = [O.OracleIndex(t.X, t.G, storage, t.S, t.Gg) for t in sh]
    rg = A.Shards(gidx, [t.ids for t in sh])
    return X, Q, sh, gidx, oidx, rg


LINK = dict(itopk=32, max_iters=48, entry=1, ghost_max_iters=8, seed=17)


def test_links_by_search_match_the_oracle():
    X, Q, sh, gidx, oidx, rg = ring()
    rg.link(**LINK)
    for i in range(len(sh)):
        want = ppe.link_by_search(oidx[(i + 1) % len(sh)], sh[i].X, **LINK)
        assert np.array_equal(rg.get_links(i), want)


@pytest.mark.parametrize("n_forward", [0, 1, 4])
@pytest.mark.parametrize("params", [dict(k=10, itopk=32, max_iters=24, entry=1, dgs_discard=0.5, ghost_max_iters=8),
                                    dict(k=10, itopk=64, max_iters=12, entry=0)])
def test_sharded_search_matches_the_oracle(n_forward, params):
    X, Q, sh, gidx, oidx, rg = ring()
    links = [ppe.link_by_search(oidx[(i + 1) % len(sh)], sh[i].X, **LINK) for i in range(len(sh))]
    for i, l in enumerate(links):
        rg.set_links(i, l)
    ids, d, st = rg.search(torch.from_numpy(Q).cuda(), n_forward=n_forward, stats=True, seed=5, **params)
    torch.cuda.synchronize()
    g_ids = ids.cpu().numpy().view(np.uint32)
    g_d = d.cpu().numpy()
    o_ids, o_d, o_c = ppe.ppe_search(oidx, [t.ids for t in sh], links if n_forward else None, Q,
                                     n_forward=n_forward, seed=5, **params)
    assert np.array_equal(g_ids, o_ids)
    assert np.array_equal(g_d.view(np.uint32), o_d.view(np.uint32))
    import paper_2507_17094_gb300 as A
    gst = st.cpu().numpy().astype(np.uint32).reshape(len(sh), len(Q), -1)
    for t in range(len(sh)):
        g = np.ascontiguousarray(gst[t]).view(A.STATS_DTYPE).reshape(-1)
        assert (g["status"] == 0).all()
        exact = g["hash_resets"] == 0
        for f in ("iters", "parents", "vec_rows", "ghost_vec_rows"):
            assert np.array_equal(g[f][exact].astype(np.int64), o_c[f][t][exact].astype(np.int64)), (t, f)


def test_low_precision_ring_and_one_shard():
    """FP16 shards with rerank, and a ring of one shard, which is the plain
    search of that index."""
    import paper_2507_17094_gb300 as A
    X, Q, sh, gidx, oidx, rg = ring(3, O.F16)
    rg.link(**LINK)
    links = [rg.get_links(i) for i in range(3)]
    p = dict(k=10, itopk=32, max_iters=24, entry=1, dgs_discard=0.5, ghost_max_iters=8, rerank=1, seed=8)
    ids, d, _ = rg.search(torch.from_numpy(Q).cuda(), n_forward=1, **p)
    torch.cuda.synchronize()
    o_ids, o_d, _ = ppe.ppe_search(oidx, [t.ids for t in sh], links, Q, n_forward=1, **p)
    assert np.array_equal(ids.cpu().numpy().view(np.uint32), o_ids)
    assert np.array_equal(d.cpu().numpy().view(np.uint32), o_d.view(np.uint32))
    one = A.Shards([gidx[0]], [sh[0].ids])
    one.set_links(0, np.arange(gidx[0].n, dtype=np.uint32))
    i1, d1, _ = one.search(torch.from_numpy(Q).cuda(), n_forward=1, **p)
    i2, d2, _ = gidx[0].search(torch.from_numpy(Q).cuda(), **p)
    torch.cuda.synchronize()
    assert np.array_equal(i1.cpu().numpy().view(np.uint32), sh[0].ids[i2.cpu().numpy().view(np.uint32)])
    assert torch.equal(d1, d2)
    one.close()


def test_ring_rejects_bad_arguments():
    import paper_2507_17094_gb300 as A
    X, Q, sh, gidx, oidx, rg = ring()
    with pytest.raises(A.AnnError):
        rg.set_links(0, np.full(gidx[0].n, gidx[1].n, dtype=np.uint32))      # beyond the next shard
    with pytest.raises(A.AnnError):
        rg.search(torch.from_numpy(Q).cuda(), n_forward=11, k=10, itopk=32)    # more than k forwarded
    with pytest.raises(A.AnnError):
        rg.search(torch.from_numpy(Q).cuda(), n_forward=1, k=10, itopk=32, entry=3)
