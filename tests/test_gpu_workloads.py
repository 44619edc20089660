"""Medium-size parity: each workload's recipe (data distribution, graph
builder, ghost ratio, degree, precision, search settings) at a size where the
CPU oracle searches every query in seconds, large enough to reach the
kernel's full-size paths: several 16-row staging rounds per parent (degree
64 without DGS), the global visited tables with their resets, the ghost
stage's bitmap, integer distance ties (workload 3's data), Zipf cluster
sizes (workload 4), and serving with the full k / itopk mix (workload 5).

Every query's ids and distances must equal the oracle's (see gpu_cases for
the bar) and, where no visited table reset, so must its counters. The
full-size versions of these checks are in test_gpu_fullsize.py (opt-in).
"""
import functools

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2507_17094_gb300 as A
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    A.build()


from gpu_cases import Case, assert_parity  # noqa: E402


@functools.lru_cache(maxsize=None)
def workload_case(number, n, nq, n_clusters, ghost_n, off_fraction=0.0):
    """Workload `number`'s recipe scaled to n base vectors: same mixture
    family, graph builder (partitioned kNN + detour pruning + bridges),
    degree and ghost degree."""
    from workloads import WORKLOADS, build_graph, ghost_sample, make_queries
    s = WORKLOADS[number].scaled(n, nq=nq, n_clusters=n_clusters, ghost_n=ghost_n)
    X, _ = s.mixture().sample(s.n, s.seeds["base"])
    G = build_graph(X, s.degree, s.knn_k, "partitioned", n_parts=max(2, n // 1000), seed=s.seeds["base"])
    S = ghost_sample(s.n, s.ghost_n, s.seeds["ghost"])
    Gg = build_graph(X[S], s.ghost_degree, 2 * s.ghost_degree, "exact", seed=s.seeds["ghost"])
    return Case(X, G, make_queries(s, off_fraction=off_fraction), S, Gg)


def recall10(case, ids):
    gt, gd = O.knn_f64(case.X, case.Q, 10)
    return O.recall_at_k(ids, gt, gd, case.X, case.Q, 10)[0]


# Workload 2's recipe (96-d, anisotropic, normalised, degree 64) at 100,000
# points: the benchmark's headline setting and the paper's discard 0.5.
W2_PARAMS = [
    dict(k=10, itopk=32, max_iters=48, entry=1, dgs_discard=0.75, ghost_max_iters=12, ghost_search_width=4),
    dict(k=10, itopk=32, max_iters=96, entry=1, dgs_discard=0.5, ghost_max_iters=64),
    dict(k=10, itopk=64, max_iters=80, entry=0),                       # no ghost stage, no DGS: 4 rounds of 16
    dict(k=10, itopk=256, max_iters=300, entry=1, dgs_discard=0.5, search_width=2),
]


@pytest.mark.parametrize("params", W2_PARAMS, ids=lambda p: "-".join(f"{k}{v}" for k, v in p.items()))
def test_workload2_recipe(params):
    c = workload_case(2, 100_000, 2000, 100, 1000)
    g, o = c.run(O.F32, seed=4002, **params)
    assert_parity(g, o)
    if params["itopk"] == 32 and params["dgs_discard"] == 0.75:
        assert recall10(c, g[0]) >= 0.95


@pytest.mark.parametrize("storage,k,itopk", [(O.F16, 10, 128), (O.E4M3, 10, 128), (O.F16, 100, 256),
                                             (O.F32, 10, 64)])
def test_workload3_recipe_integer_ties(storage, k, itopk):
    """Integer data in [0, 255]: FP32 sums of integer squares are exact, so
    distances tie often; FP16 stores the integers exactly, so the reranked
    FP16 distances must equal the FP64 ones exactly."""
    c = workload_case(3, 200_000, 600, 200, 2000)
    p = dict(k=k, itopk=itopk, max_iters=2 * itopk + 32, entry=1, dgs_discard=0.5, ghost_max_iters=64,
             rerank=0 if storage == O.F32 else 1, seed=4003)
    g, o = c.run(storage, **p)
    assert_parity(g, o)
    if storage == O.F16:
        ids = g[0]
        ok = ids != O.INVALID
        exact = O.pair_dist_f64(c.X, c.Q, np.where(ok, ids, 0).astype(np.uint32))
        assert np.array_equal(g[1][ok].astype(np.float64), exact[ok])


@pytest.mark.parametrize("storage", [O.F32, O.F16])
def test_workload4_recipe_zipf(storage):
    """256-d with Zipf(1.1) cluster sizes and 20% of the queries between
    clusters."""
    c = workload_case(4, 150_000, 500, 150, 1500, off_fraction=0.2)
    g, o = c.run(storage, k=10, itopk=64, max_iters=160, entry=1, dgs_discard=0.5, ghost_max_iters=64,
                 rerank=0 if storage == O.F32 else 1, seed=4004)
    assert_parity(g, o)


def test_workload5_recipe_serving_mix():
    """Workload 5's serving mix (batches of uneven size, k in {10, 100},
    itopk in {64, 256}, FP16 + rerank) on its recipe at 150,000 points:
    every served request equals the batch search of its queries, which
    itself equals the oracle on a sample of requests."""
    import paper_2507_17094_gb300 as A
    c = workload_case(5, 150_000, 3000, 150, 1500)
    ix = c.gpu_index(O.F16)
    srv = A.Server(ix, capacity=4096, max_requests=32,
                   max_params=dict(k=100, itopk=256, max_iters=544, entry=1, dgs_discard=0.5, rerank=1,
                                   ghost_itopk=64))
    rng = np.random.default_rng(55)
    trace, t = [], 0.0
    for rid in range(24):
        n = int(rng.integers(1, 700))
        off = int(rng.integers(0, len(c.Q) - n))
        k = int(rng.choice([10, 100]))
        L = max(k, int(rng.choice([64, 256])))
        prm = dict(k=k, itopk=L, max_iters=2 * L + 32, entry=1, dgs_discard=0.5, ghost_max_iters=64, rerank=1,
                   seed=5, qid_base=rid << 20)
        t += float(rng.exponential(0.001))
        trace.append((t, rid, c.Q[off:off + n], prm))
    res, _ = A.replay(srv, trace, timeout_s=120)
    srv.close()
    oi = c.oracle_index(O.F16)
    for j, (_, rid, q, prm) in enumerate(trace):
        ids, d, _ = ix.search(torch.from_numpy(np.ascontiguousarray(q)).cuda(), **prm)
        torch.cuda.synchronize()
        b_ids, b_d = ids.cpu().numpy().view(np.uint32), d.cpu().numpy()
        assert np.array_equal(b_ids, res[rid][0]) and np.array_equal(b_d, res[rid][1])
        if j % 4 == 0:
            o_ids, o_d, _ = O.search(oi, q, **prm)
            assert np.array_equal(b_ids, o_ids) and np.array_equal(b_d.view(np.uint32), o_d.view(np.uint32))


@pytest.mark.parametrize("d", [768, 960])
@pytest.mark.parametrize("storage,params", [
    (O.F32, dict(k=10, itopk=32, max_iters=48, entry=1, dgs_discard=0.5, ghost_max_iters=12, ghost_search_width=4)),
    (O.F32, dict(k=10, itopk=32, max_iters=48, entry=1, ghost_max_iters=12, ghost_search_width=4)),
    (O.F16, dict(k=10, itopk=64, max_iters=48, entry=1, dgs_discard=0.5, ghost_max_iters=12, rerank=1)),
    (O.E4M3, dict(k=16, itopk=16, max_iters=24, entry=0, dgs_discard=0.75, rerank=1)),
])
def test_wide_recipe(d, storage, params):
    """The wide workloads' recipe (768-d and 960-d: rows of 1.5-3.75 KB,
    distances by four lanes per row, fewer rows per round; a direction table
    of 24-30 words per edge) at 30,000 points."""
    c = workload_case(6 if d == 768 else 7, 30_000, 300, 30, 300)
    g, o = c.run(storage, seed=4006, **params)
    assert_parity(g, o)
