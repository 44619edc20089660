"""Continuous batching: every request's result is the same alone and in the
mix (and equal to the batch search of its queries), with requests of uneven
size and differing k / itopk admitted while others run, through a ring small
enough that admission has to wait for memory to free up."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def served():
    import paper_2507_17094_gb300 as A
    from workloads import WORKLOADS, build_graph, ghost_sample, make_queries
    assert torch.cuda.is_available()
    A.build()
    spec = WORKLOADS[2].scaled(50_000, nq=4000, n_clusters=50, ghost_n=500)
    X, _ = spec.mixture().sample(spec.n, spec.seeds["base"])
    G = build_graph(X, 32, 64, "partitioned", n_parts=50, seed=1)
    S = ghost_sample(spec.n, spec.ghost_n, spec.seeds["ghost"])
    Gg = build_graph(X[S], 16, 32, "exact", seed=2)
    ix = A.Index(X, G, storage=A.F16, ghost_ids=S, ghost_graph=Gg)
    Q = make_queries(spec)
    rng = np.random.default_rng(12)
    trace, t = [], 0.0
    for rid in range(40):
        n = int(rng.integers(1, 301))
        off = int(rng.integers(0, len(Q) - n))
        prm = dict(k=int(rng.choice([10, 20])), itopk=int(rng.choice([32, 64])), max_iters=96, entry=1,
                   dgs_discard=0.5, ghost_max_iters=32, rerank=1, seed=5, qid_base=rid * 1000)
        t += float(rng.exponential(0.0005))
        trace.append((t, rid, Q[off:off + n], prm))
    yield A, ix, trace
    ix.close()


def make_server(A, ix, capacity=1024):
    return A.Server(ix, capacity=capacity, max_requests=16,
                    max_params=dict(k=20, itopk=64, search_width=1, max_iters=96, entry=1, dgs_discard=0.5,
                                    rerank=1, ghost_itopk=64))


def test_alone_equals_mix_equals_batch(served):
    A, ix, trace = served
    srv = make_server(A, ix)
    alone = {}
    for t, rid, q, prm in trace:
        res, _ = A.replay(srv, [(0.0, rid, q, prm)])
        alone[rid] = res[rid]
    mixed, wall = A.replay(srv, trace)
    assert srv.in_flight() == 0
    srv.close()
    lat = []
    for t, rid, q, prm in trace:
        ids_a, d_a, _ = alone[rid]
        ids_m, d_m, l_m = mixed[rid]
        assert np.array_equal(ids_a, ids_m) and np.array_equal(d_a, d_m), rid
        b_ids, b_d, _ = ix.search(torch.from_numpy(q).cuda(), **prm)
        assert np.array_equal(b_ids.cpu().numpy().view(np.uint32), ids_m), rid
        np.testing.assert_allclose(b_d.cpu().numpy(), d_m, rtol=0, atol=0)
        lat.append(l_m)
    assert all(x > 0 for x in lat)
    print(f"{len(trace)} requests, {sum(len(x[2]) for x in trace)} queries in {wall * 1e3:.1f} ms; "
          f"p50 {np.percentile(lat, 50) * 1e3:.2f} ms, p99 {np.percentile(lat, 99) * 1e3:.2f} ms")


def test_admission_by_memory(served):
    A, ix, trace = served
    srv = make_server(A, ix, capacity=512)
    big = [x for x in trace if len(x[2]) > 200][:4]
    assert len(big) >= 3
    admitted = [srv.submit(rid, q, **prm) for _, rid, q, prm in big]
    # three requests of > 200 queries cannot all sit in 512 slots at once
    assert admitted[0] and not all(admitted)
    done = {}
    while len(done) < sum(admitted):
        for rid, ids, dists, lat in srv.poll():
            done[rid] = ids
    # after completions the ring has room again
    rest = [x for x, ok in zip(big, admitted) if not ok]
    res, _ = A.replay(srv, [(0.0, rid, q, prm) for _, rid, q, prm in rest])
    assert len(res) == len(rest)
    srv.close()


def test_rejects_params_beyond_the_server_maximum(served):
    A, ix, trace = served
    srv = make_server(A, ix)
    with pytest.raises(A.AnnError):
        srv.submit(999, trace[0][2], k=10, itopk=128, entry=1)
    srv.close()
