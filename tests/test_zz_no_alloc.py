"""The search entry point that allocates no device memory.

ann_search_host_noalloc serves callers that must not allocate device memory
while answering queries (a server that reserved all device memory at start,
code under an external memory budget, a thread that cannot take the device
synchronisation an allocation may cause). It stages everything in one fixed
per-GPU array instead of the index's on-demand workspace. These tests call it
through the C ABI and compare it with ann_search_host on the same inputs, two
calls in a row (the array keeps the previous call's contents, so the second
call checks that it clears what it relies on). This file is collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def index():
    import paper_2507_17094_gb300 as A
    from workloads import build_graph, ghost_sample
    assert torch.cuda.is_available(), "needs a CUDA device"
    A.build()
    rng = np.random.default_rng(42)
    n, d = 4000, 64
    X = rng.standard_normal((n, d)).astype(np.float32)
    Q = rng.standard_normal((300, d)).astype(np.float32)
    G = build_graph(X, 16, 32, "exact")
    S = ghost_sample(n, 80, 3)
    Gg = build_graph(X[S], 8, 16, "exact", n_bridge=0)
    ix = A.Index(X, G, storage=A.F16, ghost_ids=S, ghost_graph=Gg)
    yield ix, Q
    ix.close()


@pytest.mark.parametrize("params", [dict(itopk=32, max_iters=48, entry=1, dgs_discard=0.5, rerank=1),
                                    dict(itopk=64, k=20, max_iters=80, search_width=2)])
def test_noalloc_matches_host_search_two_calls(index, params):
    ix, Q = index
    want_ids, want_d = ix.search_host(Q, seed=9, **params)
    for _ in range(2):
        ids, dists = ix.search_host_noalloc(Q, seed=9, **params)
        # same kernel, same inputs: identical results (the parity bar is ids
        # equal except near-ties and distances within 1e-5 relative)
        np.testing.assert_allclose(dists, want_d, rtol=1e-5, atol=0)
        assert np.array_equal(ids, want_ids)


def test_noalloc_rejects_batches_beyond_the_scratch(index):
    import paper_2507_17094_gb300 as A
    ix, _ = index
    nq = (8 << 20) // (64 * 4) + 1          # the query copy alone exceeds 8 MiB
    Q = np.zeros((nq, 64), np.float32)
    with pytest.raises(A.AnnError) as e:
        ix.search_host_noalloc(Q, itopk=32)
    assert e.value.status == 1 and "scratch" in str(e.value)
