"""Graph construction on the GPU against the builder's oracle: the exact kNN
lists (ids equal to the FP64 oracle's except where two candidates' FP64
distances lie within the FP32 error bound of each other), the pruning
bit-exact on the same kNN input (ragged sizes, a degree not a multiple of 4,
a hub-heavy list set), and the whole build on data without near-ties."""
import numpy as np
import pytest

from oracle import INVALID, knn_f64
from oracle import graph as OG

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2507_17094_gb300 as A
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    A.build()


def fp32_bound(X, d):
    """Relative error bound of an FP32 sum of d squared differences."""
    return 2.0 * d * 2.0 ** -24


@pytest.mark.parametrize("n,d,K", [(1000, 24, 16), (3001, 128, 64), (777, 100, 33), (300, 384, 8)])
def test_knn_exact_matches_fp64(n, d, K):
    import paper_2507_17094_gb300 as A
    rng = np.random.default_rng(n + d)
    X = (rng.standard_normal((n, d)) * rng.uniform(0.5, 2.0, d)).astype(np.float32)
    got = A.knn_exact(torch.from_numpy(X).cuda(), K).cpu().numpy().view(np.uint32)
    want = OG.knn_lists(X, K)
    diff = got != want
    if diff.any():
        # every disagreement must be a near-tie: the two ids' FP64 distances
        # to the row's node within the FP32 error of the sums
        for u, j in zip(*np.nonzero(diff)):
            a, b = int(got[u, j]), int(want[u, j])
            da = float(((X[a].astype(np.float64) - X[u]) ** 2).sum())
            db = float(((X[b].astype(np.float64) - X[u]) ** 2).sum())
            assert abs(da - db) <= fp32_bound(X, d) * max(da, db), (u, j, da, db)
    assert diff.mean() < 0.01
    assert (got != np.arange(n)[:, None]).all()          # never the node itself


@pytest.mark.parametrize("n,K,degree", [(2000, 32, 16), (1501, 24, 10), (700, 64, 64), (33, 20, 7)])
def test_prune_bit_exact(n, K, degree):
    import paper_2507_17094_gb300 as A
    rng = np.random.default_rng(n + K)
    X = rng.standard_normal((n, 8)).astype(np.float32)
    knn = OG.knn_lists(X, K)
    got = A.graph_prune(torch.from_numpy(knn.view(np.int32)).cuda(), degree).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, OG.prune(knn, degree))


def test_prune_hub_lists_bit_exact():
    """Lists crowded onto a few hubs (thousands of reverse offers to one
    node) and INVALID tails."""
    import paper_2507_17094_gb300 as A
    rng = np.random.default_rng(5)
    n, K = 3000, 16
    knn = np.empty((n, K), np.uint32)
    for u in range(n):
        hubs = [h for h in (0, 1, 2, 3) if h != u]
        rest = rng.choice(np.setdiff1d(np.arange(n), hubs + [u]), K - len(hubs), replace=False)
        knn[u] = np.concatenate([hubs, rest]).astype(np.uint32)
    knn[::7, -3:] = INVALID
    got = A.graph_prune(torch.from_numpy(knn.view(np.int32)).cuda(), 12).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, OG.prune(knn, 12))


def test_whole_build_matches_the_oracle():
    """kNN then pruning on integer data small enough that FP32 sums are
    exact (6 x 1000^2 < 2^24): both sides rank the same exact distances and
    break ties by id."""
    import paper_2507_17094_gb300 as A
    rng = np.random.default_rng(9)
    n, d = 1200, 6
    X = rng.integers(0, 1000, size=(n, d)).astype(np.float32)
    Xt = torch.from_numpy(X).cuda()
    knn = A.knn_exact(Xt, 24)
    G = A.graph_prune(knn, 12).cpu().numpy().view(np.uint32)
    want_knn = OG.knn_lists(X, 24)
    assert np.array_equal(knn.cpu().numpy().view(np.uint32), want_knn)
    assert np.array_equal(G, OG.prune(want_knn, 12))
