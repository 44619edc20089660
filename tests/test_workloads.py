"""The input generators are deterministic and produce well-formed graphs."""
import numpy as np

from workloads import WORKLOADS, build_graph, ghost_sample, make_queries


def test_mixture_is_seeded_and_shaped():
    s = WORKLOADS[2].scaled(5000, nq=50, n_clusters=20, ghost_n=50)
    a, _ = s.mixture().sample(s.n, s.seeds["base"])
    b, _ = s.mixture().sample(s.n, s.seeds["base"])
    assert a.shape == (5000, 96) and a.dtype == np.float32 and np.array_equal(a, b)
    np.testing.assert_allclose(np.linalg.norm(a, axis=1), 1.0, rtol=1e-5)   # normalised recipe
    q = make_queries(s, off_fraction=0.2)
    assert q.shape == (50, 96)


def test_integer_recipe():
    s = WORKLOADS[3].scaled(2000, nq=10, n_clusters=10)
    x, _ = s.mixture().sample(s.n, s.seeds["base"])
    assert x.min() >= 0 and x.max() <= 255 and np.array_equal(x, np.rint(x))


def test_graph_is_fixed_degree_without_self_loops_or_duplicates():
    s = WORKLOADS[1]
    x, _ = s.mixture().sample(3000, s.seeds["base"])
    g = build_graph(x, 16, 32, "exact", device="cpu")
    assert g.shape == (3000, 16) and g.dtype == np.uint32
    assert (g < 3000).all()
    assert (g != np.arange(3000)[:, None]).all()
    assert all(len(set(r)) == 16 for r in g)


def test_ghost_sample():
    s = ghost_sample(1000, 37, 5)
    assert len(set(s.tolist())) == 37 and np.all(np.diff(s.astype(np.int64)) > 0)
    assert np.array_equal(s, ghost_sample(1000, 37, 5))


def test_off_distribution_queries_are_mixed_in():
    """Workload 4's off-distribution queries sit at seeded random positions:
    a prefix (a ground-truth sample) holds both kinds in proportion, and the
    mask names exactly the queries far from every cluster center."""
    from workloads import off_distribution_mask
    s = WORKLOADS[4].scaled(5000, nq=2000, n_clusters=40)
    q = make_queries(s, off_fraction=0.2)
    m = off_distribution_mask(s, 0.2)
    assert q.shape == (2000, 256) and m.sum() == 400
    assert 0.1 < m[:500].mean() < 0.3
    c = s.mixture().centers
    d = ((q[:, None, :].astype(np.float64) - c[None]) ** 2).sum(-1).min(1)
    assert d[m].min() > d[~m].max()
