"""Shared GPU-test helpers: seeded cases and a GPU-vs-oracle comparison.

The same seeded inputs go to the CUDA library (through the C ABI) and to the
CPU oracle; nothing the oracle sees comes from the GPU.
"""
from __future__ import annotations

import functools

import numpy as np

import oracle as O
from workloads import WORKLOADS, build_graph, ghost_sample, make_queries

# Distances are FP32 on both sides, one fused multiply-add per element into
# four interleaved partial sums combined pairwise, so the expected agreement
# is exact. The bar the
# method sets is looser: ids equal except at distance ties within 1e-5
# relative, distances within 1e-5 relative.
DIST_RTOL = 1e-5

STAT_KEYS = ("iters", "parents", "dgs_parents", "vec_rows", "ghost_iters", "ghost_parents",
             "ghost_vec_rows", "rerank_rows")


class Case:
    def __init__(self, X, G, Q, S=None, Gg=None):
        self.X, self.G, self.Q, self.S, self.Gg = X, G, Q, S, Gg
        self._gpu = {}
        self._or = {}

    def gpu_index(self, storage):
        import paper_2507_17094_gb300 as A
        if storage not in self._gpu:
            self._gpu[storage] = A.Index(self.X, self.G, storage=storage, ghost_ids=self.S, ghost_graph=self.Gg,
                                         keep_fp32=True, build_dir=True)
        return self._gpu[storage]

    def oracle_index(self, storage):
        if storage not in self._or:
            self._or[storage] = O.OracleIndex(self.X, self.G, storage, self.S, self.Gg)
        return self._or[storage]

    def run(self, storage, queries=None, given=None, **params):
        import torch
        import paper_2507_17094_gb300 as A
        Q = self.Q if queries is None else queries
        gi = self.gpu_index(storage)
        qt = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
        gt = None if given is None else torch.from_numpy(given.astype(np.uint32).view(np.int32)).cuda()
        ids, dists, st = gi.search(qt, given=gt, stats=True, **params)
        torch.cuda.synchronize()
        gi.sync()
        g_ids = ids.cpu().numpy().view(np.uint32)
        g_d = dists.cpu().numpy()
        g_st = A.stats_to_numpy(st)
        o_ids, o_d, o_c = O.search(self.oracle_index(storage), Q, given_ghost_seeds=given, **params)
        return (g_ids, g_d, g_st), (o_ids, o_d, o_c)


def assert_parity(g, o, counters=True):
    g_ids, g_d, g_st = g
    o_ids, o_d, o_c = o
    assert (g_st["status"] == 0).all(), "a query reported a device failure"
    # the bar: distances within 1e-5 relative, ids equal except near-ties
    np.testing.assert_allclose(g_d, o_d, rtol=DIST_RTOL, atol=0)
    diff = g_ids != o_ids
    if diff.any():
        near = np.abs(g_d - o_d) <= DIST_RTOL * np.maximum(np.abs(o_d), 1e-30)
        assert near[diff].all(), f"{diff.sum()} ids differ beyond ties"
    # what this design delivers: bit-identical results
    assert np.array_equal(g_ids, o_ids), f"{diff.sum()} ids differ"
    assert np.array_equal(g_d.view(np.uint32), o_d.view(np.uint32)), "distances differ in the last bit"
    if counters:
        exact = g_st["hash_resets"] == 0
        for k in STAT_KEYS:
            gv = g_st[k].astype(np.int64)
            ov = o_c[k].astype(np.int64)
            assert np.array_equal(gv[exact], ov[exact]), f"counter {k} differs"
            if k in ("vec_rows", "ghost_vec_rows"):
                assert (gv >= ov).all(), f"counter {k} below the oracle's"


@functools.lru_cache(maxsize=None)
def tiny_case():
    """Workload 1 as specified: 10,000 x 128 FP32, 50 clusters, degree 32,
    100 queries, ghost set 1% (100 nodes) with a degree-16 graph."""
    s = WORKLOADS[1]
    X, _ = s.mixture().sample(s.n, s.seeds["base"])
    G = build_graph(X, s.degree, s.knn_k, s.graph)
    S = ghost_sample(s.n, s.ghost_n, s.seeds["ghost"])
    Gg = build_graph(X[S], s.ghost_degree, 2 * s.ghost_degree, "exact")
    return Case(X, G, make_queries(s), S, Gg)


@functools.lru_cache(maxsize=None)
def ragged_case(n=3000, d=40, deg=12, nq=77, gdeg=6, seed=7):
    """Dimension not a multiple of 32, degree not a multiple of 4, a query
    count that is not a multiple of the warps per block."""
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((n, d)) * rng.uniform(0.5, 3.0, (1, d))).astype(np.float32)
    Q = (rng.standard_normal((nq, d)) * rng.uniform(0.5, 3.0, (1, d))).astype(np.float32)
    G = build_graph(X, deg, 2 * deg, "exact", n_bridge=2)
    S = ghost_sample(n, n // 20, seed + 1)
    Gg = build_graph(X[S], gdeg, 2 * gdeg, "exact", n_bridge=0)
    return Case(X, G, Q, S, Gg)


@functools.lru_cache(maxsize=None)
def int_case(n=4000, d=128, deg=16, nq=64, seed=9):
    """Integer data in [0, 255] (the precision workload's recipe): many exact
    distance ties, FP16 storage exact."""
    s = WORKLOADS[3].scaled(n, nq=nq, n_clusters=20)
    X, _ = s.mixture().sample(n, s.seeds["base"])
    Q = make_queries(s)
    G = build_graph(X, deg, 2 * deg, "exact")
    S = ghost_sample(n, n // 50, s.seeds["ghost"])
    Gg = build_graph(X[S], 8, 16, "exact", n_bridge=0)
    return Case(X, G, Q, S, Gg)


@functools.lru_cache(maxsize=None)
def hub_case(n=6000, d=32, deg=32, nq=96, seed=13):
    """A graph built to crowd the visited table: every adjacency row starts
    with the same four hub nodes and repeats neighbours (slot j + 16 copies
    slot j for j < 8), so lanes of one warp insert equal ids at once and
    long probe runs form; long searches fill the table towards its reset
    threshold."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d)).astype(np.float32)
    Q = rng.standard_normal((nq, d)).astype(np.float32)
    G = build_graph(X, deg, 2 * deg, "exact", n_bridge=2).copy()
    G[:, :4] = np.array([1, 2, 3, 5], dtype=np.uint32)
    G[:, 16:24] = G[:, 0:8]
    S = ghost_sample(n, n // 20, seed + 1)
    Gg = build_graph(X[S], 8, 16, "exact", n_bridge=0)
    return Case(X, G, Q, S, Gg)
