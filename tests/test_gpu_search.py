"""GPU parity: the CUDA library (called through the C ABI) against the CPU
oracle on the same seeded inputs.

Preprocessing (codec, direction table, ghost rows) must be bit-exact. The
search must return the oracle's ids and distances (see gpu_cases for the
bar) and, where the visited table never reset, the oracle's exact counters.
"""
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
    A.lib()


from gpu_cases import assert_parity, int_case, ragged_case, tiny_case  # noqa: E402


# ------------------------------------------------------------ preprocessing
@pytest.mark.parametrize("storage", [O.F16, O.E4M3])
def test_encode_bit_exact(storage):
    import paper_2507_17094_gb300 as A
    rng = np.random.default_rng(21)
    X = (rng.standard_normal((513, 100)) * np.exp(rng.uniform(-30, 30, (513, 1)))).astype(np.float32)
    X[0] = 0.0
    X[1, :] = 1e-40                              # subnormal-only row
    X[2, :50] = 65504.0 * 3
    X[3] = np.float32(2.0) ** np.arange(-50, 50)
    codes, scales = A.encode(torch.from_numpy(X).cuda(), storage)
    torch.cuda.synchronize()
    oc, os_ = O.encode(X, storage)
    assert np.array_equal(scales.cpu().numpy().view(np.uint32), os_.view(np.uint32))
    g = codes.cpu().numpy().view(np.uint16 if storage == O.F16 else np.uint8)
    assert np.array_equal(g, oc)


@pytest.mark.parametrize("storage", [O.F32, O.F16, O.E4M3])
@pytest.mark.parametrize("case", ["tiny", "ragged"])
def test_index_preprocessing_bit_exact(storage, case):
    c = tiny_case() if case == "tiny" else ragged_case()
    gi = c.gpu_index(storage)
    oi = c.oracle_index(storage)
    assert np.array_equal(gi.export(2), oi.dir)
    if storage != O.F32:
        codes, scales = O.encode(c.X, storage)
        assert np.array_equal(gi.export(0), codes)
        assert np.array_equal(gi.export(1), scales)
        assert np.array_equal(gi.export(3), codes[c.S])
        assert np.array_equal(gi.export(4), scales[c.S])
    else:
        assert np.array_equal(gi.export(0), c.X)
        assert np.array_equal(gi.export(3), c.X[c.S])


def test_dir_table_primitive_matches_oracle():
    import paper_2507_17094_gb300 as A
    c = ragged_case()
    Xt = torch.from_numpy(c.X).cuda()
    Gt = torch.from_numpy(c.G.view(np.int32)).cuda()
    for storage in (O.F32, O.F16, O.E4M3):
        if storage == O.F32:
            vec, sc = Xt, None
        else:
            vec, sc = A.encode(Xt, storage)
        d = A.dir_table(vec, sc, storage, Gt)
        torch.cuda.synchronize()
        want = O.dir_table(O.stored_vectors(c.X, storage), c.G)
        assert np.array_equal(d.cpu().numpy().view(np.uint32), want)


# ------------------------------------------------------------------ search
TINY_PARAMS = [
    dict(itopk=64, max_iters=64),                                             # plain, random entry
    dict(itopk=64, max_iters=64, entry=1),                                    # ghost staging
    dict(itopk=64, max_iters=64, dgs_discard=0.5),                            # DGS
    dict(itopk=64, max_iters=64, entry=1, dgs_discard=0.5),                   # GS + DGS
    dict(itopk=64, max_iters=64, entry=1, dgs_discard=0.5, dgs_reexpand=1),   # DGS with re-expansion
    dict(itopk=32, max_iters=96, search_width=2, entry=1, dgs_discard=0.3),
    dict(itopk=16, k=16, max_iters=40, search_width=4),
    dict(itopk=128, max_iters=300, entry=1, dgs_discard=0.7, dgs_cooldown=0.5),
    dict(itopk=256, max_iters=300, num_seeds=300),
    dict(itopk=512, k=100, max_iters=600, search_width=8, entry=1, ghost_itopk=100, ghost_seeds_out=7),
    dict(itopk=64, max_iters=0),                                              # seeds only
    dict(itopk=64, max_iters=0, entry=1),                                     # ghost stage only
    dict(itopk=32, max_iters=48, entry=1, dgs_discard=0.7, ghost_search_width=2, ghost_max_iters=24),
    dict(itopk=64, max_iters=64, entry=1, ghost_search_width=4, ghost_itopk=48),
    dict(itopk=64, max_iters=64, entry=1, dgs_discard=0.5, ghost_search_width=8, ghost_itopk=64),  # Wg > W
    dict(itopk=64, max_iters=64, dgs_min_match=0.55),                       # DGS by similarity
    dict(itopk=64, max_iters=64, entry=1, dgs_min_match=0.6, dgs_reexpand=1),
    dict(itopk=32, max_iters=96, search_width=2, entry=1, dgs_min_match=0.5, dgs_cooldown=0.5),
]


@pytest.mark.parametrize("params", TINY_PARAMS, ids=lambda p: "-".join(f"{k}{v}" for k, v in p.items()))
def test_tiny_f32(params):
    g, o = tiny_case().run(O.F32, seed=4001, **params)
    assert_parity(g, o)


@pytest.mark.parametrize("storage", [O.F16, O.E4M3])
@pytest.mark.parametrize("rerank", [0, 1])
@pytest.mark.parametrize("width", [1, 3])
def test_tiny_low_precision(storage, rerank, width):
    g, o = tiny_case().run(storage, seed=4001, itopk=64, max_iters=64, entry=1, dgs_discard=0.5, rerank=rerank,
                           search_width=width)
    assert_parity(g, o)


@pytest.mark.parametrize("storage", [O.F16, O.E4M3])
def test_tiny_low_precision_min_match(storage):
    g, o = tiny_case().run(storage, seed=4001, itopk=64, max_iters=64, entry=1, dgs_min_match=0.55, rerank=1)
    assert_parity(g, o)


@pytest.mark.parametrize("storage", [O.F32, O.F16, O.E4M3])
@pytest.mark.parametrize("params", [dict(), dict(entry=1, dgs_discard=0.5), dict(search_width=3, itopk=48, k=7),
                                    dict(entry=1, dgs_discard=0.25, dgs_reexpand=1, rerank=1)])
def test_ragged_shapes(storage, params):
    if params.get("rerank") and storage == O.F32:
        params = dict(params, rerank=0)
    g, o = ragged_case().run(storage, seed=11, max_iters=70, **params)
    assert_parity(g, o)


@pytest.mark.parametrize("storage", [O.F32, O.F16])
def test_integer_ties(storage):
    g, o = int_case().run(storage, seed=3, itopk=128, k=100, max_iters=150, entry=1, dgs_discard=0.5,
                          rerank=int(storage != O.F32))
    assert_parity(g, o)


def test_given_ghost_seeds_with_fallback():
    c = tiny_case()
    rng = np.random.default_rng(5)
    given = rng.integers(0, len(c.S), size=(len(c.Q), 8)).astype(np.uint32)
    given[::3, 0] = O.INVALID
    g, o = c.run(O.F32, given=given, seed=4001, itopk=64, max_iters=64, entry=2)
    assert_parity(g, o)


def test_given_ghost_seeds_with_judge():
    """The judge of given seeds continues some queries' ghost stage and not
    others' (median distance), as the oracle does."""
    c = tiny_case()
    rng = np.random.default_rng(6)
    given = rng.integers(0, len(c.S), size=(len(c.Q), 2)).astype(np.uint32)
    given[::5, 0] = O.INVALID
    p = dict(seed=4001, itopk=64, max_iters=64, entry=2, ghost_itopk=32, ghost_max_iters=16,
             ghost_max_iters_given=1)
    best = c.run(O.F32, given=given, **dict(p, k=1, itopk=32, max_iters=0))[1][1][:, 0]
    judge = float(np.median(best))
    g, o = c.run(O.F32, given=given, ghost_judge=judge, **p)
    assert_parity(g, o)
    far = best > np.float32(judge)
    assert (o[2]["ghost_iters"][far & (given[:, 0] != O.INVALID)] > 1).any()


def test_full_queue_is_brute_force_on_gpu():
    # queue larger than the graph: the search is exhaustive
    c = ragged_case(n=400, d=40, deg=12, nq=9, gdeg=6, seed=13)
    g, o = c.run(O.F32, seed=1, itopk=512, k=10, max_iters=5000, search_width=8)
    assert_parity(g, o)
    gt, gd = O.knn_f64(c.X, c.Q, 10)
    np.testing.assert_allclose(g[1], gd, rtol=1e-5)
    assert (g[2]["vec_rows"] == 400).all()


def test_qid_base_and_seed_change_the_stream():
    c = tiny_case()
    g1, o1 = c.run(O.F32, seed=1, qid_base=1000, itopk=32, max_iters=20)
    assert_parity(g1, o1)
    g2, _ = c.run(O.F32, seed=2, qid_base=1000, itopk=32, max_iters=20)
    assert not np.array_equal(g1[2]["vec_rows"], g2[2]["vec_rows"]) or not np.array_equal(g1[0], g2[0])


def test_search_host_equals_device_search():
    c = tiny_case()
    gi = c.gpu_index(O.F32)
    ids, dists = gi.search_host(c.Q, seed=4001, entry=1, dgs_discard=0.5)
    g, _ = c.run(O.F32, seed=4001, entry=1, dgs_discard=0.5)
    assert np.array_equal(ids, g[0]) and np.array_equal(dists, g[1])


def test_empty_batch_and_errors():
    import paper_2507_17094_gb300 as A
    c = tiny_case()
    gi = c.gpu_index(O.F32)
    q = torch.zeros((0, 128), device="cuda")
    ids, dists, _ = gi.search(q)
    assert ids.shape == (0, 10)
    with pytest.raises(A.AnnError):
        gi.search(torch.zeros((1, 128), device="cuda"), k=65, itopk=64)
    with pytest.raises(A.AnnError):
        gi.search(torch.zeros((1, 128), device="cuda"), itopk=1024)
    with pytest.raises(A.AnnError):
        gi.search(torch.zeros((1, 128), device="cuda"), rerank=1, entry=2)   # given seeds missing
    with pytest.raises(A.AnnError):
        gi.search(torch.zeros((1, 128), device="cuda"), dgs_min_match=0.5, dgs_discard=0.5)   # alternatives
    with pytest.raises(A.AnnError):
        gi.search(torch.zeros((1, 128), device="cuda"), dgs_min_match=1.5)


def test_searches_on_two_streams_of_one_index():
    """Searches of one index launched on different streams share its visited
    tables and work counter; the library orders them, so each result equals
    the same search run alone."""
    c = tiny_case()
    gi = c.gpu_index(O.F32)
    Q = torch.from_numpy(c.Q).cuda()
    p1 = dict(seed=11, entry=1, dgs_discard=0.5, itopk=64, max_iters=64)
    p2 = dict(seed=12, entry=0, itopk=32, max_iters=40)
    a1, d1, _ = gi.search(Q, **p1)
    a2, d2, _ = gi.search(Q, **p2)
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for _ in range(4):
        with torch.cuda.stream(s1):
            outs.append((1, gi.search(Q, stream=s1, **p1)))
        with torch.cuda.stream(s2):
            outs.append((2, gi.search(Q, stream=s2, **p2)))
    torch.cuda.synchronize()
    gi.sync()
    for which, (ids, dists, _) in outs:
        want = (a1, d1) if which == 1 else (a2, d2)
        assert torch.equal(ids, want[0]) and torch.equal(dists, want[1])


@pytest.mark.parametrize("params", [dict(itopk=256, max_iters=400, search_width=4),
                                    dict(itopk=512, k=50, max_iters=800, search_width=8, entry=1),
                                    dict(itopk=64, max_iters=200, search_width=2, dgs_discard=0.5)])
def test_visited_set_under_collisions(params):
    """Equal ids inserted by several lanes at once, long probe runs and a
    table filled towards its reset threshold: results still match the
    oracle's exact visited set."""
    from gpu_cases import hub_case
    g, o = hub_case().run(O.F32, seed=5, **params)
    assert_parity(g, o)


def test_bounded_wait_timeout_is_reported_and_recoverable():
    """A device wait on a barrier nothing completes runs out, is reported
    through the error word as ANN_ETIMEOUT, and the index keeps working."""
    c = tiny_case()
    gi = c.gpu_index(O.F32)
    gi.selftest_timeout()
    gi.sync()                                   # the error word was cleared
    g, o = c.run(O.F32, seed=4001, itopk=64, max_iters=64, entry=1)
    assert_parity(g, o)


@pytest.mark.parametrize("params", [dict(itopk=32, max_iters=48, entry=1, dgs_discard=0.75, ghost_search_width=4,
                                         ghost_max_iters=12),
                                    dict(itopk=64, max_iters=64, entry=0, rerank=1)])
def test_search_profile_same_results_and_phases(params):
    """The profiling build returns what ann_search returns, and charges
    cycles to the phases that ran: no ghost stage without ghost entry, no
    DGS cycles without DGS."""
    import paper_2507_17094_gb300 as A
    c = tiny_case()
    storage = O.F16 if params.get("rerank") else O.F32
    gi = c.gpu_index(storage)
    Q = torch.from_numpy(c.Q).cuda()
    ids, d, _ = gi.search(Q, seed=3, **params)
    pids, pd, cyc = gi.search_profile(Q, seed=3, **params)
    torch.cuda.synchronize()
    assert torch.equal(ids, pids) and torch.equal(d, pd)
    S = {n: i for i, n in enumerate(A.PROFILE_STAGE_NAMES)}
    P = {n: i for i, n in enumerate(A.PROFILE_PHASE_NAMES)}
    base = cyc[S["base"]]
    assert base[P["select+adjacency"]] > 0 and base[P["gather_wait"]] > 0 and base[P["distance"]] > 0
    assert base[P["merge"]] > 0 and base[P["visited"]] > 0
    assert (cyc[S["ghost"]].sum() > 0) == (params["entry"] == 1)
    assert (base[P["dgs"]] > 0) == (params.get("dgs_discard", 0) > 0)
    assert cyc[:, P["unused"]].sum() == 0
    if params.get("rerank"):
        assert cyc[S["finish"], P["distance"]] > 0
