"""Learned entry end to end on the GPU: labels from the method's own ghost
staging, MLP training by the library's kernels, and the gain over plain ghost
staging on held-out queries (20% drawn between clusters)."""
import dataclasses
import time

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    import paper_2507_17094_gb300 as A
    from workloads import WORKLOADS, build_graph, ghost_sample, make_queries
    assert torch.cuda.is_available()
    A.build()
    spec = dataclasses.replace(WORKLOADS[2].scaled(200_000, nq=2000, n_clusters=200, ghost_n=2000))
    X, _ = spec.mixture().sample(spec.n, spec.seeds["base"])
    G = build_graph(X, spec.degree, spec.knn_k, "partitioned", n_parts=200, seed=1)
    S = ghost_sample(spec.n, spec.ghost_n, spec.seeds["ghost"])
    Gg = build_graph(X[S], spec.ghost_degree, 2 * spec.ghost_degree, "exact", seed=2)
    Qtrain = make_queries(spec, nq=40_000, seed=spec.seeds["query"] + 100)
    Qval = make_queries(spec, nq=2000, seed=spec.seeds["query"] + 200)
    Qtest = make_queries(spec, nq=2000, seed=spec.seeds["query"] + 300, off_fraction=0.2)
    ix = A.Index(X, G, storage=A.F32, ghost_ids=S, ghost_graph=Gg)
    yield dict(A=A, spec=spec, X=X, G=G, S=S, Gg=Gg, Qtrain=Qtrain, Qval=Qval, Qtest=Qtest, ix=ix)
    ix.close()


def test_labels_are_the_ghost_stage_top1(setup):
    from paper_2507_17094_gb300.entry import ghost_labels
    s = setup
    Q = s["Qtrain"][:300]
    lab = ghost_labels(s["ix"], torch.from_numpy(Q).cuda(), seed=7).cpu().numpy().view(np.uint32)
    oi = O.OracleIndex(s["X"], s["G"], O.F32, s["S"], s["Gg"], with_dir=False)
    ids, _, _ = O.search(oi, Q, k=1, itopk=64, max_iters=0, entry=1, ghost_itopk=64, ghost_max_iters=64, seed=7)
    want = np.searchsorted(s["S"], ids[:, 0]).astype(np.uint32)
    assert np.array_equal(s["S"][want], ids[:, 0])
    assert np.array_equal(lab, want)


def test_ghost_index_of_marks_non_ghost_nodes(setup):
    s = setup
    S = s["S"]
    ids = np.concatenate([S[::7], np.setdiff1d(np.arange(5000, dtype=np.uint32), S)[:50]]).astype(np.uint32)
    got = s["ix"].ghost_index_of(torch.from_numpy(ids.view(np.int32)).cuda()).cpu().numpy().view(np.uint32)
    assert np.array_equal(got[: len(S[::7])], np.arange(0, len(S), 7, dtype=np.uint32))
    assert (got[len(S[::7]):] == O.INVALID).all()


def test_learned_entry_beats_plain_ghost_staging(setup):
    from paper_2507_17094_gb300.entry import LearnedEntry, ghost_labels
    from workloads import init_mlp_params
    s = setup
    A, ix, spec = s["A"], s["ix"], s["spec"]
    Qtr, Qva, Qte = (torch.from_numpy(q).cuda() for q in (s["Qtrain"], s["Qval"], s["Qtest"]))
    ytr = ghost_labels(ix, Qtr, seed=11)
    yva = ghost_labels(ix, Qva, seed=11)
    le = LearnedEntry(ix, init_mlp_params(spec.d, 512, 512, spec.ghost_n, spec.seeds["mlp"]))
    losses = le.fit(Qtr, ytr, epochs=8, batch=1024, lr=1e-3, seed=3)
    assert losses[-1] < 0.5 * losses[0], losses
    tau, val_hit = le.calibrate(Qva, yva)
    assert val_hit > 0.8, val_hit
    gt, gd = O.knn_f64(s["X"], s["Qtest"], 10)
    common = dict(k=10, itopk=32, max_iters=96, dgs_discard=0.5, seed=11, ghost_itopk=32)

    def run(**kw):
        ids, _, st = ix.search(Qte, stats=True, **common, **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            ix.search(Qte, **common, **kw)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) / 5 * 1e3
        rec = O.recall_at_k(ids.cpu().numpy().view(np.uint32), gt, gd, s["X"], s["Qtest"], 10)[0]
        return rec, A.stats_to_numpy(st), ms

    r_gs, st_gs, ms_gs = run(entry=1, ghost_max_iters=64)
    seeds, pmax = le.seeds(Qte)
    r_le, st_le, ms_le = run(entry=2, given=seeds, ghost_max_iters=64, ghost_max_iters_given=4)
    from workloads import off_distribution_mask
    fb = (seeds[:, 0] == -1).cpu().numpy()
    off = off_distribution_mask(spec, 0.2, nq=len(fb), seed=spec.seeds["query"] + 300)
    _, pv = le.seeds(Qva)
    fb_val = float((pv.cpu().numpy() < np.float32(tau)).mean())
    print(f"ghost staging: recall {r_gs:.3f}, ghost rows {st_gs['ghost_vec_rows'].mean():.0f}, "
          f"ghost iters {st_gs['ghost_iters'].mean():.1f}, {ms_gs:.2f} ms | learned: recall {r_le:.3f}, "
          f"ghost rows {st_le['ghost_vec_rows'].mean():.0f}, ghost iters {st_le['ghost_iters'].mean():.1f}, "
          f"{ms_le:.2f} ms, fallback validation {fb_val:.3f} test in/off {fb[~off].mean():.3f}/"
          f"{fb[off].mean():.3f}, tau {tau:.3g}")
    assert r_le >= r_gs - 0.01
    assert st_le["ghost_vec_rows"].mean() < 0.5 * st_gs["ghost_vec_rows"].mean()
    # tau is the validation split's 5% quantile: that share of it falls back
    assert abs(fb_val - 0.05) <= 0.005
    # the judge continues the queries whose ghost result stays far after the
    # short stage: at least the learned recall, fewer ghost rows than plain
    # ghost staging
    judge = le.calibrate_judge(Qva, continue_fraction=0.05, **common, ghost_max_iters=64, ghost_max_iters_given=4)
    assert judge > 0
    r_j, st_j, _ = run(entry=2, given=seeds, ghost_max_iters=64, ghost_max_iters_given=4, ghost_judge=judge)
    print(f"judged: recall {r_j:.3f}, ghost rows {st_j['ghost_vec_rows'].mean():.0f}, continued in/off "
          f"{(st_j['ghost_iters'][~off] > 4).mean():.3f}/{(st_j['ghost_iters'][off] > 4).mean():.3f}")
    assert r_j >= r_le - 0.005
    assert st_j["ghost_vec_rows"].mean() < st_gs["ghost_vec_rows"].mean()
    le.close()
