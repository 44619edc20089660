"""The benchmark's own FP64 ground truth and recall agree with the oracle's
(the benchmark runs the oracle only in its CPU-baseline leg)."""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")


def test_truth_knn_and_recall_match_the_oracle():
    import bench
    rng = np.random.default_rng(5)
    X = rng.integers(0, 6, (3000, 12)).astype(np.float32)       # many exact ties
    Q = rng.integers(0, 6, (40, 12)).astype(np.float32)
    ids, d = bench.truth_knn(X, Q, 10, "cpu")
    o_ids, o_d = O.knn_f64(X, Q, 10)
    assert np.array_equal(d, o_d)
    assert np.array_equal(ids, o_ids)
    # recall of a perturbed answer set, both definitions
    ann = o_ids.copy()
    ann[::3, 4:] = rng.integers(0, 3000, ann[::3, 4:].shape).astype(np.uint32)
    ann[1, 9] = 0xFFFFFFFF
    ann[2, 8] = ann[2, 7]
    want = O.recall_at_k(ann, o_ids, o_d, X, Q, 10)[0]
    got = bench.recall_at(ann.view(np.int32), d, X, Q, 10)
    assert abs(got - want) < 1e-12
    assert np.array_equal(bench.pair_dist(X, Q, ann[:, :5]), O.pair_dist_f64(X, Q, ann[:, :5]))


def test_form_selection_and_operating_points():
    import bench
    from workloads import WORKLOADS
    forms = bench.forms_for(WORKLOADS[2])
    default = bench.selected_forms(forms, "")
    assert "paper_fp32" in default and "simdgs_fp32" not in default      # optional forms only on request
    assert bench.selected_forms(forms, "simdgs_fp32,paper_fp32") == ["paper_fp32", "simdgs_fp32"]
    sim = forms["simdgs_fp32"]
    assert sim["dgs_discard"] == 0.0 and 0.0 < sim["dgs_min_match"] <= 1.0   # the two rules are alternatives
    p = bench.params_for(forms["paper_fp32"], 32, 7)
    assert p["itopk"] == 32 and p["max_iters"] == 32 + 16 and "storage" not in p


def test_side_legs_keep_to_the_wall_budget(monkeypatch):
    """A side leg that would start with too little budget left is skipped; one
    that runs past its deadline is ended (its whole process group) and
    recorded, so the benchmark's line is still printed."""
    import argparse
    import subprocess
    import time
    import bench
    args = argparse.Namespace(budget_s=0.0, steps=3, warmup=3, gt_sample=10, train_queries=10, epochs=1,
                              serve_requests=1)
    assert "skipped" in bench.run_leg_child("3", args, 0, False)

    real_popen = subprocess.Popen
    monkeypatch.setattr(bench, "MIN_LEG_S", 1.0)
    monkeypatch.setattr(bench.subprocess, "Popen",
                        lambda cmd, **kw: real_popen(["sleep", "30"], **kw))
    args.budget_s = (time.time() - bench.T_START) + bench.FINAL_RESERVE_S + 2.0
    t0 = time.time()
    res = bench.run_leg_child("3", args, 0, False)
    assert "ended at the wall budget" in res["skipped"]
    assert time.time() - t0 < 10.0


def test_side_leg_registry_and_failed_child(monkeypatch):
    """Every default side leg has a runner and a result key; a child that
    exits with an error is recorded as failed, not parsed."""
    import argparse
    import subprocess
    import time
    import bench
    for w in bench.DEFAULT_LEGS.split(","):
        assert w in bench.LEG_FNS and w in bench.LEG_KEYS
    real_popen = subprocess.Popen
    monkeypatch.setattr(bench.subprocess, "Popen",
                        lambda cmd, **kw: real_popen(["sh", "-c", "echo '{\"partial\": 1}'; exit 3"], **kw))
    args = argparse.Namespace(budget_s=(time.time() - bench.T_START) + bench.FINAL_RESERVE_S + bench.MIN_LEG_S + 60,
                              steps=3, warmup=3, gt_sample=10, train_queries=10, epochs=1, serve_requests=1)
    res = bench.run_leg_child("4", args, 0, False)
    assert res["failed"] == "child exited 3"
