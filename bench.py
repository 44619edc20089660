#!/usr/bin/env python3
"""Benchmark: batched graph beam search on one GB300 (PathWeaver's hot path).

Metric: queries per second at recall@10 >= 0.95 (tie-aware, against the FP64
exact kNN of the CPU oracle), on the 1M x 96-d workload (1,000 anisotropic
Gaussians, L2-normalised, degree-64 graph, 10,000 queries, k = 10). The
queue size itopk is swept over {16, 32, 64, 128, 256} and the fastest setting
reaching the recall target is timed.

A step is one batched search of all queries: entry (ghost staging), the
iterations with DGS, merges and output, in the library's search kernel,
launched through the C ABI. Inputs are resident in HBM when the timed region
starts; L2 is flushed between steps (a 256 MB write outside the timed
events). ``e2e`` repeats the measurement through ann_search_host with host
buffers, so host<->device copies are inside its timed region.

``--impl reference`` times the CPU oracle (the same search, plain C, all host
cores) on a bounded sample of the same workload and prints the same line.
Under torchrun with N > 1 every rank searches its own replica and the value
is the whole job's queries over the slowest rank's time.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

T_START = time.time()
ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QPS at recall@10>=0.95 on 1 GB300: plain FP32 vs FP16/FP8+learned entry"
UNIT = "queries/s"
RECALL_TARGET = 0.95
SWEEP = (16, 32, 64, 128, 256)
KERNEL_SOURCES = ("paper_2507_17094_gb300/csrc/search.cu", "paper_2507_17094_gb300/csrc/ann_internal.cuh")


# ------------------------------------------------------------------ helpers
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def dist_init(world: int, backend: str):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist if world > 1 else None


def max_over_ranks(value: float, dist, device=None) -> float:
    """The slowest rank's time (the job finishes with it)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist, device=None) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d.get("bf16_tflops", 1900.0)),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str, form: str):
    """DRAM bytes per launch of the search kernel from the committed ncu
    summary (a line 'traffic <workload> <form>: <bytes> bytes per launch,
    kernel source <hash>'), if it was taken on the current kernel source."""
    import re
    p = os.path.join(ROOT, "profiles", "search_kernel_scale-1M-96d.md")
    if not os.path.exists(p):
        return None
    pat = re.compile(r"traffic (\S+) (\S+): (\d+) bytes per launch, kernel source ([0-9a-f]+)")
    for line in open(p):
        m = pat.search(line)
        if m and m.group(1) == workload and m.group(2) == form and m.group(4) == kernel_hash():
            return {"dram_bytes_per_launch": int(m.group(3))}
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ forms
# Operating points on the 1M x 96 workload (measured sweeps at itopk 32).
# Ghost staging from random ghost seeds: ghost-stage length 8-64 with 1, 2
# or 4 parents per ghost iteration, DGS discard 0.5-0.75, iteration cap
# itopk + 16 or 2 itopk + 32; 12 ghost iterations of 4 parents, discard
# 0.75 and cap itopk + 16 reach recall@10 0.967 at 7.5M QPS (one parent per
# ghost iteration needs 48 iterations for 0.968 at 6.9M; 8 iterations of 4
# fall to 0.948). From the learned entry's seeds (2 or 4 ghost iterations of
# 1, 2 or 4 parents, discard 0.5 or 0.6, itopk 16): 2 iterations of one
# parent and discard 0.5 reach 0.967 at 9.8M QPS with the prediction
# included (4 parents: 9.0M); the few queries below the confidence
# threshold fall back to one-parent ghost staging of 48 iterations.
GHOST_ITERS = 12
GHOST_WIDTH = 4
DGS_DISCARD = 0.75
# DGS by a similarity threshold: keep the neighbours agreeing with the query
# in >= ceil(0.65 d) dimensions (measured on workload 2: recall 0.963 at
# itopk 32, as the top-n rule at discard 0.75). Optional forms run only
# when named in --forms.
SIM_MATCH = 0.65
OPTIONAL_FORMS = ("simdgs_fp32",)
DGS_DISCARD_LEARNED = 0.5
LEARNED = dict(dgs_discard=DGS_DISCARD_LEARNED, ghost_max_iters_given=2, ghost_max_iters=48, ghost_search_width=1)


def forms_for(spec):
    """Search configurations compared (each swept over itopk)."""
    base = dict(k=10, search_width=1, dgs_cooldown=0.3, ghost_max_iters=GHOST_ITERS, ghost_search_width=GHOST_WIDTH)
    return {
        # the paper's method: ghost staging + DGS, FP32 storage (headline)
        "paper_fp32": dict(storage=0, entry=1, dgs_discard=DGS_DISCARD, rerank=0, **base),
        # the method without its two techniques (CAGRA-style random entry)
        "plain_fp32": dict(storage=0, entry=0, dgs_discard=0.0, rerank=0, **base),
        # low-precision storage with FP32 rerank of the final queue
        "f16_rerank": dict(storage=1, entry=1, dgs_discard=DGS_DISCARD, rerank=1, **base),
        "e4m3_rerank": dict(storage=2, entry=1, dgs_discard=DGS_DISCARD, rerank=1, **base),
        # low precision + learned entry: the MLP's top-8 ghost nodes seed a
        # 2-iteration ghost stage (fallback to ghost staging below tau)
        "f16_learned": dict(base, storage=1, entry=2, rerank=1, **LEARNED),
        "e4m3_learned": dict(base, storage=2, entry=2, rerank=1, **LEARNED),
        # ghost staging + DGS by a similarity threshold instead of a fixed
        # top n (the alternative the paper names), FP32
        "simdgs_fp32": dict(storage=0, entry=1, dgs_discard=0.0, dgs_min_match=SIM_MATCH, rerank=0, **base),
    }


def selected_forms(forms: dict, arg: str) -> list:
    """Forms a run measures: those named in --forms, else every form but the
    optional ones."""
    if arg:
        named = arg.split(",")
        return [n for n in forms if n in named]
    return [n for n in forms if n not in OPTIONAL_FORMS]


def params_for(form: dict, L: int, seed: int) -> dict:
    p = {k: v for k, v in form.items() if k != "storage"}
    p.update(itopk=L, max_iters=L // form["search_width"] + 16, seed=seed)
    return p


def train_entry(ds, spec, index, dev, verbose, n_train=200_000, epochs=8, judge_params=None):
    """The learned entry for this workload: labels from ghost staging on
    200,000 training queries, 8 epochs of AdamW, tau from a validation split
    and, with `judge_params` (the ghost settings of the search), labels from
    that ghost stage and the judge distance from the same split."""
    import torch
    from paper_2507_17094_gb300.entry import LearnedEntry, ghost_labels
    from workloads import init_mlp_params, make_queries
    t0 = time.time()
    Qtr = torch.from_numpy(make_queries(spec, nq=n_train, seed=spec.seeds["query"] + 100)).to(dev)
    Qva = torch.from_numpy(make_queries(spec, nq=5_000, seed=spec.seeds["query"] + 200)).to(dev)
    # labels from the search's own ghost stage when its settings are given
    lab = {k: judge_params[k] for k in ("ghost_itopk", "ghost_max_iters", "ghost_search_width")
           if judge_params and k in judge_params}
    ytr = ghost_labels(index, Qtr, seed=spec.seeds["search"], **lab)
    yva = ghost_labels(index, Qva, seed=spec.seeds["search"], **lab)
    le = LearnedEntry(index, init_mlp_params(spec.d, 512, 512, spec.ghost_n, spec.seeds["mlp"]))
    losses = le.fit(Qtr, ytr, epochs=epochs, batch=1024, lr=1e-3, seed=spec.seeds["mlp"])
    tau, hit = le.calibrate(Qva, yva)
    if judge_params is not None:
        le.calibrate_judge(Qva, seed=spec.seeds["search"], **judge_params)
    info = {"train_queries": n_train, "epochs": epochs, "loss_first_last": [float(losses[0]), float(losses[-1])],
            "val_label_in_top8": hit, "tau": tau, "ghost_judge": le.judge, "train_s": time.time() - t0,
            "mlp": f"{spec.d}->512->512->{spec.ghost_n}"}
    if verbose:
        print(f"[bench] learned entry: {info}", file=sys.stderr, flush=True)
    return le, info


def algorithmic_bytes(st, spec, storage: int, rerank: bool) -> np.ndarray:
    """Bytes the search must move per query (from the kernel's own exact
    counters): query + adjacency rows + direction rows + gathered vector rows
    (ghost and base, with the per-vector scale) + FP32 rerank rows + results."""
    d, deg, k = spec.d, spec.degree, 10
    w = (d + 31) // 32
    eb = {0: 4, 1: 2, 2: 1}[storage]
    row = d * eb + (4 if storage else 0)
    return (4 * d + st["parents"].astype(np.int64) * 4 * deg
            + st["dgs_parents"].astype(np.int64) * 4 * deg * w
            + st["vec_rows"].astype(np.int64) * row
            + st["ghost_parents"].astype(np.int64) * 4 * spec.ghost_degree
            + st["ghost_vec_rows"].astype(np.int64) * row
            + st["rerank_rows"].astype(np.int64) * 4 * d * (1 if rerank else 0)
            + 8 * k)


# ------------------------------------------------------------------ serving leg
def serve_leg(A, index, entry, ds, spec, args):
    """Poisson arrivals of query batches (sizes uniform in 1..4,096, k in
    {10, 100}, itopk in {64, 256}) into the continuous-batching server on the
    FP16 index, with the learned entry when one was trained (else ghost
    staging). First the same trace arrives all at once (the server's capacity
    in queries per second), then at half that load as a Poisson process: the
    per-request latency percentiles there are the serving latency."""
    rng = np.random.default_rng(spec.seeds["search"] + 7)
    learned = entry is not None
    base = dict(entry=2 if learned else 1, dgs_discard=0.5, ghost_max_iters=64, ghost_max_iters_given=4,
                rerank=1, seed=spec.seeds["search"])
    srv = A.Server(index, capacity=65536, max_requests=128,
                   max_params=dict(k=100, itopk=256, max_iters=544, ghost_itopk=64, **base),
                   mlp=entry.mlp if learned else None, seeds_per_query=8, tau=entry.tau if learned else 0.0)
    reqs = []
    for rid in range(args.serve_requests):
        n = int(rng.integers(1, 4097))
        off = int(rng.integers(0, len(ds.Q) - n))
        k = int(rng.choice([10, 100]))
        L = max(k, int(rng.choice([64, 256])))      # a queue holds at least the k results
        reqs.append((rid, ds.Q[off:off + n], dict(k=k, itopk=L, max_iters=2 * L + 32, qid_base=rid << 20, **base)))
    nq = sum(len(q) for _, q, _ in reqs)
    warm = [(0.0, 10**9 + i, ds.Q[:64], dict(reqs[0][2], qid_base=0)) for i in range(4)]
    A.replay(srv, warm)

    def play(rate):
        t, trace = 0.0, []
        for rid, q, prm in reqs:
            if rate:
                t += float(rng.exponential(1.0 / rate))
            trace.append((t, rid, q, prm))
        res, wall = A.replay(srv, trace, timeout_s=300)
        lat = np.array([res[r][2] for _, r, _, _ in trace]) * 1e3
        return {"qps": nq / wall, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "offered_req_s": rate or None}

    burst = play(0.0)
    half_rate = 0.5 * burst["qps"] / (nq / len(reqs))
    half = play(half_rate)
    srv.close()
    return {"requests": len(reqs), "queries": nq, "capacity_qps": burst["qps"],
            "qps": half["qps"], "p50_ms": half["p50_ms"], "p99_ms": half["p99_ms"],
            "offered_rate_req_s": half_rate, "offered_qps": 0.5 * burst["qps"],
            "all_at_once": burst, "entry": "learned" if learned else "ghost", "storage": "f16",
            "mix": "batch 1-4096 uniform, k {10,100}, itopk {64,256} raised to k, Poisson arrivals at half "
                   "the measured capacity"}


# ------------------------------------------------------------------ evaluation
# Ground truth and recall for the measurement, computed here in FP64 (torch on
# the device for the shortlist, numpy for the exact distances); the CPU oracle
# is only run in the CPU-baseline leg and the reference arm.
def truth_knn(X: np.ndarray, Q: np.ndarray, k: int, dev, shortlist: int = 64):
    """Exact k nearest neighbours (squared L2, FP64, ties by smaller id): an
    FP64 expanded-form shortlist of `shortlist` ids on the device, then the
    direct form sum (q - x)^2 over the shortlist."""
    import torch
    Xt = torch.from_numpy(np.ascontiguousarray(X)).to(dev, torch.float64)
    xn = (Xt * Xt).sum(1)
    ids = np.empty((len(Q), k), dtype=np.uint32)
    dists = np.empty((len(Q), k), dtype=np.float64)
    step = int(max(16, min(256, 2_000_000_000 // max(1, Xt.shape[0]))))   # a chunk's FP64 matrix <= 16 GB
    for s0 in range(0, len(Q), step):
        q = torch.from_numpy(np.ascontiguousarray(Q[s0:s0 + step])).to(dev, torch.float64)
        d2 = xn[None, :] - 2.0 * (q @ Xt.T) + (q * q).sum(1)[:, None]
        cand = torch.topk(d2, min(shortlist, Xt.shape[0]), dim=1, largest=False).indices.cpu().numpy()
        for i in range(cand.shape[0]):
            c = np.sort(cand[i])
            ex = ((X[c].astype(np.float64) - Q[s0 + i].astype(np.float64)) ** 2).sum(1)
            o = np.lexsort((c, ex))[:k]
            ids[s0 + i] = c[o]
            dists[s0 + i] = ex[o]
    return ids, dists


def pair_dist(X: np.ndarray, Q: np.ndarray, ids: np.ndarray) -> np.ndarray:
    """FP64 squared L2 between each query and its listed ids."""
    safe = np.where(ids == 0xFFFFFFFF, 0, ids).astype(np.int64)
    return ((X[safe].astype(np.float64) - Q[:, None, :].astype(np.float64)) ** 2).sum(2)


def recall_at(ann_ids: np.ndarray, gt_dists: np.ndarray, X: np.ndarray, Q: np.ndarray, k: int = 10) -> float:
    """Tie-aware recall@k: a returned id is a hit when it is valid, not a
    repeat, and its FP64 distance is within the exact k-th distance."""
    a = np.ascontiguousarray(ann_ids[:, :k]).view(np.uint32)
    da = pair_dist(X, Q, a)
    kth = gt_dists[:, k - 1]
    hits = 0
    for i in range(a.shape[0]):
        seen = set()
        for j in range(k):
            v = int(a[i, j])
            if v != 0xFFFFFFFF and v not in seen and da[i, j] <= kth[i]:
                hits += 1
            seen.add(v)
    return hits / (a.shape[0] * k)


# ------------------------------------------------------------------ other workloads
# Operating points of workloads 3 and 4 (measured on the GB300; the
# diagnosis that chose them: recall on workload 3 was bounded by the ghost
# stage reaching the query's cluster -- 85% with a 64-entry one-parent ghost
# queue, 98-100% with 128-256 entries and 4 parents. On workload 4 the
# queries drawn between clusters set the bound: their true 10 nearest
# ghosts were found for 65% of them by a 128-entry 4-parent ghost stage and
# for 90% by a 512-entry 8-parent one, and their recall@10 at itopk 512
# rose from 0.67 to 0.82 (0.89 from the exact nearest ghosts).
W3_GHOST = dict(ghost_itopk=128, ghost_search_width=4, ghost_max_iters=32)
W3_GHOST_K100 = dict(ghost_itopk=256, ghost_search_width=4, ghost_max_iters=48)
W4_GHOST = dict(ghost_itopk=512, ghost_search_width=8, ghost_max_iters=64)
# Workload 5 (20,000 clusters, 200,000 ghosts): the ghost stage again sets
# recall@10 at itopk 64: 0.75 with a 64-entry 4-parent ghost queue, 0.84 with
# 128 entries, 0.93 with 256 entries, 0.96 with 256 entries and 8 parents.
W5_GHOST = dict(ghost_itopk=256, ghost_search_width=8, ghost_max_iters=48)


class Timer:
    """CUDA-event timing of a step on `stream`, L2 flushed before each step."""

    def __init__(self, dev, stream):
        import torch
        self.dev, self.stream = dev, stream
        self.flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def __call__(self, run, steps=3, warm=1):
        import torch
        for _ in range(warm):
            run()
        torch.cuda.synchronize(self.dev)
        ts = []
        for _ in range(steps):
            self.flush.add_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            run()
            e1.record(self.stream)
            ts.append((e0, e1))
        torch.cuda.synchronize(self.dev)
        return statistics.median(a.elapsed_time(b) for a, b in ts)


def sweep_forms(A, ds, spec, forms, timer, gt, verbose, tag, entries=None, subsets=None):
    """Each form: storage, fixed params, an itopk sweep and k. The smallest
    itopk reaching recall@10 >= 0.95 on the ground-truth sample is the
    form's operating point (else the best recall seen); there the line gets
    QPS (all queries), the counted HBM bytes and their fraction, the mean
    rows and, for low-precision storage, the distance error against FP64
    before and after the FP32 rerank. `subsets` (name -> boolean mask over
    the ground-truth sample) adds each sweep row's recall on those queries."""
    import torch
    dev, stream = timer.dev, timer.stream
    Qd = torch.from_numpy(ds.Q).to(dev)
    nq = Qd.shape[0]
    gt_ids, gt_d = gt
    ns = gt_ids.shape[0]
    indexes, res = {}, {}
    peak = measured_peaks()["hbm_gbs"]

    def index_for(storage):
        if storage not in indexes:
            indexes[storage] = A.Index(ds.X, ds.G, storage=storage, ghost_ids=ds.S, ghost_graph=ds.Gg,
                                       keep_fp32=True, build_dir=True, device=dev.index or 0)
        return indexes[storage]

    for name, f in forms.items():
        ix = index_for(f["storage"])
        le = (entries or {}).get(f["storage"]) if f["params"].get("entry") == 2 else None
        if f["params"].get("entry") == 2 and le is None:
            continue

        def run(p, stats=False, ix=ix, le=le):
            if le is not None:
                seeds, _ = le.seeds(Qd, stream=stream)
                return ix.search(Qd, given=seeds, stream=stream, stats=stats, **p)
            return ix.search(Qd, stream=stream, stats=stats, **p)

        sweep, chosen = [], None
        for L in f["sweep"]:
            p = dict(f["params"], k=f["k"], itopk=L, max_iters=L + 16, seed=spec.seeds["search"])
            ids, _, _ = run(p)
            torch.cuda.synchronize(dev)
            a = ids[:ns].cpu().numpy().view(np.uint32)
            rec = recall_at(a, gt_d, ds.X, ds.Q[:ns], 10)
            row = {"itopk": L, "recall": rec}
            for sname, m in (subsets or {}).items():
                row.setdefault("recall_by_subset", {})[sname] = recall_at(a[m], gt_d[m], ds.X, ds.Q[:ns][m], 10)
            if f["k"] >= 100 and gt_ids.shape[1] >= 100:
                row["recall_at_100"] = recall_at(a, gt_d, ds.X, ds.Q[:ns], 100)
            ms = timer(lambda: run(p))
            row.update(ms=ms, qps=nq / (ms / 1e3))
            sweep.append(row)
            if chosen is None and rec >= RECALL_TARGET:
                chosen = L
                break
        if chosen is None:
            chosen = max(sweep, key=lambda r: r["recall"])["itopk"]
        at = next(r for r in sweep if r["itopk"] == chosen)
        p = dict(f["params"], k=f["k"], itopk=chosen, max_iters=chosen + 16, seed=spec.seeds["search"])
        _, _, st = run(p, stats=True)
        torch.cuda.synchronize(dev)
        stn = A.stats_to_numpy(st)
        b = float(algorithmic_bytes(stn, spec, f["storage"], bool(p.get("rerank"))).sum())
        gbs = b / (at["ms"] / 1e3) / 1e9
        r = {"storage": ("f32", "f16", "e4m3")[f["storage"]], "k": f["k"], "itopk": chosen,
             "params": {k: v for k, v in p.items() if k not in ("itopk", "seed")},
             "recall": at["recall"], "qps": at["qps"], "ms_per_step": at["ms"], "gbs": gbs, "hbm_frac": gbs / peak,
             "mean_vec_rows": float(stn["vec_rows"].mean()), "mean_ghost_rows": float(stn["ghost_vec_rows"].mean()),
             "mean_iters": float(stn["iters"].mean()), "sweep": sweep}
        if "recall_at_100" in at:
            r["recall_at_100"] = at["recall_at_100"]
        if p.get("entry") == 2:
            # queries whose ghost stage ran past the seeds' short stage (fallback by tau, or the judge)
            full = stn["ghost_iters"] > p.get("ghost_max_iters_given", 4)
            r["full_ghost_stage_fraction"] = float(full.mean())
            for sname, m in (subsets or {}).items():
                r.setdefault("full_ghost_stage_by_subset", {})[sname] = float(full[:ns][m].mean())
        if f["storage"] != 0:
            errs = {}
            for tagr, rr in (("stored", 0), ("reranked", 1)):
                ids_e, d_e, _ = run(dict(p, rerank=rr))
                torch.cuda.synchronize(dev)
                ie = ids_e[:ns].cpu().numpy().view(np.uint32)
                de = d_e[:ns].cpu().numpy().astype(np.float64)
                ok = ie != 0xFFFFFFFF
                ex = pair_dist(ds.X, ds.Q[:ns], np.where(ok, ie, 0).astype(np.uint32))
                rel = np.abs(de - ex)[ok] / np.maximum(ex[ok], 1e-30)
                errs[tagr] = {"max_rel": float(rel.max()), "mean_rel": float(rel.mean()),
                              "exact_fraction": float((de[ok] == ex[ok]).mean())}
            r["distance_error_vs_fp64"] = errs
        if le is not None:
            pred_ms = timer(lambda: le.seeds(Qd, stream=stream), steps=5, warm=2)
            flop = 2.0 * nq * (spec.d * 512 + 512 * 512 + 512 * spec.ghost_n)
            tf = flop / (pred_ms / 1e3) / 1e12
            pk = measured_peaks()["bf16_tflops"]
            r["predict"] = {"ms": pred_ms, "fallback_fraction": le.fallback_fraction(le.seeds(Qd)[0]),
                            "roofline": {"bound": "tensor", "achieved": tf, "peak": pk, "unit": "TFLOP/s",
                                         "frac": tf / pk, "flop_per_step": flop}}
        res[name] = r
        if verbose:
            print(f"[bench] {tag} {name}: " + ", ".join(f"L{s['itopk']} r={s['recall']:.3f} {s['qps'] / 1e6:.2f}M/s"
                                                      for s in sweep), file=sys.stderr, flush=True)
    for ix in indexes.values():
        ix.close()
    return res


def leg_workload3(A, args, timer, verbose):
    """Workload 3 (10M x 128 integers): FP32 against FP16 / E4M3 storage with
    FP32 rerank, k = 10 and k = 100."""
    from workloads import WORKLOADS, load_dataset
    spec = WORKLOADS[3]
    t0 = time.time()
    ds = load_dataset(spec, device=timer.dev, verbose=verbose)
    gt = truth_knn(ds.X, ds.Q[:args.gt_sample], 100, timer.dev, shortlist=128)
    base = dict(entry=1, dgs_discard=0.5, dgs_cooldown=0.3, **W3_GHOST)
    k100 = dict(entry=1, dgs_discard=0.5, dgs_cooldown=0.3, **W3_GHOST_K100)
    sw = (32, 64, 128, 256)
    forms = {
        "paper_fp32": dict(storage=0, k=10, sweep=sw, params=dict(base, rerank=0)),
        "f16_rerank": dict(storage=1, k=10, sweep=sw, params=dict(base, rerank=1)),
        "e4m3_rerank": dict(storage=2, k=10, sweep=sw, params=dict(base, rerank=1)),
        "f16_rerank_k100": dict(storage=1, k=100, sweep=(128, 256, 512), params=dict(k100, rerank=1)),
        "e4m3_rerank_k100": dict(storage=2, k=100, sweep=(128, 256, 512), params=dict(k100, rerank=1)),
    }
    res = sweep_forms(A, ds, spec, forms, timer, gt, verbose, "w3")
    return {"workload": spec.name, "n": spec.n, "dim": spec.d, "degree": spec.degree, "nq": spec.nq,
            "gt_sample": int(gt[0].shape[0]), "forms": res, "leg_s": time.time() - t0}


def leg_workload4(A, args, timer, verbose):
    """Workload 4 (5M x 256, Zipf cluster sizes, ghost set 50,000): plain
    ghost staging against the learned entry (MLP 256 -> 512 -> 512 ->
    50,000 trained on the GPU), FP32 and FP16 / E4M3 with rerank. Recall is
    also split into the in-distribution queries and the 20% drawn between
    clusters."""
    from workloads import WORKLOADS, load_dataset, off_distribution_mask
    spec = WORKLOADS[4]
    t0 = time.time()
    ds = load_dataset(spec, off_fraction=0.2, device=timer.dev, verbose=verbose)
    gt = truth_knn(ds.X, ds.Q[:args.gt_sample], 10, timer.dev)
    sw = (64, 128, 256, 512)
    ghost = dict(entry=1, dgs_discard=0.5, dgs_cooldown=0.3, **W4_GHOST)
    learned = dict(entry=2, dgs_discard=0.5, dgs_cooldown=0.3, ghost_max_iters_given=4, **W4_GHOST)
    entries, info = {}, {}
    ix16 = A.Index(ds.X, ds.G, storage=1, ghost_ids=ds.S, ghost_graph=ds.Gg, keep_fp32=True, build_dir=False,
                   device=timer.dev.index or 0)
    le, info = train_entry(ds, spec, ix16, timer.dev, verbose, args.train_queries, args.epochs,
                           judge_params=dict(ghost_max_iters_given=4, **W4_GHOST))
    learned["ghost_judge"] = le.judge
    for st_ in (0, 1, 2):
        entries[st_] = le    # the network predicts ghost indices: one model serves every storage
    ix16.close()
    forms = {
        "paper_fp32": dict(storage=0, k=10, sweep=sw, params=dict(ghost, rerank=0)),
        "f16_ghost": dict(storage=1, k=10, sweep=sw, params=dict(ghost, rerank=1)),
        "f16_learned": dict(storage=1, k=10, sweep=sw, params=dict(learned, rerank=1)),
        "e4m3_learned": dict(storage=2, k=10, sweep=sw, params=dict(learned, rerank=1)),
    }
    off = off_distribution_mask(spec, 0.2)[:gt[0].shape[0]]
    res = sweep_forms(A, ds, spec, forms, timer, gt, verbose, "w4", entries,
                      subsets={"in_distribution": ~off, "off_distribution": off})
    le.close()
    return {"workload": spec.name, "n": spec.n, "dim": spec.d, "degree": spec.degree, "nq": spec.nq,
            "off_distribution_fraction": 0.2, "gt_sample": int(gt[0].shape[0]), "learned_entry": info,
            "forms": res, "leg_s": time.time() - t0}


def serve_trace(A, srv, reqs, rng, timer, per_request, batch_search):
    """One request trace through a server: capacity with every request at
    once, latency at half that rate (Poisson arrivals), the same requests as
    one call each (per_request), and the share of sampled served results
    equal to their batch search (batch_search(q, prm) -> ids)."""
    nq = sum(len(q) for _, q, _ in reqs)

    def play(rate):
        t, trace = 0.0, []
        for rid, q, prm in reqs:
            if rate:
                t += float(rng.exponential(1.0 / rate))
            trace.append((t, rid, q, prm))
        res, wall = A.replay(srv, trace, timeout_s=300)
        lat = np.array([res[r][2] for _, r, _, _ in trace]) * 1e3
        return res, {"qps": nq / wall, "p50_ms": float(np.percentile(lat, 50)),
                     "p99_ms": float(np.percentile(lat, 99))}

    served, burst = play(0.0)
    _, half = play(0.5 * burst["qps"] / (nq / len(reqs)))
    ms = timer(per_request, steps=3, warm=1)
    same = sum(int(np.array_equal(batch_search(q, prm), served[rid][0])) for rid, q, prm in reqs[::10])
    per_req_qps = nq / (ms / 1e3)
    return {"requests": len(reqs), "queries": nq, "server_capacity_qps": burst["qps"],
            "server_all_at_once": burst, "per_request_search_qps": per_req_qps,
            "capacity_ratio_server_vs_per_request": burst["qps"] / per_req_qps,
            "half_load": dict(half, offered_qps=0.5 * burst["qps"]),
            "sampled_requests_equal_to_batch_search": f"{same}/{len(reqs[::10])}"}


def leg_workload5(A, args, timer, verbose):
    """Workload 5 (20M x 96 FP16): request traces (k in {10, 100}, itopk in
    {64, 256}) through the continuous-batching server and as one ann_search
    per request with identical parameters: the capacity of each, the
    server's latency at half its capacity, and whether each served result
    equals its batch search. Two size mixes with ghost staging: the
    recipe's batches of 1-4,096 queries, and small requests of 1-64 queries,
    where a launch per request leaves most of the GPU idle. Then the
    recipe's batches with the learned entry (MLP 96 -> 512 -> 512 ->
    200,000 trained on the GPU; the server predicts each request's ghost
    seeds as it arrives, and ghost staging judges them)."""
    import torch
    from workloads import WORKLOADS, load_dataset
    spec = WORKLOADS[5]
    t0 = time.time()
    ds = load_dataset(spec, device=timer.dev, verbose=verbose)
    ix = A.Index(ds.X, ds.G, storage=1, ghost_ids=ds.S, ghost_graph=ds.Gg, keep_fp32=True, build_dir=True,
                 device=timer.dev.index or 0)
    base = dict(entry=1, dgs_discard=0.5, rerank=1, seed=spec.seeds["search"], **W5_GHOST)

    def make_reqs(lo, hi, nreq, prm_base):
        rng = np.random.default_rng(spec.seeds["search"] + 7)
        reqs = []
        for rid in range(nreq):
            n = int(rng.integers(lo, hi))
            off = int(rng.integers(0, len(ds.Q) - n))
            k = int(rng.choice([10, 100]))
            L = max(k, int(rng.choice([64, 256])))
            reqs.append((rid, ds.Q[off:off + n], dict(prm_base, k=k, itopk=L, max_iters=L + 16,
                                                        qid_base=rid << 20)))
        return reqs, rng

    def dev_queries(reqs):
        return [torch.from_numpy(np.ascontiguousarray(q)).to(timer.dev) for _, q, _ in reqs]

    def ids_of(t):
        torch.cuda.synchronize(timer.dev)
        return t.cpu().numpy().view(np.uint32)

    srv = A.Server(ix, capacity=65536, max_requests=512,
                   max_params=dict(base, k=100, itopk=256, max_iters=272))
    A.replay(srv, [(0.0, 10**9 + i, ds.Q[:64], dict(base, k=10, itopk=64, max_iters=80, qid_base=0))
                   for i in range(4)])
    out = {}
    for mix, (lo, hi, nreq) in (("batches_1_4096", (1, 4097, args.serve_requests)),
                                ("small_1_64", (1, 65, 4 * args.serve_requests))):
        reqs, rng = make_reqs(lo, hi, nreq, base)
        dq = dev_queries(reqs)

        def per_request(reqs=reqs, dq=dq):
            # one ann_search per request, back to back on one stream (queries
            # already on the device; results stay there)
            for (rid, q, prm), qt in zip(reqs, dq):
                ix.search(qt, stream=timer.stream, **prm)

        def batch_search(q, prm):
            return ids_of(ix.search(torch.from_numpy(np.ascontiguousarray(q)).to(timer.dev), **prm)[0])

        out[mix] = serve_trace(A, srv, reqs, rng, timer, per_request, batch_search)
        if verbose:
            r = out[mix]
            print(f"[bench] serving {mix}: server {r['server_capacity_qps'] / 1e6:.3f}M/s, per request "
                  f"{r['per_request_search_qps'] / 1e6:.3f}M/s, half load p50 {r['half_load']['p50_ms']:.2f} ms "
                  f"p99 {r['half_load']['p99_ms']:.2f} ms", file=sys.stderr, flush=True)
    srv.close()
    # the learned entry: a second server that predicts each request's seeds
    le, info = train_entry(ds, spec, ix, timer.dev, verbose, args.train_queries, args.epochs,
                           judge_params=dict(ghost_max_iters_given=4, **W5_GHOST))
    lbase = dict(base, entry=2, ghost_max_iters_given=4, ghost_judge=le.judge)
    le.seeds(torch.from_numpy(np.ascontiguousarray(ds.Q[:4096])).to(timer.dev))   # size the scratch once
    srv = A.Server(ix, capacity=65536, max_requests=512, max_params=dict(lbase, k=100, itopk=256, max_iters=272),
                   mlp=le.mlp, seeds_per_query=le.P, tau=le.tau)
    A.replay(srv, [(0.0, 10**9 + i, ds.Q[:64], dict(lbase, k=10, itopk=64, max_iters=80, qid_base=0))
                   for i in range(4)])
    reqs, rng = make_reqs(1, 4097, args.serve_requests, lbase)
    dq = dev_queries(reqs)

    def per_request_learned():
        # prediction + ann_search per request, back to back on one stream
        for (rid, q, prm), qt in zip(reqs, dq):
            seeds, _ = le.seeds(qt, stream=timer.stream)
            ix.search(qt, given=seeds, stream=timer.stream, **prm)

    def batch_search_learned(q, prm):
        qt = torch.from_numpy(np.ascontiguousarray(q)).to(timer.dev)
        return ids_of(ix.search(qt, given=le.seeds(qt)[0], **prm)[0])

    out["learned_batches_1_4096"] = serve_trace(A, srv, reqs, rng, timer, per_request_learned, batch_search_learned)
    out["learned_batches_1_4096"]["learned_entry"] = info
    if verbose:
        r = out["learned_batches_1_4096"]
        print(f"[bench] serving learned: server {r['server_capacity_qps'] / 1e6:.3f}M/s, per request "
              f"{r['per_request_search_qps'] / 1e6:.3f}M/s, half load p50 {r['half_load']['p50_ms']:.2f} ms "
              f"p99 {r['half_load']['p99_ms']:.2f} ms", file=sys.stderr, flush=True)
    srv.close()
    # recall and the FP16 distance error against FP64 on a 1,000-query sample,
    # at k 10 and the mix's itopk values, stored (itopk 64) and reranked
    ns = min(args.gt_sample, len(ds.Q))
    gt = truth_knn(ds.X, ds.Q[:ns], 10, timer.dev)
    qd = torch.from_numpy(np.ascontiguousarray(ds.Q[:ns])).to(timer.dev)
    quality = {}
    for tag, rr, L in (("stored", 0, 64), ("reranked", 1, 64), ("reranked_itopk256", 1, 256)):
        ids_e, d_e, _ = ix.search(qd, **dict(base, k=10, itopk=L, max_iters=L + 16, rerank=rr))
        torch.cuda.synchronize(timer.dev)
        ie = ids_e.cpu().numpy().view(np.uint32)
        de = d_e.cpu().numpy().astype(np.float64)
        ok = ie != 0xFFFFFFFF
        ex = pair_dist(ds.X, ds.Q[:ns], np.where(ok, ie, 0).astype(np.uint32))
        rel = np.abs(de - ex)[ok] / np.maximum(ex[ok], 1e-30)
        quality[tag] = {"recall_at_10": recall_at(ie, gt[1], ds.X, ds.Q[:ns], 10),
                        "max_rel_distance_error": float(rel.max()), "mean_rel_distance_error": float(rel.mean())}
    ids_l, _, st_l = ix.search(qd, given=le.seeds(qd)[0], stats=True, **dict(lbase, k=10, itopk=64, max_iters=80))
    stn_l = A.stats_to_numpy(st_l)
    _, _, st_g = ix.search(qd, stats=True, **dict(base, k=10, itopk=64, max_iters=80))
    quality["learned_reranked"] = {"recall_at_10": recall_at(ids_of(ids_l), gt[1], ds.X, ds.Q[:ns], 10),
                                   "ghost_rows": float(stn_l["ghost_vec_rows"].mean()),
                                   "ghost_rows_ghost_staging": float(A.stats_to_numpy(st_g)["ghost_vec_rows"].mean())}
    le.close()
    ix.close()
    return {"workload": spec.name, "n": spec.n, "dim": spec.d, "degree": spec.degree, "storage": "f16",
            "entry": "ghost staging; learned entry (learned_batches_1_4096)", "mixes": out,
            "quality_k10": quality,
            "mix": "k {10,100}, itopk {64,256} raised to k, Poisson arrivals; batch sizes per mix",
            "leg_s": time.time() - t0}


def leg_wide(A, args, timer, verbose):
    """Workloads 6 and 7 (1M x 768 and 1M x 960, the shapes of the paper's
    Wiki and Gist sets): ghost staging with and without DGS, FP32 and FP16
    with rerank, each at its smallest itopk reaching recall@10 0.95."""
    from workloads import WORKLOADS, load_dataset
    out = {}
    for w in (6, 7):
        spec = WORKLOADS[w]
        t0 = time.time()
        ds = load_dataset(spec, device=timer.dev, verbose=verbose)
        gt = truth_knn(ds.X, ds.Q[:args.gt_sample], 10, timer.dev)
        gs = dict(entry=1, dgs_cooldown=0.3, ghost_max_iters=GHOST_ITERS, ghost_search_width=GHOST_WIDTH)
        sw = (16, 32, 64, 128, 256)
        forms = {
            "paper_fp32": dict(storage=0, k=10, sweep=sw, params=dict(gs, dgs_discard=0.5, rerank=0)),
            "no_dgs_fp32": dict(storage=0, k=10, sweep=sw, params=dict(gs, dgs_discard=0.0, rerank=0)),
            "f16_rerank": dict(storage=1, k=10, sweep=sw, params=dict(gs, dgs_discard=0.5, rerank=1)),
            "no_dgs_f16_rerank": dict(storage=1, k=10, sweep=sw, params=dict(gs, dgs_discard=0.0, rerank=1)),
        }
        res = sweep_forms(A, ds, spec, forms, timer, gt, verbose, f"w{w}")
        out[spec.name] = {"n": spec.n, "dim": spec.d, "degree": spec.degree, "nq": spec.nq,
                          "gt_sample": int(gt[0].shape[0]), "forms": res,
                          "dgs_speedup_fp32": res["paper_fp32"]["qps"] / res["no_dgs_fp32"]["qps"],
                          "dgs_speedup_f16": res["f16_rerank"]["qps"] / res["no_dgs_f16_rerank"]["qps"],
                          "leg_s": time.time() - t0}
        del ds
    return {"workload": "wide", "sets": out}


def leg_build(A, args, timer, verbose):
    """Build times of the index on workload 2 (1M x 96), the paper's Section
    5.7 (Fig. 16) measurement: the graph by the library's own kernels (exact
    kNN lists of 96, detour pruning to degree 64), the ghost graph the same
    way, the index (FP32 rows and the direction table, DGS's preprocessing),
    against the search it serves; and the search on the library-built graph
    at the headline setting beside the same search on the input graph."""
    import torch
    from workloads import WORKLOADS, load_dataset
    spec = WORKLOADS[2]
    ds = load_dataset(spec, device=timer.dev, verbose=verbose)
    gt = truth_knn(ds.X, ds.Q[:args.gt_sample], 10, timer.dev)
    ns = gt[0].shape[0]
    dev_i = timer.dev.index or 0

    def timed(fn):
        torch.cuda.synchronize(timer.dev)
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize(timer.dev)
        return r, time.perf_counter() - t0

    Xt = torch.from_numpy(ds.X).to(timer.dev)
    knn, t_knn = timed(lambda: A.knn_exact(Xt, spec.knn_k))
    G, t_prune = timed(lambda: A.graph_prune(knn, spec.degree))
    Xg = Xt[torch.from_numpy(ds.S.astype(np.int64)).to(timer.dev)].contiguous()
    gk, t_gknn = timed(lambda: A.knn_exact(Xg, 2 * spec.ghost_degree))
    Gg, t_gprune = timed(lambda: A.graph_prune(gk, spec.ghost_degree))
    Gh = G.cpu().numpy().view(np.uint32)
    Ggh = Gg.cpu().numpy().view(np.uint32)
    del knn, gk
    ix, t_index = timed(lambda: A.Index(ds.X, Gh, storage=0, ghost_ids=ds.S, ghost_graph=Ggh, keep_fp32=True,
                                        build_dir=True, device=dev_i))
    Qd = torch.from_numpy(ds.Q).to(timer.dev)
    p = params_for(forms_for(spec)["paper_fp32"], 32, spec.seeds["search"])
    res = {}
    ix_in = A.Index(ds.X, ds.G, storage=0, ghost_ids=ds.S, ghost_graph=ds.Gg, keep_fp32=True, build_dir=True,
                    device=dev_i)
    for name, ixx in (("library_graph", ix), ("input_graph", ix_in)):
        ids, _, _ = ixx.search(Qd, stream=timer.stream, **p)
        torch.cuda.synchronize(timer.dev)
        rec = recall_at(ids[:ns].cpu().numpy().view(np.uint32), gt[1], ds.X, ds.Q[:ns], 10)
        ms = timer(lambda ixx=ixx: ixx.search(Qd, stream=timer.stream, **p))
        res[name] = {"recall": rec, "search_ms": ms, "qps": len(ds.Q) / (ms / 1e3)}
    ix.close()
    ix_in.close()
    return {"workload": spec.name, "knn_k": spec.knn_k, "degree": spec.degree,
            "graph_build_s": {"knn_exact": t_knn, "prune": t_prune},
            "ghost_graph_build_s": {"knn_exact": t_gknn, "prune": t_gprune},
            "index_create_s": t_index,
            "note": "the library graph is exact kNN + detour pruning without the input graph's bridge edges",
            "search_at_headline_setting": res}


def leg_ppe(A, args, timer, verbose):
    """Path extension on simulated shards (Section 3.1.2) on workload 2: the
    dataset in 4 random shards, each with its graph and 1% ghost set, links
    built by search (Section 4); recall@10 against the per-shard iteration cap
    for the unsharded search, the baseline sharding (every shard from ghost
    staging) and path extension (later shards from the linked node of the
    previous result), as the paper's Fig. 12 reports it."""
    import torch
    from workloads import WORKLOADS, build_shards, load_dataset
    spec = WORKLOADS[2]
    t0 = time.time()
    ds = load_dataset(spec, device=timer.dev, verbose=verbose)
    gt = truth_knn(ds.X, ds.Q[:args.gt_sample], 10, timer.dev)
    ns = gt[0].shape[0]
    N = 4
    # each shard's ghost set has as many nodes as the whole dataset's (4% of a
    # quarter): the first stage then starts as well as the unsharded search
    sh = build_shards(ds.X, N, spec.degree, spec.knn_k, spec.graph, 0.04, spec.ghost_degree, seed=77,
                      device=timer.dev)
    dev_i = timer.dev.index or 0
    sidx = [A.Index(t.X, t.G, storage=0, ghost_ids=t.S, ghost_graph=t.Gg, keep_fp32=True, build_dir=False,
                    device=dev_i) for t in sh]
    ring = A.Shards(sidx, [t.ids for t in sh])
    link_p = dict(k=1, itopk=32, max_iters=48, entry=1, ghost_itopk=32, ghost_max_iters=12, ghost_search_width=4,
                  seed=5)
    t1 = time.time()
    ring.link(**link_p)
    link_s = time.time() - t1
    full = A.Index(ds.X, ds.G, storage=0, ghost_ids=ds.S, ghost_graph=ds.Gg, keep_fp32=True, build_dir=False,
                   device=dev_i)
    Qd = torch.from_numpy(ds.Q).to(timer.dev)
    nq = Qd.shape[0]
    p0 = dict(k=10, itopk=32, entry=1, ghost_itopk=32, ghost_max_iters=12, ghost_search_width=4,
              seed=spec.seeds["search"])
    curves = {"unsharded": [], "sharded_baseline": [], "sharded_ppe": []}
    for T in (2, 4, 6, 8, 12, 16, 24, 32, 48, 64):
        p = dict(p0, max_iters=T)
        for mode in curves:
            if mode == "unsharded":
                run = lambda p=p: full.search(Qd, stream=timer.stream, **p)   # noqa: E731
            else:
                fwd = 1 if mode == "sharded_ppe" else 0
                run = lambda p=p, fwd=fwd: ring.search(Qd, n_forward=fwd, stream=timer.stream, **p)   # noqa: E731
            if mode == "unsharded":
                ids, _, st = full.search(Qd, stream=timer.stream, stats=True, **p)
            else:
                ids, _, st = ring.search(Qd, n_forward=1 if mode == "sharded_ppe" else 0, stats=True,
                                         stream=timer.stream, **p)
            torch.cuda.synchronize(timer.dev)
            stn = A.stats_to_numpy(st.reshape(-1, st.shape[-1]))
            # iterations per query summed over its stages: base and ghost
            it_q = (stn["iters"].astype(np.int64) + stn["ghost_iters"]).reshape(-1, nq).sum(axis=0)
            rec = recall_at(ids[:ns].cpu().numpy().view(np.uint32), gt[1], ds.X, ds.Q[:ns], 10)
            ms = timer(run)
            curves[mode].append({"max_iters": T, "recall": rec, "qps": nq / (ms / 1e3),
                                 "iters_per_query": float(it_q.mean()),
                                 "rows_per_query": float((stn["vec_rows"].astype(np.int64) + stn["ghost_vec_rows"])
                                                         .reshape(-1, nq).sum(axis=0).mean())})
    reach = {m: next((c["max_iters"] for c in v if c["recall"] >= 0.90), None) for m, v in curves.items()}
    reach_it = {m: next((c["iters_per_query"] for c in v if c["recall"] >= 0.90), None) for m, v in curves.items()}
    ring.close()
    for ix in sidx:
        ix.close()
    full.close()
    if verbose:
        print(f"[bench] ppe: iterations to recall 0.90 {reach}", file=sys.stderr, flush=True)
    return {"workload": spec.name, "shards": N, "shard_n": [int(len(t.ids)) for t in sh], "forwarded": 1,
            "link_params": link_p, "link_build_s": link_s, "search": {k: v for k, v in p0.items() if k != "seed"},
            "iters_to_recall_0.90": reach, "total_iters_per_query_at_recall_0.90": reach_it, "curves": curves,
            "leg_s": time.time() - t0}


# ------------------------------------------------------------------ our arm
LEG_FNS = {"3": leg_workload3, "4": leg_workload4, "5": leg_workload5, "wide": leg_wide, "ppe": leg_ppe,
           "build": leg_build}
LEG_KEYS = {"3": "precision-10M-128d-int", "4": "learned-5M-256d-zipf", "5": "serving-20M-96d",
            "wide": "wide_vectors", "ppe": "path_extension", "build": "index_build"}
DEFAULT_LEGS = "3,4,5,wide,ppe,build"
FINAL_RESERVE_S = 30.0   # kept back for the JSON line after the last leg
MIN_LEG_S = 60.0         # a leg is not started with less than this left


def run_leg_child(w: str, args, device: int, verbose: bool) -> dict:
    """Run one side leg as `bench.py --leg w` in a child process (its own
    CUDA context, its own process group) with a deadline of what is left of
    --budget-s. A leg that would start too late is skipped, one that runs
    past the deadline is ended; either is recorded in its place."""
    left = args.budget_s - (time.time() - T_START) - FINAL_RESERVE_S
    if left < MIN_LEG_S:
        return {"skipped": f"wall budget: {max(left, 0.0):.0f} s left of --budget-s {args.budget_s:.0f}"}
    cmd = [sys.executable, os.path.abspath(__file__), "--leg", w, "--leg-device", str(device),
           "--steps", str(args.steps), "--warmup", str(args.warmup), "--gt-sample", str(args.gt_sample),
           "--train-queries", str(args.train_queries), "--epochs", str(args.epochs),
           "--serve-requests", str(args.serve_requests)] + (["-v"] if verbose else [])
    env = {k: v for k, v in os.environ.items()
           if k not in ("RANK", "LOCAL_RANK", "WORLD_SIZE", "LOCAL_WORLD_SIZE", "GROUP_RANK", "ROLE_RANK",
                        "TORCHELASTIC_RUN_ID")}
    t0 = time.time()
    proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=None, text=True, env=env, cwd=ROOT,
                            start_new_session=True)
    try:
        out, _ = proc.communicate(timeout=left)
    except subprocess.TimeoutExpired:
        os.killpg(proc.pid, 9)
        proc.communicate()
        return {"skipped": f"ended at the wall budget after {time.time() - t0:.0f} s "
                           f"(--budget-s {args.budget_s:.0f})"}
    if verbose:
        print(f"[bench] leg {w} done in {time.time() - t0:.0f}s (rc {proc.returncode})", file=sys.stderr,
              flush=True)
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    if proc.returncode != 0 or not lines:
        return {"failed": f"child exited {proc.returncode}", "stdout_tail": out[-500:]}
    return json.loads(lines[-1])


def run_leg(args):
    """Child side of run_leg_child: one leg on one GPU, its result as one
    JSON line on stdout."""
    import torch
    import paper_2507_17094_gb300 as A
    torch.cuda.set_device(args.leg_device)
    dev = torch.device("cuda", args.leg_device)
    A.build()
    timer = Timer(dev, torch.cuda.current_stream(dev))
    res = LEG_FNS[args.leg](A, args, timer, args.verbose)
    torch.cuda.synchronize(dev)
    print(json.dumps(res), flush=True)


def run_ours(args):
    import torch
    import paper_2507_17094_gb300 as A
    from workloads import WORKLOADS, load_dataset

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    dev = torch.device("cuda", local)
    spec = WORKLOADS[args.workload]
    if args.nq:
        import dataclasses
        spec = dataclasses.replace(spec, nq=args.nq)
    verbose = rank == 0 and args.verbose
    A.build()
    ds = load_dataset(spec, device=dev, verbose=verbose)
    forms = forms_for(spec)
    headline = "paper_fp32"
    if args.forms and headline not in args.forms.split(","):
        headline = args.forms.split(",")[0]
    seed = spec.seeds["search"]

    gt_sample = min(args.gt_sample, spec.nq)
    cpu = None
    gt_ids = gt_d = None
    if rank == 0:
        # ground truth first: the recall sweep needs it
        t0 = time.time()
        gt_ids, gt_d = truth_knn(ds.X, ds.Q[:gt_sample], 10, dev)
        if verbose:
            print(f"[bench] FP64 ground truth ({gt_sample} queries) in {time.time() - t0:.1f}s",
                  file=sys.stderr, flush=True)

    indexes = {}

    def index_for(storage):
        if storage not in indexes:
            indexes[storage] = A.Index(ds.X, ds.G, storage=storage, ghost_ids=ds.S, ghost_graph=ds.Gg,
                                       keep_fp32=True, build_dir=True, device=local)
        return indexes[storage]

    Qd = torch.from_numpy(ds.Q).to(dev)
    nq = Qd.shape[0]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2

    def timed_steps(run, params, steps, warm):
        for _ in range(warm):
            run(params)
        torch.cuda.synchronize(dev)
        times = []
        for _ in range(steps):
            flush.add_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run(params)
            e1.record(stream)
            times.append((e0, e1))
        torch.cuda.synchronize(dev)
        return [a.elapsed_time(b) for a, b in times]

    out = (torch.empty((nq, 10), dtype=torch.int32, device=dev), torch.empty((nq, 10), device=dev))
    results = {}
    entries = {}

    def stepper(ix, name, form):
        """One step of a form: the search, preceded for learned forms by the
        fused MLP prediction of this batch's ghost seeds."""
        if form["entry"] != 2:
            return lambda p, out=out, stats=False: ix.search(Qd, stream=stream, out=out, stats=stats, **p)
        le = entries[form["storage"]]

        def run(p, out=out, stats=False):
            seeds, _ = le.seeds(Qd, stream=stream)
            return ix.search(Qd, given=seeds, stream=stream, out=out, stats=stats, **p)
        return run

    for name in selected_forms(forms, args.forms):
        form = forms[name]
        ix = index_for(form["storage"])
        if form["entry"] == 2 and form["storage"] not in entries:
            entries[form["storage"]], info = train_entry(ds, spec, ix, dev, verbose, args.train_queries,
                                                         args.epochs)
            results.setdefault("_learned_entry", {})[form["storage"]] = info
        run = stepper(ix, name, form)
        sweep = []
        chosen = None
        for L in SWEEP:
            p = params_for(form, L, seed)
            ids, dists, _ = run(p)
            ms = statistics.median(timed_steps(run, p, 3, 1))
            rec = None
            if rank == 0:
                a_ids = ids[:gt_sample].cpu().numpy().view(np.uint32)
                rec = recall_at(a_ids, gt_d, ds.X, ds.Q[:gt_sample], 10)
            rec = float(max_over_ranks(rec if rec is not None else 0.0, dist, dev))
            sweep.append({"itopk": L, "recall": rec, "ms": ms, "qps": nq / (ms / 1e3)})
            if chosen is None and rec >= RECALL_TARGET:
                chosen = L
        if chosen is None:
            chosen = max(sweep, key=lambda s: s["recall"])["itopk"]
        results[name] = {"storage": {0: "f32", 1: "f16", 2: "e4m3"}[form["storage"]],
                         "entry": {0: "random", 1: "ghost", 2: "learned"}[form["entry"]],
                         "dgs_discard": form["dgs_discard"], "dgs_min_match": form.get("dgs_min_match", 0.0),
                         "rerank": bool(form["rerank"]),
                         "itopk": chosen, "sweep": sweep}
        if verbose:
            print(f"[bench] {name}: " + ", ".join(f"L{s['itopk']} r={s['recall']:.3f} "
                                                   f"{s['qps'] / 1e6:.2f}M/s" for s in sweep),
                  file=sys.stderr, flush=True)

    # ---------------------------------------------------- the timed region
    form = forms[headline]
    ix = index_for(form["storage"])
    head_run = stepper(ix, headline, form)
    L = results[headline]["itopk"]
    p = params_for(form, L, seed)
    ids, dists, st = head_run(p, out=None, stats=True)
    torch.cuda.synchronize(dev)
    ix.sync()
    st_np = A.stats_to_numpy(st)
    bytes_per_launch = float(algorithmic_bytes(st_np, spec, form["storage"], bool(form["rerank"])).sum())
    head_recall = next(s["recall"] for s in results[headline]["sweep"] if s["itopk"] == L)

    # per-phase split of the headline search (a separate profiling build of
    # the kernel, run once outside the timed region; Section 5.5's method)
    phase_profile = None
    if form["entry"] != 2:
        _, _, cyc = ix.search_profile(Qd, stream=stream, **p)
        tot = float(cyc.sum())
        phase_profile = {"kernel": "search_kernel profiling build (same results)", "total_warp_cycles": tot,
                         "share": {f"{sn}/{pn}": float(cyc[i, j]) / tot
                                   for i, sn in enumerate(A.PROFILE_STAGE_NAMES)
                                   for j, pn in enumerate(A.PROFILE_PHASE_NAMES) if cyc[i, j] > 0}}
    for _ in range(args.warmup):
        head_run(p)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.start()
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    step_ms = timed_steps(head_run, p, args.steps, 0)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    total_queries = sum_over_ranks(float(nq * args.steps), dist, dev)
    value = total_queries / (total_ms / 1e3)
    ms_per_step = total_ms / args.steps
    mean_launch_s = statistics.mean(step_ms) / 1e3
    ix.sync()

    # other forms at their chosen itopk (a few steps each, reported beside)
    for name, r in results.items():
        if name.startswith("_"):
            continue
        f = forms[name]
        ixf = index_for(f["storage"])
        runf = stepper(ixf, name, f)
        pf = params_for(f, r["itopk"], seed)
        _, _, stf = runf(pf, out=None, stats=True)
        torch.cuda.synchronize(dev)
        stn = A.stats_to_numpy(stf)
        ms = statistics.median(timed_steps(runf, pf, max(5, args.steps // 10), 2))
        b = float(algorithmic_bytes(stn, spec, f["storage"], bool(f["rerank"])).sum())
        r.update(qps=nq / (ms / 1e3), ms_per_step=ms, recall=next(s["recall"] for s in r["sweep"]
                                                                   if s["itopk"] == r["itopk"]),
                 gbs=b / (ms / 1e3) / 1e9, hbm_frac=(b / (ms / 1e3) / 1e9) / measured_peaks()["hbm_gbs"],
                 mean_vec_rows=float(stn["vec_rows"].mean()), mean_iters=float(stn["iters"].mean()),
                 mean_ghost_rows=float(stn["ghost_vec_rows"].mean()),
                 mean_ghost_iters=float(stn["ghost_iters"].mean()),
                 hash_resets=int(stn["hash_resets"].sum()))
        if f["storage"] != 0 and rank == 0:
            # distance error against FP64 on the recall sample, for the
            # stored-precision distances (rerank off) and the returned ones
            errs = {}
            for tag, rr in (("stored", 0), ("reranked", 1)):
                ids_e, d_e, _ = runf(dict(pf, rerank=rr))
                torch.cuda.synchronize(dev)
                ie = ids_e[:gt_sample].cpu().numpy().view(np.uint32)
                de = d_e[:gt_sample].cpu().numpy().astype(np.float64)
                ok = ie != 0xFFFFFFFF
                ex = pair_dist(ds.X, ds.Q[:gt_sample], np.where(ok, ie, 0).astype(np.uint32))
                rel = np.abs(de - ex)[ok] / np.maximum(ex[ok], 1e-30)
                errs[tag] = {"max_rel": float(rel.max()), "mean_rel": float(rel.mean())}
            r["distance_error_vs_fp64"] = errs
        if f["entry"] == 2:
            # the entry network's fused predict alone: tensor-core roofline
            le = entries[f["storage"]]
            pred = timed_steps(lambda _p: le.seeds(Qd, stream=stream), None, max(5, args.steps // 10), 2)
            pred_ms = statistics.median(pred)
            flop = 2.0 * nq * (spec.d * 512 + 512 * 512 + 512 * spec.ghost_n)
            tf = flop / (pred_ms / 1e3) / 1e12
            r["predict"] = {"ms": pred_ms, "kernel": "gemm_kernel<EPI_TOPP> + hidden layers + topp_merge",
                            "roofline": {"bound": "tensor", "achieved": tf, "peak": measured_peaks()["bf16_tflops"],
                                         "unit": "TFLOP/s", "frac": tf / measured_peaks()["bf16_tflops"],
                                         "flop_per_step": flop}}
        del r["sweep"]

    # ------------------------------------------------------------ serving (continuous batching)
    serving = None
    if rank == 0 and not args.no_serving:
        serving = serve_leg(A, index_for(1), entries.get(1), ds, spec, args)
        if verbose:
            print(f"[bench] serving: {serving}", file=sys.stderr, flush=True)

    # ------------------------------------------------------------ e2e (host buffers)
    # every step copies the queries in from pinned host memory and the
    # results out: through ann_search_host for the plain forms; for learned
    # forms the queries go to the device, the MLP picks the seeds there and
    # the search reads them, and the results come back
    Qpin = torch.from_numpy(ds.Q).pin_memory()
    Qh = Qpin.numpy()
    e2e_steps = max(3, min(args.steps, 50))
    if form["entry"] == 2:
        le = entries[form["storage"]]
        res_ids = torch.empty((nq, 10), dtype=torch.int32).pin_memory()
        res_d = torch.empty((nq, 10), dtype=torch.float32).pin_memory()

        def e2e_step():
            Qd.copy_(Qpin, non_blocking=True)
            seeds, _ = le.seeds(Qd, stream=stream)
            i_, d_, _ = ix.search(Qd, given=seeds, stream=stream, out=out, **p)
            res_ids.copy_(i_, non_blocking=True)
            res_d.copy_(d_, non_blocking=True)
            torch.cuda.synchronize(dev)
        e2e_api = "LearnedEntry.seeds + Index.search (ann_mlp_predict + ann_search), pinned host copies"
    else:
        def e2e_step():
            ix.search_host(Qh, **p)
        e2e_api = "ann_search_host (pinned host buffers)"
    e2e_step()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
    e2e_value = sum_over_ranks(float(nq * e2e_steps), dist, dev) / e2e_s

    # ------------------------------------------------------------ CPU baseline (rank 0, N = 1 only)
    cpu_baseline = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle as O   # the CPU oracle, as it stands, timed on the host cores
        sample = min(args.cpu_sample, spec.nq)
        oi = O.OracleIndex(ds.X, ds.G, form["storage"], ds.S, ds.Gg)
        cores = O.default_threads()
        reps, done, t0 = 0, 0, time.perf_counter()
        while True:   # repeat the sample until about a second of wall time (~cores core-seconds)
            o_ids, o_d, o_c = O.search(oi, ds.Q[:sample], threads=cores, **p)
            reps += 1
            done += sample
            if time.perf_counter() - t0 >= 1.0 or reps >= 50:
                break
        dt = time.perf_counter() - t0
        g_ids = ids[:sample].cpu().numpy().view(np.uint32)
        match = float((g_ids == o_ids).mean())
        cpu_baseline = {"value": done / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                        "sample": f"the first {sample} of the {spec.nq} queries x {reps} passes, same search "
                                  f"parameters (itopk {L}), plain-C oracle on all host cores, {dt:.2f} s wall",
                        "ids_match_gpu": match}

    # ------------------------------------------------------------ workloads 3-5 and path extension
    # each leg runs in a child process with what is left of the wall budget,
    # so the line below is printed in bounded time whatever the legs cost
    legs = {}
    if rank == 0 and world == 1 and args.workloads:
        for le_ in entries.values():
            le_.close()
        entries.clear()
        for ix_ in indexes.values():
            ix_.close()
        indexes.clear()
        torch.cuda.synchronize(dev)
        torch.cuda.empty_cache()
        for w in args.workloads.split(","):
            if w in LEG_FNS:
                legs[w] = run_leg_child(w, args, local, verbose)

    peaks = measured_peaks()
    achieved = bytes_per_launch / mean_launch_s / 1e9
    tr = ncu_traffic(spec.name, headline)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "peak_source": peaks["source"],
                "traffic": tr["dram_bytes_per_launch"] if tr else None,
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "kernel": f"search_kernel<{('F32', 'F16', 'E4M3')[form['storage']]}>"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded Gaussian mixture; no dataset files)",
        "config": {"workload": spec.name, "n": spec.n, "dim": spec.d, "degree": spec.degree, "nq": nq,
                   "form": headline, "k": 10, "itopk": L, "search_width": 1, "max_iters": p["max_iters"],
                   "entry": ("random", "ghost", "learned")[form["entry"]], "ghost_n": spec.ghost_n,
                   "ghost_max_iters": form["ghost_max_iters"], "ghost_search_width": form["ghost_search_width"],
                   "dgs_discard": form["dgs_discard"], "dgs_cooldown": form["dgs_cooldown"],
                   "storage": ("f32", "f16", "e4m3")[form["storage"]],
                   "recall_at_10": head_recall, "recall_target": RECALL_TARGET,
                   "l2": "flushed between steps (256 MB write outside the timed events)",
                   "parallelism": f"replicas x{world}"},
        "forms": results,
        "roofline": roofline,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(nq * spec.d * 4),
                "d2h_bytes_per_step": int(nq * 10 * 8), "steps": e2e_steps,
                "api": e2e_api},
        "gpu_launches": args.steps,
        "cpu_baseline": cpu_baseline,
        "serving": serving,
        "phase_profile": phase_profile,
        "workloads": {LEG_KEYS[w]: legs[w] for w in legs},
        "wall_s": time.time() - T_START, "budget_s": args.budget_s,
    }
    for le in entries.values():
        le.close()
    for ix_ in indexes.values():
        ix_.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle as O
    from workloads import WORKLOADS, load_dataset
    spec = WORKLOADS[args.workload]
    if args.nq:
        import dataclasses
        spec = dataclasses.replace(spec, nq=args.nq)
    dev = None
    try:
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
    except ImportError:
        pass
    ds = load_dataset(spec, device=dev, verbose=args.verbose)   # input generation only
    form = forms_for(spec)["paper_fp32"]
    seed = spec.seeds["search"]
    sample = min(args.cpu_sample, spec.nq)
    gt_sample = min(args.gt_sample, sample)
    gt_ids, gt_d = O.knn_f64(ds.X, ds.Q[:gt_sample], 10)
    oi = O.OracleIndex(ds.X, ds.G, form["storage"], ds.S, ds.Gg)
    cores = O.default_threads()
    chosen, rec_at = None, None
    for L in SWEEP:
        p = params_for(form, L, seed)
        ids, _, _ = O.search(oi, ds.Q[:gt_sample], threads=cores, **p)
        rec = O.recall_at_k(ids, gt_ids, gt_d, ds.X, ds.Q[:gt_sample], 10)[0]
        if rec >= RECALL_TARGET:
            chosen, rec_at = L, rec
            break
    if chosen is None:
        chosen, rec_at = SWEEP[-1], rec
    p = params_for(form, chosen, seed)
    Qs = ds.Q[:sample]
    for _ in range(args.warmup):
        O.search(oi, Qs, threads=cores, **p)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.search(oi, Qs, threads=cores, **p)
    dt = time.perf_counter() - t0
    value = sample * args.steps / dt
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "reference",
            "config": {"workload": spec.name, "n": spec.n, "dim": spec.d, "degree": spec.degree,
                       "nq": sample, "form": "paper_fp32", "k": 10, "itopk": chosen, "search_width": 1,
                       "max_iters": p["max_iters"], "entry": "ghost", "ghost_n": spec.ghost_n,
                       "ghost_max_iters": form["ghost_max_iters"], "ghost_search_width": form["ghost_search_width"],
                       "dgs_discard": form["dgs_discard"], "dgs_cooldown": form["dgs_cooldown"], "storage": "f32",
                       "recall_at_10": rec_at},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{sample} queries per step of the {spec.nq}-query workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_predict_shapes(args):
    """The learned entry's prediction alone (hidden layers, fused top-8
    logits, merge) on 10,000 queries for workload 2's network (96 -> 512 ->
    512 -> 10,000) and workload 4's (256 -> 512 -> 512 -> 50,000), random
    initial weights, CUDA-event timed; one JSON line. Used to profile the
    GEMM kernels (ncu on this command)."""
    import torch
    import paper_2507_17094_gb300 as A
    from workloads import init_mlp_params
    A.build()
    out = {}
    for d, n_out in ((96, 10_000), (256, 50_000)):
        m = A.MLP(d, 512, 512, n_out, 16384)
        m.set_params(*init_mlp_params(d, 512, 512, n_out, 1))
        X = torch.randn(10_000, d, device="cuda", generator=torch.Generator("cuda").manual_seed(d))
        for _ in range(args.warmup):
            m.predict(X, P=8)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            m.predict(X, P=8)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        flop = 2.0 * 10_000 * (d * 512 + 512 * 512 + 512 * n_out)
        out[f"{d}->512->512->{n_out}"] = {"ms": ms, "tflops": flop / ms / 1e9,
                                          "frac_of_bf16_peak": flop / ms / 1e9 / measured_peaks()["bf16_tflops"]}
        m.sync()
        m.close()
    print(json.dumps({"predict_shapes": out, "queries": 10_000, "steps": args.steps, "warmup": args.warmup}),
          flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", type=int, default=2)
    ap.add_argument("--nq", type=int, default=0)
    ap.add_argument("--forms", default="")
    ap.add_argument("--gt-sample", type=int, default=1000)
    ap.add_argument("--cpu-sample", type=int, default=10000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--train-queries", type=int, default=200_000)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=120)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--workloads", default=DEFAULT_LEGS,
                    help="legs beside the headline (rank 0, one GPU): 3, 4, 5, wide, ppe and build; empty for none")
    ap.add_argument("--budget-s", type=float, default=1020.0,
                    help="wall-clock budget of the whole run; the side legs get what the headline leaves")
    ap.add_argument("--leg", default="", help=argparse.SUPPRESS)
    ap.add_argument("--leg-device", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--predict-shapes", action="store_true",
                    help="time only the learned entry's prediction on two network shapes (GEMM profiling)")
    ap.add_argument("-v", "--verbose", action="store_true")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.leg:
        run_leg(args)
    elif args.predict_shapes:
        run_predict_shapes(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
