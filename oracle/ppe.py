"""Oracle for pipelining-based path extension (PPE) on simulated shards.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use it; the CUDA library never imports it.

The paper (Section 3.1.2) partitions the dataset into N shards with
independent graphs and links every node u of shard i to its nearest node in
shard (i + 1) mod N (Eq. 3, the inter-shard map I). Queries are split into N
chunks; chunk c starts on shard c and, after each shard's search converges,
continues on the next shard of the ring from I(z) for the nodes z of the
local result it forwards, until it has visited every shard; the N local
top-k lists are then reduced to the final top-k (on the CPU in the paper).
The implementation section (Section 4) builds I by searching shard i + 1 with
each node of shard i as the query and keeping the top-1 result, and forwards
one node per query. With no forwarding every stage starts from the entry
the parameters give (random or ghost staging): the paper's baseline sharding.

Everything here calls the plain search of ``oracle.search`` per stage; the
only arithmetic of its own is the reduction, a sort by (distance, global id).
"""

from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np

from . import INVALID, OracleIndex, knn_f64, search


def chunk_bounds(nq: int, n_shards: int) -> List[tuple]:
    """Query chunk c is rows [floor(c nq / N), floor((c + 1) nq / N))."""
    return [(c * nq // n_shards, (c + 1) * nq // n_shards) for c in range(n_shards)]


def link_exact(X_from: np.ndarray, X_next: np.ndarray) -> np.ndarray:
    """Eq. 3 as written: I(u) = argmin over the next shard's nodes w of
    dist(u, w), in FP64, ties to the smaller local index (uint32)."""
    ids, _ = knn_f64(X_next, X_from, 1)
    return ids[:, 0].copy()


def link_by_search(next_index: OracleIndex, X_from: np.ndarray, **params) -> np.ndarray:
    """Section 4's construction of I: every node u of shard i is a query of a
    search on shard i + 1; its top-1 result is I(u) (local index in shard
    i + 1, uint32). The query stream of node u is its local index."""
    p = dict(params, k=1)
    ids, _, _ = search(next_index, np.ascontiguousarray(X_from, dtype=np.float32), **p)
    return ids[:, 0].copy()


def ppe_search(shards: Sequence[OracleIndex], global_ids: Sequence[np.ndarray],
               links: Optional[Sequence[np.ndarray]], Q: np.ndarray, n_forward: int = 1,
               threads: Optional[int] = None, **params):
    """The sharded search. shards[s] holds shard s (local node indices),
    global_ids[s] maps them to dataset ids, links[s] is I from shard s to
    shard (s + 1) mod N (None with n_forward = 0). n_forward nodes of each
    local result (its best ones) are forwarded; 0 is the baseline sharding.
    A query's random-seed stream is its row in Q (plus params' qid_base) on
    every shard. Returns (global ids uint32 nq x k, dists float32 nq x k,
    per-stage counters: an N x nq record array, row t = the stage-t
    searches)."""
    N = len(shards)
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    nq = Q.shape[0]
    k = params.get("k", 10)
    if n_forward and (links is None or not 1 <= n_forward <= k):
        raise ValueError("forwarding needs the links and 1 <= n_forward <= k")
    base_qid = params.pop("qid_base", 0)
    loc_ids = np.full((N, nq, k), INVALID, dtype=np.uint32)   # stage t, local ids in shard (c + t) mod N
    loc_d = np.full((N, nq, k), np.inf, dtype=np.float32)
    cnt = None
    for c, (lo, hi) in enumerate(chunk_bounds(nq, N)):
        if hi == lo:
            continue
        for t in range(N):
            s = (c + t) % N
            p = dict(params, qid_base=base_qid + lo)
            given = None
            if t > 0 and n_forward:
                prev = (s - 1) % N
                z = loc_ids[t - 1, lo:hi, :n_forward]
                given = np.where(z == INVALID, INVALID, links[prev][np.where(z == INVALID, 0, z)]).astype(np.uint32)
                p["entry"] = 3
            ids, d, ct = search(shards[s], Q[lo:hi], given_seeds=given, threads=threads, **p)
            loc_ids[t, lo:hi] = ids
            loc_d[t, lo:hi] = d
            if cnt is None:
                cnt = np.zeros((N, nq), dtype=ct.dtype)
            cnt[t, lo:hi] = ct
    # reduction: the N local lists, as dataset ids, by (distance, id)
    gid = np.full((nq, N * k), INVALID, dtype=np.uint32)
    gd = np.full((nq, N * k), np.inf, dtype=np.float32)
    for c, (lo, hi) in enumerate(chunk_bounds(nq, N)):
        for t in range(N):
            s = (c + t) % N
            li = loc_ids[t, lo:hi]
            ok = li != INVALID
            gid[lo:hi, t * k:(t + 1) * k] = np.where(ok, global_ids[s][np.where(ok, li, 0)], INVALID)
            gd[lo:hi, t * k:(t + 1) * k] = loc_d[t, lo:hi]
    order = np.lexsort((gid, gd), axis=1)[:, :k]
    out_ids = np.take_along_axis(gid, order, axis=1)
    out_d = np.take_along_axis(gd, order, axis=1)
    return out_ids, out_d, cnt
