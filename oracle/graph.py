"""Oracle for the graph builder (test infrastructure only).

The paper takes the proximity graph as given and builds it with CAGRA's
builder (Section 2.1, Section 5.1); its build-time study (Section 5.7, Fig.
16) times the graph next to the method's own preprocessing. The builder here
follows one written recipe, and this module states it in plain loops over
small inputs, sharing no code with the CUDA builder or with the input
tooling under workloads/:

1. kNN lists: for every node u, the K nodes nearest to u other than u, in
   FP64, ordered by (distance, id);
2. detour count: edge u -> v at rank r of u's list is detoured via the node
   w at rank a < r of u's list when v appears in w's own list at a rank
   c < r; det(r) counts such (a, c) pairs;
3. order u's list by (det, rank) and keep the first half = degree // 2
   edges (the least detoured);
4. reverse edges: every kept edge w -> v (at position p of w's kept list)
   offers w to v; v takes the offers ordered by (p, w), at most
   degree - half of them;
5. v's row: its kept edges, then its reverse edges, then the rest of its
   ordered list, with repeats (first occurrence kept) and v itself dropped,
   cut to `degree` (padded with INVALID if fewer remain).
"""

from __future__ import annotations

import numpy as np

from . import INVALID, knn_f64


def knn_lists(X: np.ndarray, K: int) -> np.ndarray:
    """Step 1: exact kNN of every node among the others, FP64, ties to the
    smaller id (uint32 n x K)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    n = X.shape[0]
    ids, _ = knn_f64(X, X, min(K + 1, n))
    out = np.empty((n, K), dtype=np.uint32)
    for u in range(n):
        row = [int(v) for v in ids[u] if int(v) != u][:K]
        out[u] = row + [INVALID] * (K - len(row))
    return out


def detour_counts(knn: np.ndarray) -> np.ndarray:
    """Step 2 for every node (int64 n x K): det[u, r] = #{(a, c): a < r,
    c < r, knn[knn[u, a], c] == knn[u, r]}."""
    n, K = knn.shape
    det = np.zeros((n, K), dtype=np.int64)
    for u in range(n):
        rank = {}
        for r, v in enumerate(knn[u].tolist()):
            rank.setdefault(v, r)
        for a in range(K):
            w = int(knn[u, a])
            if w == INVALID:
                continue
            for c in range(K):
                x = int(knn[w, c])
                r = rank.get(x)
                if r is not None and a < r and c < r:
                    det[u, r] += 1
    return det


def prune(knn: np.ndarray, degree: int) -> np.ndarray:
    """Steps 2-5: the pruned graph (uint32 n x degree)."""
    knn = np.ascontiguousarray(knn, dtype=np.uint32)
    n, K = knn.shape
    half = degree // 2
    det = detour_counts(knn)
    ordered = np.empty_like(knn)
    for u in range(n):
        order = sorted(range(K), key=lambda r: (int(det[u, r]), r))
        ordered[u] = knn[u, order]
    offers = [[] for _ in range(n)]
    for w in range(n):
        for p in range(half):
            v = int(ordered[w, p])
            if v != INVALID:
                offers[v].append((p, w))
    out = np.full((n, degree), INVALID, dtype=np.uint32)
    for v in range(n):
        rev = [w for _, w in sorted(offers[v])][:degree - half]
        row, seen = [], set()
        for x in list(ordered[v, :half].tolist()) + rev + list(ordered[v, half:].tolist()):
            if x == INVALID or x == v or x in seen:
                continue
            seen.add(x)
            row.append(x)
            if len(row) == degree:
                break
        out[v, :len(row)] = row
    return out
