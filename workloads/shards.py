"""Shards for pipelining-based path extension (an input of the method).

The paper partitions the dataset at random into one shard per GPU and builds
an independent graph per shard (Section 3.1.2). On one GPU the shards are
simulated: each is its own index in the same device memory. This module makes
the partition and each shard's graph and ghost sample; it computes nothing of
the search or of the inter-shard links (those are the method's: the CUDA
library and the CPU oracle each build them on their own).
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np

from .graph import build_graph, ghost_sample


@dataclass
class Shard:
    ids: np.ndarray        # global ids of the shard's points, ascending (uint32)
    X: np.ndarray          # n_i x d float32, row j = global point ids[j]
    G: np.ndarray          # n_i x degree uint32 over local indices
    S: np.ndarray          # ghost sample, local indices ascending (uint32)
    Gg: np.ndarray         # ghost graph over ghost indices


def shard_split(n: int, n_shards: int, seed: int) -> List[np.ndarray]:
    """A seeded random partition of 0..n-1 into n_shards parts of sizes
    differing by at most one; each part's ids ascending (uint32)."""
    if not 1 <= n_shards <= n:
        raise ValueError("need 1 <= n_shards <= n")
    perm = np.random.Generator(np.random.PCG64(seed)).permutation(n)
    return [np.sort(p).astype(np.uint32) for p in np.array_split(perm, n_shards)]


def build_shards(X: np.ndarray, n_shards: int, degree: int, knn_k: int, method: str, ghost_ratio: float,
                 ghost_degree: int, seed: int, device=None, n_bridge: int = -1) -> List[Shard]:
    """Partition X and build, per shard, the graph (same builder as the whole
    dataset's) and a ghost sample of ghost_ratio of its points with its own
    exact-kNN graph."""
    out = []
    for i, ids in enumerate(shard_split(X.shape[0], n_shards, seed)):
        Xi = np.ascontiguousarray(X[ids])
        G = build_graph(Xi, degree, knn_k, method, device=device, seed=seed + 101 * i, n_bridge=n_bridge)
        ng = max(ghost_degree + 1, int(round(ghost_ratio * len(ids))))
        S = ghost_sample(len(ids), ng, seed + 7 + i)
        Gg = build_graph(Xi[S], ghost_degree, 2 * ghost_degree, "exact", device=device, seed=seed + 13 + i,
                         n_bridge=0)
        out.append(Shard(ids, Xi, G, S, Gg))
    return out
