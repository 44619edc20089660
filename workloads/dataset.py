"""A complete seeded workload (base vectors, queries, graph, ghost sample and
ghost graph), built once and cached on disk by recipe.

The cache directory is ``$ANN_CACHE_DIR`` or ``~/.cache/paper_2507_17094_gb300``.
"""

from __future__ import annotations

import hashlib
import sys
import json
import os
import time
from dataclasses import asdict, dataclass
from typing import Optional

import numpy as np

from .graph import build_graph, ghost_sample
from .mixtures import WorkloadSpec, make_queries


def cache_dir() -> str:
    d = os.environ.get("ANN_CACHE_DIR") or os.path.join(os.path.expanduser("~"), ".cache",
                                                          "paper_2507_17094_gb300")
    os.makedirs(d, exist_ok=True)
    return d


@dataclass
class Dataset:
    spec: WorkloadSpec
    X: np.ndarray          # n x d float32
    Q: np.ndarray          # nq x d float32
    G: np.ndarray          # n x degree uint32
    S: np.ndarray          # ghost ids, ascending uint32
    Gg: np.ndarray         # n_ghost x ghost_degree uint32
    build_s: float = 0.0


def _key(spec: WorkloadSpec, off_fraction: float) -> str:
    blob = json.dumps({"spec": asdict(spec), "off": off_fraction, "v": 5}, sort_keys=True, default=str)
    return f"{spec.name}-{hashlib.sha256(blob.encode()).hexdigest()[:16]}"


def load_dataset(spec: WorkloadSpec, off_fraction: float = 0.0, device=None, use_cache: bool = True,
                 verbose: bool = False) -> Dataset:
    key = _key(spec, off_fraction)
    path = os.path.join(cache_dir(), key)
    names = ("X", "Q", "G", "S", "Gg")
    if use_cache and all(os.path.exists(os.path.join(path, n + ".npy")) for n in names):
        arrs = {n: np.load(os.path.join(path, n + ".npy"), mmap_mode=None) for n in names}
        return Dataset(spec, **arrs)
    t0 = time.time()
    X, _ = spec.mixture().sample(spec.n, spec.seeds["base"])
    Q = make_queries(spec, off_fraction=off_fraction)
    if verbose:
        print(f"[dataset] {spec.name}: vectors in {time.time() - t0:.1f}s", file=sys.stderr, flush=True)
    G = build_graph(X, spec.degree, spec.knn_k, spec.graph, device=device, seed=spec.seeds["base"],
                    n_near=spec.n_near, part_size=spec.part_size)
    if verbose:
        print(f"[dataset] {spec.name}: graph in {time.time() - t0:.1f}s", file=sys.stderr, flush=True)
    S = ghost_sample(spec.n, spec.ghost_n, spec.seeds["ghost"])
    Gg = build_graph(X[S], spec.ghost_degree, 2 * spec.ghost_degree, "exact", device=device,
                     seed=spec.seeds["ghost"])
    ds = Dataset(spec, X, Q, G, S, Gg, time.time() - t0)
    if use_cache:
        os.makedirs(path, exist_ok=True)
        for n in names:
            tmp = os.path.join(path, f"{n}.{os.getpid()}.npy")
            np.save(tmp, getattr(ds, n))
            os.replace(tmp, os.path.join(path, n + ".npy"))
    if verbose:
        print(f"[dataset] {spec.name}: built in {ds.build_s:.1f}s", file=sys.stderr, flush=True)
    return ds


def write_index_file(path: str, X: np.ndarray, G: np.ndarray, S: Optional[np.ndarray] = None,
                     Gg: Optional[np.ndarray] = None) -> None:
    """The library's index file: magic "ANNIDX01", u64 n, u32 dim, degree,
    n_ghost, ghost_degree, then X (f32), G, S, Gg (u32), little-endian."""
    X = np.ascontiguousarray(X, dtype="<f4")
    G = np.ascontiguousarray(G, dtype="<u4")
    S = np.zeros(0, "<u4") if S is None else np.ascontiguousarray(S, dtype="<u4")
    Gg = np.zeros((0, 0), "<u4") if Gg is None else np.ascontiguousarray(Gg, dtype="<u4")
    with open(path, "wb") as f:
        f.write(b"ANNIDX01")
        f.write(np.array([X.shape[0]], "<u8").tobytes())
        f.write(np.array([X.shape[1], G.shape[1], S.shape[0], Gg.shape[1] if Gg.size else 0], "<u4").tobytes())
        for a in (X, G, S, Gg):
            f.write(a.tobytes())
