"""CPU oracle for the graph search (PathWeaver, arXiv 2507.17094).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use it; the CUDA library and its Python binding never import
it. It is plain C (``ann_oracle.c``, built with gcc) driven from numpy, and it
shares no code, header or table with the CUDA path.

Every function names the passage of the paper it follows. Parts with no pin
to anything outside themselves say "parity unpinned".
"""

from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading
from typing import Optional

import numpy as np

INVALID = 0xFFFFFFFF
F32, F16, E4M3 = 0, 1, 2
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ann_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no GPU, no CUDA). Contraction of a*b+c into
    fma is switched off so the only fused operations are the explicit fmaf
    calls; the result is then identical on x86-64 and aarch64."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [(n, C.c_uint32) for n in
                ("k", "L", "W", "T", "m", "n_keep", "it_cool", "reexpand", "entry", "Lg", "Tg",
                 "Tg_given", "g", "rerank")] + [("seed", C.c_uint64), ("qid_base", C.c_uint64),
                                                ("Wg", C.c_uint32), ("min_match", C.c_uint32),
                                                ("judge", C.c_float)]


class Index(C.Structure):
    _fields_ = [("n", C.c_uint64), ("d", C.c_uint32), ("deg", C.c_uint32),
                ("Xs", C.c_void_p), ("X32", C.c_void_p), ("G", C.c_void_p), ("dir", C.c_void_p),
                ("nS", C.c_uint32), ("deg_g", C.c_uint32), ("S", C.c_void_p), ("Gg", C.c_void_p)]


COUNTER_FIELDS = ("iters", "parents", "dgs_parents", "vec_rows",
                  "ghost_iters", "ghost_parents", "ghost_vec_rows", "rerank_rows")
COUNTER_DTYPE = np.dtype([(f, np.uint64) for f in COUNTER_FIELDS])


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, u32, u64 = C.c_void_p, C.c_uint32, C.c_uint64
            L.oracle_f32_to_f16.restype = C.c_uint16
            L.oracle_f32_to_f16.argtypes = [C.c_float]
            L.oracle_f16_to_f32.restype = C.c_float
            L.oracle_f16_to_f32.argtypes = [C.c_uint16]
            L.oracle_f32_to_e4m3.restype = C.c_uint8
            L.oracle_f32_to_e4m3.argtypes = [C.c_float]
            L.oracle_e4m3_to_f32.restype = C.c_float
            L.oracle_e4m3_to_f32.argtypes = [C.c_uint8]
            L.oracle_encode.argtypes = [vp, u64, u32, C.c_int, vp, vp]
            L.oracle_decode.argtypes = [vp, vp, u64, u32, C.c_int, vp]
            L.oracle_dir_table.argtypes = [vp, u64, u32, vp, u32, vp]
            L.oracle_splitmix64.restype = u64
            L.oracle_splitmix64.argtypes = [u64]
            L.oracle_knn_f64.argtypes = [vp, u64, u32, vp, u32, u32, vp, vp, C.c_int]
            L.oracle_pair_dist_f64.argtypes = [vp, u32, vp, u32, u32, vp, vp]
            L.oracle_search.restype = C.c_int
            L.oracle_search.argtypes = [C.POINTER(Index), vp, u32, C.POINTER(Params), vp, u32, vp, vp, vp,
                                        C.c_int]
            _lib = L
        return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


# ---------------------------------------------------------------- formats
def f32_to_f16(x) -> np.ndarray:
    """IEEE 754 binary16, round to nearest even (oracle's own encoder)."""
    L = lib()
    a = np.asarray(x, dtype=np.float32).ravel()
    return np.array([L.oracle_f32_to_f16(float(v)) for v in a], dtype=np.uint16)


def f16_to_f32(h) -> np.ndarray:
    L = lib()
    a = np.asarray(h, dtype=np.uint16).ravel()
    return np.array([L.oracle_f16_to_f32(int(v)) for v in a], dtype=np.float32)


def f32_to_e4m3(x) -> np.ndarray:
    """OCP FP8 E4M3, round to nearest even, saturating to +-448."""
    L = lib()
    a = np.asarray(x, dtype=np.float32).ravel()
    return np.array([L.oracle_f32_to_e4m3(float(v)) for v in a], dtype=np.uint8)


def e4m3_to_f32(c) -> np.ndarray:
    L = lib()
    a = np.asarray(c, dtype=np.uint8).ravel()
    return np.array([L.oracle_e4m3_to_f32(int(v)) for v in a], dtype=np.float32)


def encode(X: np.ndarray, storage: int):
    """Per-vector scale + codes (FP16 power-of-two scale; E4M3 max/448)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    n, d = X.shape
    codes = np.empty((n, d), dtype=np.uint16 if storage == F16 else np.uint8)
    scales = np.empty(n, dtype=np.float32)
    lib().oracle_encode(_p(X), n, d, storage, _p(codes), _p(scales))
    return codes, scales


def decode(codes: np.ndarray, scales: Optional[np.ndarray], storage: int) -> np.ndarray:
    """Stored values as FP32: scale * decode(code)."""
    codes = np.ascontiguousarray(codes)
    n, d = codes.shape
    out = np.empty((n, d), dtype=np.float32)
    sc = np.ascontiguousarray(scales, dtype=np.float32) if scales is not None else np.ones(n, np.float32)
    lib().oracle_decode(_p(codes), _p(sc), n, d, storage, _p(out))
    return out


def stored_vectors(X32: np.ndarray, storage: int) -> np.ndarray:
    """The representation the search reads: X itself for FP32, else the
    decoded codes."""
    if storage == F32:
        return np.ascontiguousarray(X32, dtype=np.float32)
    codes, scales = encode(X32, storage)
    return decode(codes, scales, storage)


def dir_table(Xs: np.ndarray, G: np.ndarray) -> np.ndarray:
    """Sign-bit direction table, Section 3.3.2 (a): uint32 n x deg x ceil(d/32)."""
    Xs = np.ascontiguousarray(Xs, dtype=np.float32)
    G = np.ascontiguousarray(G, dtype=np.uint32)
    n, d = Xs.shape
    deg = G.shape[1]
    w = (d + 31) // 32
    out = np.empty((n, deg, w), dtype=np.uint32)
    lib().oracle_dir_table(_p(Xs), n, d, _p(G), deg, _p(out))
    return out


def splitmix64(x: int) -> int:
    return int(lib().oracle_splitmix64(C.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


# ---------------------------------------------------------------- ground truth
def knn_f64(X: np.ndarray, Q: np.ndarray, k: int, threads: Optional[int] = None):
    """Exact kNN (Eq. 1, squared L2) in FP64; ties by smaller id."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    ids = np.empty((Q.shape[0], k), dtype=np.uint32)
    dists = np.empty((Q.shape[0], k), dtype=np.float64)
    lib().oracle_knn_f64(_p(X), X.shape[0], X.shape[1], _p(Q), Q.shape[0], k, _p(ids), _p(dists),
                         threads or default_threads())
    return ids, dists


def pair_dist_f64(X: np.ndarray, Q: np.ndarray, ids: np.ndarray) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float32)
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    out = np.empty(ids.shape, dtype=np.float64)
    lib().oracle_pair_dist_f64(_p(X), X.shape[1], _p(Q), Q.shape[0], ids.shape[1], _p(ids), _p(out))
    return out


def recall_at_k(ann_ids: np.ndarray, gt_ids: np.ndarray, gt_dists: np.ndarray, X: np.ndarray,
                Q: np.ndarray, k: int = 10):
    """Recall@k (Section 5.1): |N_k^exact ∩ N_k^approx| / k, averaged over
    queries. Returns (tie-aware, strict). Tie-aware counts an approximate id
    as a hit when its FP64 distance is <= the exact k-th distance (so equal
    distances are interchangeable); strict is the plain id-set overlap."""
    a = np.ascontiguousarray(ann_ids[:, :k], dtype=np.uint32)
    strict = np.mean([len(set(a[i].tolist()) & set(gt_ids[i, :k].tolist())) / k for i in range(a.shape[0])])
    da = pair_dist_f64(X, Q, a)
    kth = gt_dists[:, k - 1:k]
    hits = np.zeros(a.shape, dtype=bool)
    for i in range(a.shape[0]):
        seen = set()
        for j in range(k):
            v = int(a[i, j])
            if v != INVALID and v not in seen and da[i, j] <= kth[i, 0]:
                hits[i, j] = True
            seen.add(v)
    return float(hits.sum(axis=1).mean() / k), float(strict)


# ---------------------------------------------------------------- search
def derived_counts(degree: int, max_iters: int, dgs_discard: float, dgs_cooldown: float):
    """Readings of Section 3.3.2: DGS keeps n = deg - round(rho * deg) of a
    parent's neighbours (at least 1); the cool-down is the last
    round(c * T) iterations. Rounding is half-up, in double. Both ratios are
    taken at FP32 precision, the width the search parameters have."""
    dgs_discard = float(np.float32(dgs_discard))
    dgs_cooldown = float(np.float32(dgs_cooldown))
    n_keep = degree - int(math.floor(dgs_discard * degree + 0.5)) if dgs_discard > 0 else degree
    n_keep = max(1, min(degree, n_keep))
    it_cool = max_iters - int(math.floor(dgs_cooldown * max_iters + 0.5))
    return n_keep, max(0, it_cool)


def min_match_count(d: int, dgs_min_match: float) -> int:
    """Reading of the similarity-criterion alternative to DGS's fixed top n
    (the paper's comparison with static pruning, Section 6.3): a neighbour is
    kept when its direction agrees with the query's in at least
    ceil(f * d) of the d dimensions, f = dgs_min_match in (0, 1] taken at
    FP32 precision and multiplied in double; 0 keeps the top-n rule."""
    f = float(np.float32(dgs_min_match))
    if not (0.0 <= f <= 1.0):
        raise ValueError("dgs_min_match must lie in [0, 1]")
    return int(math.ceil(f * d)) if f > 0 else 0


class OracleIndex:
    """Arrays the oracle searches. ``Xs`` is the stored representation
    (decoded FP16/E4M3 or FP32 itself); ``X32`` the FP32 originals."""

    def __init__(self, X32, G, storage=F32, S=None, Gg=None, with_dir=True):
        self.X32 = np.ascontiguousarray(X32, dtype=np.float32)
        self.storage = storage
        self.Xs = stored_vectors(self.X32, storage)
        self.G = np.ascontiguousarray(G, dtype=np.uint32)
        self.dir = dir_table(self.Xs, self.G) if with_dir else None
        self.S = None if S is None else np.ascontiguousarray(S, dtype=np.uint32)
        self.Gg = None if Gg is None else np.ascontiguousarray(Gg, dtype=np.uint32)
        n, d = self.X32.shape
        self._c = Index(n, d, self.G.shape[1], _p(self.Xs), _p(self.X32), _p(self.G), _p(self.dir),
                        0 if self.S is None else self.S.shape[0],
                        0 if self.Gg is None else self.Gg.shape[1], _p(self.S), _p(self.Gg))

    @property
    def n(self):
        return self.X32.shape[0]

    @property
    def degree(self):
        return self.G.shape[1]


def make_params(index: OracleIndex, k=10, itopk=64, search_width=1, max_iters=64, num_seeds=0,
                dgs_discard=0.0, dgs_cooldown=0.3, dgs_reexpand=0, entry=0, ghost_itopk=0,
                ghost_max_iters=16, ghost_max_iters_given=4, ghost_seeds_out=0, rerank=0, seed=0,
                qid_base=0, ghost_search_width=1, dgs_min_match=0.0, ghost_judge=0.0) -> Params:
    if dgs_min_match > 0 and dgs_discard > 0:
        raise ValueError("dgs_min_match and dgs_discard are alternatives: set one")
    if not (0.0 <= ghost_judge < float("inf")):
        raise ValueError("ghost_judge must be finite and >= 0")
    n_keep, it_cool = derived_counts(index.degree, max_iters, dgs_discard, dgs_cooldown)
    min_match = min_match_count(index.X32.shape[1], dgs_min_match)
    Lg = ghost_itopk or min(itopk, 64)
    return Params(k, itopk, search_width, max_iters, num_seeds, n_keep, it_cool, dgs_reexpand, entry,
                  Lg, ghost_max_iters, ghost_max_iters_given, ghost_seeds_out or Lg, rerank, seed, qid_base,
                  ghost_search_width or 1, min_match, float(np.float32(ghost_judge)))


def search(index: OracleIndex, Q: np.ndarray, given_ghost_seeds: Optional[np.ndarray] = None,
           threads: Optional[int] = None, given_seeds: Optional[np.ndarray] = None, **kw):
    """Batched beam search (Section 2.2) with ghost staging (Section 3.2.2)
    and DGS (Section 3.3.2). Given seeds (nq x P) are ghost indices for
    entry 2 (`given_ghost_seeds`) or base node ids for entry 3
    (`given_seeds`, the start of an extended path, Section 3.1.2). Returns
    (ids uint32 nq x k, dists float32 nq x k, per-query counters)."""
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    p = make_params(index, **kw)
    nq = Q.shape[0]
    ids = np.empty((nq, p.k), dtype=np.uint32)
    dists = np.empty((nq, p.k), dtype=np.float32)
    cnt = np.zeros(nq, dtype=COUNTER_DTYPE)
    P = 0
    g = None
    if given_ghost_seeds is not None and given_seeds is not None:
        raise ValueError("give ghost seeds or base seeds, not both")
    if given_seeds is not None:
        given_ghost_seeds = given_seeds
    if given_ghost_seeds is not None:
        g = np.ascontiguousarray(given_ghost_seeds, dtype=np.uint32)
        P = g.shape[1]
    rc = lib().oracle_search(C.byref(index._c), _p(Q), nq, C.byref(p), _p(g), P, _p(ids), _p(dists),
                             _p(cnt), threads or default_threads())
    if rc != 0:
        raise ValueError("oracle_search rejected its arguments")
    return ids, dists, cnt


def algorithmic_bytes(cnt: np.ndarray, d: int, degree: int, row_bytes: int, k: int,
                      ghost_degree: int = 0, rerank_row_bytes: int = 0) -> np.ndarray:
    """Bytes the search must move per query, from the exact event counters:
    query + adjacency rows + direction rows + gathered vector rows (ghost and
    base) + rerank rows + results. Visited-set and queue traffic stay on chip."""
    w = (d + 31) // 32
    return (4 * d
            + cnt["parents"].astype(np.int64) * 4 * degree
            + cnt["dgs_parents"].astype(np.int64) * 4 * degree * w
            + cnt["vec_rows"].astype(np.int64) * row_bytes
            + cnt["ghost_parents"].astype(np.int64) * 4 * ghost_degree
            + cnt["ghost_vec_rows"].astype(np.int64) * row_bytes
            + cnt["rerank_rows"].astype(np.int64) * rerank_row_bytes
            + 8 * k)
