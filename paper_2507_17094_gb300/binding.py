"""Python binding of libann.so (ctypes). Argument marshalling only: every step
of the search runs in the library's CUDA kernels; PyTorch provides device
memory and streams.

The binding never falls back to anything: if libann.so is missing or no GPU
is present, the calls raise.
"""

from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

from .build import LIB

INVALID = 0xFFFFFFFF
F32, F16, E4M3 = 0, 1, 2
ENTRY_RANDOM, ENTRY_GHOST, ENTRY_GIVEN_GHOST = 0, 1, 2
# ann_search_profile's table: stages x phases (see include/ann.h)
PROFILE_STAGES, PROFILE_PHASES = 3, 8
PROFILE_STAGE_NAMES = ("ghost", "base", "finish")
PROFILE_PHASE_NAMES = ("select+adjacency", "dgs", "visited", "gather_wait", "distance", "merge", "other", "unused")
STATUS = {0: "ANN_OK", 1: "ANN_EINVAL", 2: "ANN_ENOMEM", 3: "ANN_ECUDA", 4: "ANN_EIO", 5: "ANN_ETIMEOUT",
          6: "ANN_EBUSY", 7: "ANN_EDEVICE"}

# Every symbol include/ann.h declares (checked by the tests).
EXPORTS = ("ann_default_params", "ann_index_create", "ann_index_load", "ann_index_free", "ann_index_info",
           "ann_index_export", "ann_search", "ann_search_host", "ann_search_host_noalloc", "ann_search_profile",
           "ann_sync", "ann_shards_create", "ann_shards_free", "ann_shards_link", "ann_shards_set_links",
           "ann_shards_get_links", "ann_shards_search", "ann_knn_exact", "ann_graph_prune",
           "ann_encode", "ann_dir_table", "ann_mlp_create", "ann_mlp_free", "ann_mlp_set_params", "ann_mlp_get",
           "ann_mlp_forward", "ann_mlp_train_step", "ann_mlp_train_epochs", "ann_mlp_predict", "ann_mlp_sync",
           "ann_mlp_save", "ann_mlp_load", "ann_mlp_set_input_norm", "ann_mlp_get_input_norm",
           "ann_mlp_fit_input_norm", "ann_mlp_confidence_threshold",
           "ann_selftest_timeout",
           "ann_ghost_index_of", "ann_server_create", "ann_server_submit", "ann_server_poll",
           "ann_server_in_flight", "ann_server_destroy", "ann_last_error")


class AnnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class SearchParams(C.Structure):
    _fields_ = [("k", C.c_uint32), ("itopk", C.c_uint32), ("search_width", C.c_uint32),
                ("max_iters", C.c_uint32), ("num_seeds", C.c_uint32), ("dgs_discard", C.c_float),
                ("dgs_cooldown", C.c_float), ("dgs_reexpand", C.c_uint32), ("entry", C.c_uint32),
                ("ghost_itopk", C.c_uint32), ("ghost_max_iters", C.c_uint32),
                ("ghost_max_iters_given", C.c_uint32), ("ghost_seeds_out", C.c_uint32),
                ("rerank", C.c_uint32), ("seed", C.c_uint64), ("qid_base", C.c_uint64),
                ("ghost_search_width", C.c_uint32), ("dgs_min_match", C.c_float), ("ghost_judge", C.c_float)]


class ServerConfig(C.Structure):
    _fields_ = [("capacity", C.c_uint32), ("max_requests", C.c_uint32), ("max_params", SearchParams),
                ("seeds_per_query", C.c_uint32), ("tau", C.c_float), ("queries_per_warp", C.c_uint32),
                ("streams", C.c_uint32)]


class Completion(C.Structure):
    _fields_ = [("req_id", C.c_uint64), ("status", C.c_uint32), ("nq", C.c_uint32), ("latency_s", C.c_double)]


STATS_FIELDS = ("iters", "parents", "dgs_parents", "vec_rows", "ghost_iters", "ghost_parents",
                "ghost_vec_rows", "rerank_rows", "hash_resets", "status")
STATS_DTYPE = np.dtype([(f, np.uint32) for f in STATS_FIELDS])

_lock = threading.Lock()
_lib = None


def lib() -> C.CDLL:
    """Load libann.so (built by ``paper_2507_17094_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise RuntimeError(f"{LIB} is missing: run paper_2507_17094_gb300.build.build() first")
            L = C.CDLL(LIB)
            vp, u32, u64, st = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int
            L.ann_default_params.argtypes = [C.POINTER(SearchParams)]
            L.ann_default_params.restype = None
            L.ann_index_create.argtypes = [C.c_int, C.c_int, u64, u32, u32, vp, vp, u32, vp, u32, vp, u32, u32,
                                           C.POINTER(vp)]
            L.ann_index_load.argtypes = [C.c_char_p, C.c_int, C.c_int, u32, u32, C.POINTER(vp)]
            L.ann_index_free.argtypes = [vp]
            L.ann_index_info.argtypes = [vp] + [vp] * 6
            L.ann_index_export.argtypes = [vp, C.c_int, vp, u64]
            L.ann_search.argtypes = [vp, vp, u32, C.POINTER(SearchParams), vp, u32, vp, vp, vp, vp]
            L.ann_search_host.argtypes = [vp, vp, u32, C.POINTER(SearchParams), vp, u32, vp, vp, vp]
            L.ann_search_host_noalloc.argtypes = [vp, vp, u32, C.POINTER(SearchParams), vp, vp, vp]
            L.ann_search_profile.argtypes = [vp, vp, u32, C.POINTER(SearchParams), vp, u32, vp, vp, vp, vp]
            L.ann_sync.argtypes = [vp, vp]
            L.ann_knn_exact.argtypes = [vp, u64, u32, u32, vp, vp]
            L.ann_graph_prune.argtypes = [vp, u64, u32, u32, vp, vp]
            L.ann_shards_create.argtypes = [vp, u32, vp, C.POINTER(vp)]
            L.ann_shards_free.argtypes = [vp]
            L.ann_shards_link.argtypes = [vp, C.POINTER(SearchParams), vp]
            L.ann_shards_set_links.argtypes = [vp, u32, vp]
            L.ann_shards_get_links.argtypes = [vp, u32, vp]
            L.ann_shards_search.argtypes = [vp, vp, u32, C.POINTER(SearchParams), u32, vp, vp, vp, vp]
            L.ann_selftest_timeout.argtypes = [vp]
            f32 = C.c_float
            L.ann_mlp_create.argtypes = [C.c_int, u32, u32, u32, u32, u32, C.POINTER(vp)]
            L.ann_mlp_free.argtypes = [vp]
            L.ann_mlp_set_params.argtypes = [vp] * 7
            L.ann_mlp_get.argtypes = [vp, C.c_int] + [vp] * 6
            L.ann_mlp_forward.argtypes = [vp, vp, u32, vp, vp]
            L.ann_mlp_train_step.argtypes = [vp, vp, vp, u32, f32, f32, f32, f32, f32, vp, vp]
            L.ann_mlp_predict.argtypes = [vp, vp, u32, u32, f32, vp, vp, vp]
            L.ann_mlp_sync.argtypes = [vp, vp]
            L.ann_mlp_save.argtypes = [vp, C.c_char_p]
            L.ann_mlp_set_input_norm.argtypes = [vp, vp, vp]
            L.ann_mlp_get_input_norm.argtypes = [vp, vp, vp]
            L.ann_mlp_fit_input_norm.argtypes = [vp, vp, u32, vp]
            L.ann_mlp_confidence_threshold.argtypes = [vp, vp, u32, C.c_double, C.POINTER(f32), vp]
            L.ann_mlp_load.argtypes = [C.c_char_p, C.c_int, u32, C.POINTER(vp)]
            L.ann_mlp_train_epochs.argtypes = [vp, vp, vp, u32, u32, u32, f32, f32, f32, f32, f32, u64, vp, vp]
            L.ann_ghost_index_of.argtypes = [vp, vp, u32, vp, vp]
            L.ann_server_create.argtypes = [vp, C.POINTER(ServerConfig), vp, C.POINTER(vp)]
            L.ann_server_submit.argtypes = [vp, u64, vp, u32, C.POINTER(SearchParams), vp, vp]
            L.ann_server_poll.argtypes = [vp, C.POINTER(Completion), u32, C.POINTER(u32)]
            L.ann_server_in_flight.argtypes = [vp]
            L.ann_server_in_flight.restype = u32
            L.ann_server_destroy.argtypes = [vp]
            L.ann_encode.argtypes = [vp, u64, u32, C.c_int, vp, vp, vp]
            L.ann_dir_table.argtypes = [vp, vp, C.c_int, u64, u32, vp, u32, vp, vp]
            L.ann_last_error.restype = C.c_char_p
            for f in EXPORTS:
                if f in ("ann_default_params", "ann_last_error", "ann_server_in_flight"):
                    continue
                getattr(L, f).restype = st
            _lib = L
        return _lib


def _check(status: int):
    if status != 0:
        raise AnnError(status, lib().ann_last_error().decode(errors="replace"))


def _np_ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def make_params(**kw) -> SearchParams:
    """ann_search_params from keyword arguments over the library defaults."""
    p = SearchParams()
    lib().ann_default_params(C.byref(p))
    names = {f for f, _ in SearchParams._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown search parameter {k!r}")
        setattr(p, k, v)
    return p


class Index:
    """A device-resident index (library-owned memory)."""

    def __init__(self, vectors: np.ndarray, graph: np.ndarray, storage: int = F32,
                 ghost_ids: Optional[np.ndarray] = None, ghost_graph: Optional[np.ndarray] = None,
                 keep_fp32: bool = True, build_dir: bool = True, device: int = 0, _handle=None):
        self._h = C.c_void_p()
        if _handle is not None:
            self._h = _handle
        else:
            X = np.ascontiguousarray(vectors, dtype=np.float32)
            G = np.ascontiguousarray(graph, dtype=np.uint32)
            S = None if ghost_ids is None else np.ascontiguousarray(ghost_ids, dtype=np.uint32)
            GG = None if ghost_graph is None else np.ascontiguousarray(ghost_graph, dtype=np.uint32)
            _check(lib().ann_index_create(device, storage, X.shape[0], X.shape[1], G.shape[1], _np_ptr(X),
                                          _np_ptr(G), 0 if S is None else S.shape[0], _np_ptr(S),
                                          0 if GG is None else GG.shape[1], _np_ptr(GG), int(keep_fp32),
                                          int(build_dir), C.byref(self._h)))
        n, d, deg, sto, ng, gd = (C.c_uint64(), C.c_uint32(), C.c_uint32(), C.c_uint32(), C.c_uint32(),
                                  C.c_uint32())
        _check(lib().ann_index_info(self._h, C.byref(n), C.byref(d), C.byref(deg), C.byref(sto), C.byref(ng),
                                    C.byref(gd)))
        self.n, self.dim, self.degree, self.storage = n.value, d.value, deg.value, sto.value
        self.n_ghost, self.ghost_degree = ng.value, gd.value
        self.device = device

    @classmethod
    def load(cls, path: str, storage: int = F32, keep_fp32: bool = True, build_dir: bool = True, device: int = 0):
        h = C.c_void_p()
        _check(lib().ann_index_load(path.encode(), device, storage, int(keep_fp32), int(build_dir), C.byref(h)))
        return cls(None, None, _handle=h, device=device)

    def close(self):
        if self._h:
            lib().ann_index_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def export(self, which: int) -> np.ndarray:
        w = (self.dim + 31) // 32
        dt = {F32: np.float32, F16: np.uint16, E4M3: np.uint8}[self.storage]
        shape, dtype = {0: ((self.n, self.dim), dt), 1: ((self.n,), np.float32),
                        2: ((self.n, self.degree, w), np.uint32), 3: ((self.n_ghost, self.dim), dt),
                        4: ((self.n_ghost,), np.float32)}[which]
        out = np.empty(shape, dtype=dtype)
        _check(lib().ann_index_export(self._h, which, _np_ptr(out), out.nbytes))
        return out

    def search(self, queries, given=None, stats: bool = False, stream=None, out=None, **params):
        """Search device queries (a CUDA float32 tensor nq x dim). Returns
        (ids int32-view of uint32, dists, stats-or-None) as CUDA tensors; the
        call is asynchronous on ``stream``."""
        import torch
        p = make_params(**params)
        nq = queries.shape[0]
        assert queries.is_cuda and queries.dtype == torch.float32 and queries.is_contiguous()
        if out is None:
            ids = torch.empty((nq, p.k), dtype=torch.int32, device=queries.device)
            dists = torch.empty((nq, p.k), dtype=torch.float32, device=queries.device)
        else:
            ids, dists = out
        st = torch.empty((nq, len(STATS_FIELDS)), dtype=torch.int32, device=queries.device) if stats else None
        g_ptr, n_given = None, 0
        if given is not None:
            assert given.is_cuda and given.dtype == torch.int32 and given.is_contiguous()
            g_ptr, n_given = given.data_ptr(), given.shape[1]
        _check(lib().ann_search(self._h, queries.data_ptr(), nq, C.byref(p), g_ptr, n_given, ids.data_ptr(),
                                dists.data_ptr(), None if st is None else st.data_ptr(), _stream_ptr(stream)))
        return ids, dists, st

    def search_host(self, queries: np.ndarray, given: Optional[np.ndarray] = None, stream=None, **params):
        """Search host queries; copies in and out inside the call (synchronous)."""
        p = make_params(**params)
        Q = np.ascontiguousarray(queries, dtype=np.float32)
        nq = Q.shape[0]
        ids = np.empty((nq, p.k), dtype=np.uint32)
        dists = np.empty((nq, p.k), dtype=np.float32)
        G = None if given is None else np.ascontiguousarray(given, dtype=np.uint32)
        _check(lib().ann_search_host(self._h, _np_ptr(Q), nq, C.byref(p), _np_ptr(G),
                                     0 if G is None else G.shape[1], _np_ptr(ids), _np_ptr(dists),
                                     _stream_ptr(stream)))
        return ids, dists

    def search_host_noalloc(self, queries: np.ndarray, stream=None, **params):
        """The host-buffer search through the entry point that allocates no
        device memory (fixed per-device scratch; see include/ann.h)."""
        p = make_params(**params)
        Q = np.ascontiguousarray(queries, dtype=np.float32)
        nq = Q.shape[0]
        ids = np.empty((nq, p.k), dtype=np.uint32)
        dists = np.empty((nq, p.k), dtype=np.float32)
        _check(lib().ann_search_host_noalloc(self._h, _np_ptr(Q), nq, C.byref(p), _np_ptr(ids), _np_ptr(dists),
                                             _stream_ptr(stream)))
        return ids, dists

    def search_profile(self, queries, given=None, stream=None, **params):
        """The search through ann_search_profile: (ids, dists, cycles) with
        cycles a (stage, phase) uint64 array of summed warp cycles."""
        import torch
        p = make_params(**params)
        nq = queries.shape[0]
        assert queries.is_cuda and queries.dtype == torch.float32 and queries.is_contiguous()
        ids = torch.empty((nq, p.k), dtype=torch.int32, device=queries.device)
        dists = torch.empty((nq, p.k), dtype=torch.float32, device=queries.device)
        cyc = np.zeros((PROFILE_STAGES, PROFILE_PHASES), dtype=np.uint64)
        g_ptr, n_given = None, 0
        if given is not None:
            g_ptr, n_given = given.data_ptr(), given.shape[1]
        _check(lib().ann_search_profile(self._h, queries.data_ptr(), nq, C.byref(p), g_ptr, n_given, ids.data_ptr(),
                                        dists.data_ptr(), _np_ptr(cyc), _stream_ptr(stream)))
        return ids, dists, cyc

    def sync(self, stream=None):
        _check(lib().ann_sync(self._h, _stream_ptr(stream)))

    def selftest_timeout(self):
        """Run the device-failure self-test (see include/ann.h); raises on failure."""
        _check(lib().ann_selftest_timeout(self._h))

    def ghost_index_of(self, ids, stream=None):
        """Ghost index of each node id (CUDA int32 tensor); INVALID if not a ghost."""
        import torch
        flat = ids.reshape(-1).contiguous()
        out = torch.empty_like(flat)
        _check(lib().ann_ghost_index_of(self._h, flat.data_ptr(), flat.numel(), out.data_ptr(), _stream_ptr(stream)))
        return out.reshape(ids.shape)


class MLP:
    """The learned-entry network (device-resident; see include/ann.h)."""

    def __init__(self, in_dim: int, hidden1: int, hidden2: int, out_dim: int, max_batch: int, device: int = 0):
        self._h = C.c_void_p()
        _check(lib().ann_mlp_create(device, in_dim, hidden1, hidden2, out_dim, max_batch, C.byref(self._h)))
        self.dims = (in_dim, hidden1, hidden2, out_dim)
        self.max_batch = max_batch

    @classmethod
    def load(cls, path: str, max_batch: int, device: int = 0) -> "MLP":
        """An MLP created from a file written by save()."""
        self = cls.__new__(cls)
        self._h = C.c_void_p()
        _check(lib().ann_mlp_load(os.fsencode(path), device, max_batch, C.byref(self._h)))
        hdr = np.fromfile(path, dtype=np.uint32, count=6)
        self.dims = tuple(int(v) for v in hdr[2:6])
        self.max_batch = max_batch
        return self

    def save(self, path: str):
        _check(lib().ann_mlp_save(self._h, os.fsencode(path)))

    def close(self):
        if self._h:
            lib().ann_mlp_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _shapes(self):
        d, h1, h2, o = self.dims
        return [(h1, d), (h1,), (h2, h1), (h2,), (o, h2), (o,)]

    def set_params(self, W1, b1, W2, b2, W3, b3):
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (W1, b1, W2, b2, W3, b3)]
        for a, shp in zip(arrs, self._shapes()):
            assert a.shape == shp, (a.shape, shp)
        _check(lib().ann_mlp_set_params(self._h, *[_np_ptr(a) for a in arrs]))

    def get(self, which: int = 0):
        """Parameters (0) or last gradients (1) as six float32 arrays."""
        out = [np.empty(shp, dtype=np.float32) for shp in self._shapes()]
        _check(lib().ann_mlp_get(self._h, which, *[_np_ptr(a) for a in out]))
        return out

    def set_input_norm(self, mean=None, inv_std=None):
        """Standardise queries per dimension on the device: (x - mean) * inv_std."""
        if mean is None:
            _check(lib().ann_mlp_set_input_norm(self._h, None, None))
            return
        mu = np.ascontiguousarray(mean, dtype=np.float32).reshape(self.dims[0])
        isd = np.ascontiguousarray(inv_std, dtype=np.float32).reshape(self.dims[0])
        _check(lib().ann_mlp_set_input_norm(self._h, _np_ptr(mu), _np_ptr(isd)))

    def fit_input_norm(self, x, stream=None):
        """Standardisation statistics of the device queries x (n x in_dim),
        computed and installed on the device (synchronous)."""
        assert x.is_cuda and x.is_contiguous() and x.shape[1] == self.dims[0]
        _check(lib().ann_mlp_fit_input_norm(self._h, x.data_ptr(), x.shape[0], _stream_ptr(stream)))

    def confidence_threshold(self, pmax, fallback: float, stream=None) -> float:
        """The `fallback` lower quantile of the device values pmax (see
        include/ann.h), computed on the device."""
        tau = C.c_float()
        assert pmax.is_cuda and pmax.is_contiguous()
        _check(lib().ann_mlp_confidence_threshold(self._h, pmax.data_ptr(), pmax.numel(), float(fallback),
                                                  C.byref(tau), _stream_ptr(stream)))
        return float(tau.value)

    def get_input_norm(self):
        mu = np.empty(self.dims[0], np.float32)
        isd = np.empty(self.dims[0], np.float32)
        _check(lib().ann_mlp_get_input_norm(self._h, _np_ptr(mu), _np_ptr(isd)))
        return mu, isd

    def forward(self, x, stream=None):
        import torch
        n = x.shape[0]
        z = torch.empty((n, self.dims[3]), dtype=torch.float32, device=x.device)
        _check(lib().ann_mlp_forward(self._h, x.data_ptr(), n, z.data_ptr(), _stream_ptr(stream)))
        return z

    def train_step(self, x, labels, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, loss=None,
                   stream=None):
        _check(lib().ann_mlp_train_step(self._h, x.data_ptr(), labels.data_ptr(), x.shape[0], lr, beta1, beta2,
                                        eps, weight_decay, None if loss is None else loss.data_ptr(),
                                        _stream_ptr(stream)))

    def train_epochs(self, x, labels, batch: int = 1024, epochs: int = 1, lr=1e-3, beta1=0.9, beta2=0.999,
                     eps=1e-8, weight_decay=0.0, seed: int = 0, stream=None) -> np.ndarray:
        losses = np.zeros(epochs, dtype=np.float32)
        _check(lib().ann_mlp_train_epochs(self._h, x.data_ptr(), labels.data_ptr(), x.shape[0], batch, epochs, lr,
                                          beta1, beta2, eps, weight_decay, seed, _np_ptr(losses),
                                          _stream_ptr(stream)))
        return losses

    def predict(self, x, P: int = 8, tau: float = 0.0, stream=None):
        import torch
        n = x.shape[0]
        seeds = torch.empty((n, P), dtype=torch.int32, device=x.device)
        pmax = torch.empty((n,), dtype=torch.float32, device=x.device)
        _check(lib().ann_mlp_predict(self._h, x.data_ptr(), n, P, tau, seeds.data_ptr(), pmax.data_ptr(),
                                     _stream_ptr(stream)))
        return seeds, pmax

    def sync(self, stream=None):
        _check(lib().ann_mlp_sync(self._h, _stream_ptr(stream)))


class Shards:
    """A path-extension ring over shard indexes (see include/ann.h)."""

    def __init__(self, indexes, global_ids):
        self.indexes = list(indexes)
        self._gids = [np.ascontiguousarray(g, dtype=np.uint32) for g in global_ids]
        arr = (C.c_void_p * len(self.indexes))(*[ix._h.value for ix in self.indexes])
        garr = (C.c_void_p * len(self._gids))(*[g.ctypes.data for g in self._gids])
        self._h = C.c_void_p()
        _check(lib().ann_shards_create(arr, len(self.indexes), garr, C.byref(self._h)))
        self.n_shards = len(self.indexes)

    def link(self, stream=None, **params):
        _check(lib().ann_shards_link(self._h, C.byref(make_params(**params)), _stream_ptr(stream)))

    def set_links(self, shard: int, links: np.ndarray):
        a = np.ascontiguousarray(links, dtype=np.uint32)
        _check(lib().ann_shards_set_links(self._h, shard, _np_ptr(a)))

    def get_links(self, shard: int) -> np.ndarray:
        out = np.empty(self.indexes[shard].n, dtype=np.uint32)
        _check(lib().ann_shards_get_links(self._h, shard, _np_ptr(out)))
        return out

    def search(self, queries, n_forward: int = 1, stats: bool = False, stream=None, **params):
        """Device queries in; (dataset ids int32-view, dists, stats (N x nq) or None) as CUDA tensors."""
        import torch
        p = make_params(**params)
        nq = queries.shape[0]
        assert queries.is_cuda and queries.dtype == torch.float32 and queries.is_contiguous()
        ids = torch.empty((nq, p.k), dtype=torch.int32, device=queries.device)
        dists = torch.empty((nq, p.k), dtype=torch.float32, device=queries.device)
        st = (torch.empty((self.n_shards, nq, len(STATS_FIELDS)), dtype=torch.int32, device=queries.device)
              if stats else None)
        _check(lib().ann_shards_search(self._h, queries.data_ptr(), nq, C.byref(p), n_forward, ids.data_ptr(),
                                       dists.data_ptr(), None if st is None else st.data_ptr(),
                                       _stream_ptr(stream)))
        return ids, dists, st

    def close(self):
        if self._h:
            lib().ann_shards_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def knn_exact(x, K: int, stream=None):
    """Exact kNN lists of the device rows x (n x dim FP32): int32-view CUDA
    tensor n x K (ann_knn_exact)."""
    import torch
    assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()
    ids = torch.empty((x.shape[0], K), dtype=torch.int32, device=x.device)
    _check(lib().ann_knn_exact(x.data_ptr(), x.shape[0], x.shape[1], K, ids.data_ptr(), _stream_ptr(stream)))
    return ids


def graph_prune(knn, degree: int, stream=None):
    """The pruned graph of device kNN lists (int32-view n x K): CUDA tensor
    n x degree (ann_graph_prune)."""
    import torch
    assert knn.is_cuda and knn.dtype == torch.int32 and knn.is_contiguous()
    g = torch.empty((knn.shape[0], degree), dtype=torch.int32, device=knn.device)
    _check(lib().ann_graph_prune(knn.data_ptr(), knn.shape[0], knn.shape[1], degree, g.data_ptr(),
                                 _stream_ptr(stream)))
    return g


def stats_to_numpy(st) -> np.ndarray:
    a = st.cpu().numpy().astype(np.uint32)
    return np.ascontiguousarray(a).view(STATS_DTYPE).reshape(-1)


def encode(x, storage: int, stream=None):
    """Device FP32 rows -> (codes, scales) as CUDA tensors (dense rows)."""
    import torch
    n, d = x.shape
    codes = torch.empty((n, d), dtype=torch.int16 if storage == F16 else torch.uint8, device=x.device)
    scales = torch.empty((n,), dtype=torch.float32, device=x.device)
    _check(lib().ann_encode(x.data_ptr(), n, d, storage, codes.data_ptr(), scales.data_ptr(),
                            _stream_ptr(stream)))
    return codes, scales


def dir_table(vectors, scales, storage: int, graph, stream=None):
    """Direction table of stored vectors (codes + scales, or FP32 rows)."""
    import torch
    n, d = vectors.shape
    deg = graph.shape[1]
    w = (d + 31) // 32
    out = torch.empty((n, deg, w), dtype=torch.int32, device=vectors.device)
    _check(lib().ann_dir_table(vectors.data_ptr(), None if scales is None else scales.data_ptr(), storage, n, d,
                               graph.data_ptr(), deg, out.data_ptr(), _stream_ptr(stream)))
    return out


class Server:
    """Continuous-batching server over an index (see include/ann.h)."""

    def __init__(self, index: Index, capacity: int, max_requests: int, max_params: dict, mlp: "MLP" = None,
                 seeds_per_query: int = 8, tau: float = 0.0, queries_per_warp: int = 0, streams: int = 0):
        cfg = ServerConfig(capacity, max_requests, make_params(**max_params), seeds_per_query, tau,
                           queries_per_warp, streams)
        self._h = C.c_void_p()
        _check(lib().ann_server_create(index._h, C.byref(cfg), None if mlp is None else mlp._h, C.byref(self._h)))
        self.index = index
        self._keep = {}

    def submit(self, req_id: int, queries: np.ndarray, **params) -> bool:
        """Admit a request; False when the server is full (ANN_EBUSY)."""
        p = make_params(**params)
        Q = np.ascontiguousarray(queries, dtype=np.float32)
        ids = np.empty((Q.shape[0], p.k), dtype=np.uint32)
        dists = np.empty((Q.shape[0], p.k), dtype=np.float32)
        st = lib().ann_server_submit(self._h, req_id, _np_ptr(Q), Q.shape[0], C.byref(p), _np_ptr(ids),
                                     _np_ptr(dists))
        if st == 6:
            return False
        _check(st)
        self._keep[req_id] = (ids, dists)
        return True

    def poll(self, max_n: int = 256):
        """Completed requests: list of (req_id, ids, dists, latency_s)."""
        buf = (Completion * max_n)()
        n = C.c_uint32()
        _check(lib().ann_server_poll(self._h, buf, max_n, C.byref(n)))
        out = []
        for i in range(n.value):
            ids, dists = self._keep.pop(buf[i].req_id)
            out.append((buf[i].req_id, ids, dists, buf[i].latency_s))
        return out

    def in_flight(self) -> int:
        return int(lib().ann_server_in_flight(self._h))

    def close(self):
        if self._h:
            lib().ann_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def replay(server: Server, trace, timeout_s: float = 120.0):
    """Drive `server` with a trace of (arrival_s, req_id, queries, params):
    submit each request at its arrival time (retrying while the server is
    full), collect completions. Returns {req_id: (ids, dists, latency_s)} and
    the wall time from the first arrival to the last completion."""
    import time
    results = {}
    pending = sorted(trace, key=lambda t: t[0])
    t0 = time.perf_counter()
    i = 0
    while len(results) < len(trace):
        now = time.perf_counter() - t0
        while i < len(pending) and pending[i][0] <= now:
            _, rid, q, prm = pending[i]
            if not server.submit(rid, q, **prm):
                break
            i += 1
        for rid, ids, dists, lat in server.poll():
            results[rid] = (ids, dists, lat)
        if time.perf_counter() - t0 > timeout_s:
            raise TimeoutError(f"serving trace did not finish: {len(results)}/{len(trace)} done")
    return results, time.perf_counter() - t0
