"""GB300-native batched graph beam search (PathWeaver, arXiv 2507.17094).

The search runs in hand-written CUDA kernels for sm_103a behind the C ABI in
``include/ann.h`` (``libann.so``); this package is its build step and a thin
ctypes binding. PyTorch supplies device memory and streams.
"""

from .binding import (E4M3, ENTRY_GHOST, ENTRY_GIVEN_GHOST, ENTRY_RANDOM, EXPORTS, F16, F32, INVALID,
                      PROFILE_PHASE_NAMES, PROFILE_PHASES, PROFILE_STAGE_NAMES, PROFILE_STAGES, STATS_DTYPE, AnnError, Index, MLP, SearchParams, Server, Shards, dir_table, encode, lib, make_params,
                      replay, stats_to_numpy, knn_exact, graph_prune)
from .build import build

__all__ = ["E4M3", "ENTRY_GHOST", "ENTRY_GIVEN_GHOST", "ENTRY_RANDOM", "EXPORTS", "F16", "F32", "INVALID",
           "PROFILE_PHASE_NAMES", "PROFILE_PHASES", "PROFILE_STAGE_NAMES", "PROFILE_STAGES",
           "STATS_DTYPE", "AnnError", "Index", "MLP", "SearchParams", "Server", "Shards", "replay", "build", "dir_table", "encode", "lib",
           "make_params", "stats_to_numpy", "knn_exact", "graph_prune"]
