"""Seeded synthetic inputs for the graph search: vectors, queries, proximity
graphs and ghost samples.

This package produces INPUTS only. It holds none of the search arithmetic
(distances inside the search, direction bits, codecs, merges): the CPU oracle
under ``oracle/`` and the CUDA library each implement those on their own, and
both consume what this package generates. The proximity graph is an input of
the method (the paper assumes it pre-constructed, Section 2.1), so its builder
lives here too.
"""

from .mixtures import (Mixture, WORKLOADS, WorkloadSpec, make_mixture, make_queries, off_distribution_mask,
                       init_mlp_params)
from .graph import knn_exact, knn_partitioned, prune_by_detours, build_graph, ghost_sample
from .dataset import Dataset, load_dataset, write_index_file, cache_dir
from .shards import Shard, shard_split, build_shards

__all__ = [
    "Mixture", "WORKLOADS", "WorkloadSpec", "make_mixture", "make_queries", "off_distribution_mask", "init_mlp_params",
    "knn_exact", "knn_partitioned", "prune_by_detours", "build_graph", "ghost_sample",
    "Dataset", "load_dataset", "write_index_file", "cache_dir", "Shard", "shard_split", "build_shards",
]
