"""Learned entry, end to end, as a sequence of C-ABI calls (no arithmetic here).

1. Labels: each training query's best ghost node, as ghost staging finds it
   (ann_search with no base iterations and k = 1, then ann_ghost_index_of).
2. Training: ann_mlp_train_epochs on (query, label) pairs.
3. Inference: ann_mlp_predict gives the top-P ghost nodes per query (or the
   fallback marker below the confidence threshold tau); ann_search with
   entry = ANN_ENTRY_GIVEN_GHOST starts its ghost stage from them.
4. Judge: ghost staging judges the network's seeds. A query whose ghost
   stage, after its few iterations from the seeds, holds no node nearer than
   the judge distance (ann_search_params.ghost_judge, calibrated like tau
   on validation queries) continues as plain ghost staging.
"""

from __future__ import annotations

import numpy as np

from .binding import ENTRY_GHOST, ENTRY_GIVEN_GHOST, INVALID, MLP, Index


def ghost_labels(index: Index, queries, seed: int, ghost_itopk: int = 64, ghost_max_iters: int = 64,
                 ghost_search_width: int = 1, stream=None):
    """Best ghost node of each query by ghost staging (CUDA int32 tensor)."""
    ids, _, _ = index.search(queries, k=1, itopk=ghost_itopk, max_iters=0, entry=ENTRY_GHOST,
                             ghost_itopk=ghost_itopk, ghost_max_iters=ghost_max_iters,
                             ghost_search_width=ghost_search_width, seed=seed, stream=stream)
    return index.ghost_index_of(ids[:, 0].contiguous(), stream=stream)


class LearnedEntry:
    """An MLP over the ghost set, trained on the index's own ghost staging."""

    def __init__(self, index: Index, params, hidden=(512, 512), max_batch: int = 16384, P: int = 8):
        self.index = index
        self.P = P
        self.mlp = MLP(index.dim, hidden[0], hidden[1], index.n_ghost, max_batch, device=index.device)
        self.mlp.set_params(*params)
        self.tau = 0.0
        self.judge = 0.0
        self.losses = None

    def fit(self, train_queries, labels, epochs: int = 5, batch: int = 1024, lr: float = 1e-3, seed: int = 0,
            standardise: bool = True):
        """Train on (query, label) pairs. With `standardise`, the network first
        takes each query dimension to zero mean and unit variance over the
        training queries (the library applies it on the device)."""
        if standardise:
            self.mlp.fit_input_norm(train_queries)
        self.losses = self.mlp.train_epochs(train_queries, labels, batch=batch, epochs=epochs, lr=lr, seed=seed)
        return self.losses

    def calibrate(self, val_queries, val_labels, fallback: float = 0.05):
        """Set tau from a validation split: the `fallback` quantile of the
        validation queries' top softmax probabilities (ann_mlp_confidence_
        threshold), so that fraction of in-distribution queries, and any query
        the network is less sure of, falls back to plain ghost staging.
        Returns tau and the fraction of validation queries whose label is
        among the P seeds."""
        seeds, pmax = self.mlp.predict(val_queries, P=self.P, tau=0.0)
        hit = (seeds == val_labels[:, None]).any(dim=1).float().mean().item()
        self.tau = self.mlp.confidence_threshold(pmax, fallback)
        return self.tau, float(hit)

    def calibrate_judge(self, val_queries, continue_fraction: float = 0.05, stream=None, **search_params):
        """Set the judge distance from a validation split: the (1 -
        continue_fraction) quantile (the same device quantile as tau) of the
        squared distance of each validation query's best ghost node after
        the ghost stage from the network's seeds, run with `search_params`'
        ghost settings. That fraction of in-distribution queries, and any
        query farther from every ghost node it reached, continues as plain
        ghost staging. Returns the judge distance."""
        seeds, _ = self.seeds(val_queries, stream=stream)
        # the ghost stage's own (stored-precision) distance, as the kernel's judge sees it
        p = dict(search_params, k=1, max_iters=0, entry=ENTRY_GIVEN_GHOST, ghost_judge=0.0, rerank=0)
        p["itopk"] = max(1, int(p.get("ghost_itopk") or 64))
        _, d, _ = self.index.search(val_queries, given=seeds, stream=stream, **p)
        self.judge = self.mlp.confidence_threshold(d[:, 0].contiguous(), 1.0 - continue_fraction, stream=stream)
        return self.judge

    def seeds(self, queries, stream=None):
        s, pmax = self.mlp.predict(queries, P=self.P, tau=self.tau, stream=stream)
        return s, pmax

    def fallback_fraction(self, seeds) -> float:
        return float((seeds[:, 0] == np.int32(np.uint32(INVALID).view(np.int32))).float().mean().item())

    def close(self):
        self.mlp.close()
