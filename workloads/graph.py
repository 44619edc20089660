"""Proximity-graph construction (an input of the search) and the ghost sample.

The search method takes a fixed-degree proximity graph as given (Section 2.1
of the paper; it uses CAGRA's builder). This module builds such graphs for the
synthetic workloads with a documented recipe of its own:

1. a kNN list per node of length K, exact (all pairs) or restricted to the
   node's k-means partition plus its nearest neighboring partitions;
2. rank-based pruning by detour count: edge u->v at rank r is detourable via
   w (rank < r in u's list) when v sits in w's list at a rank < r; keep the
   deg/2 edges with the fewest detours (ties by rank), then fill with reverse
   edges (by rank), then with the remaining forward edges;
3. bridges: the last ``n_bridge`` slots of every list point to the nearest
   node of other k-means partitions (the two nearest partitions and seeded
   random ones). Strongly clustered synthetic data otherwise yields one graph
   component per cluster, which no search can cross.

PyTorch is used here as offline tooling (CPU for small inputs, the GPU for
the large ones). Nothing here is timed, and the graph is shared verbatim by
the CPU oracle and the CUDA search.
"""

from __future__ import annotations

import numpy as np
import torch

INVALID = 0xFFFFFFFF


def _dev(device):
    if device is None:
        return torch.device("cuda" if torch.cuda.is_available() else "cpu")
    return torch.device(device)


def _sqnorm(x: torch.Tensor) -> torch.Tensor:
    return (x * x).sum(dim=1)


def _topk_smallest(d2: torch.Tensor, k: int):
    vals, idx = torch.topk(d2, k, dim=1, largest=False, sorted=True)
    return vals, idx


def knn_exact(X: np.ndarray, K: int, device=None, chunk: int = 4096) -> np.ndarray:
    """Exact (FP32 expanded-form) kNN over all pairs, self excluded.
    Returns int64 n x K ids sorted by increasing distance."""
    dev = _dev(device)
    with torch.no_grad():
        Xt = torch.from_numpy(np.ascontiguousarray(X)).to(dev, torch.float32)
        n = Xt.shape[0]
        K = min(K, n - 1)
        xn = _sqnorm(Xt)
        out = torch.empty((n, K), dtype=torch.int64, device=dev)
        for s in range(0, n, chunk):
            e = min(n, s + chunk)
            d2 = xn[s:e, None] + xn[None, :] - 2.0 * (Xt[s:e] @ Xt.T)
            d2[torch.arange(e - s, device=dev), torch.arange(s, e, device=dev)] = float("inf")
            _, idx = _topk_smallest(d2, K)
            out[s:e] = idx
        return out.cpu().numpy()


def _kmeans(Xt: torch.Tensor, n_parts: int, seed: int, iters: int = 8, sample: int = 0):
    gen = torch.Generator(device="cpu").manual_seed(seed)
    n = Xt.shape[0]
    if sample and sample < n:
        sub = Xt[torch.randperm(n, generator=gen)[:sample].to(Xt.device)]
    else:
        sub = Xt
    cent = sub[torch.randperm(sub.shape[0], generator=gen)[:n_parts].to(Xt.device)].clone()

    def assign(P):
        cn = _sqnorm(cent)
        res = torch.empty(P.shape[0], dtype=torch.int64, device=P.device)
        for s in range(0, P.shape[0], 65536):
            e = min(P.shape[0], s + 65536)
            d2 = cn[None, :] - 2.0 * (P[s:e] @ cent.T)
            res[s:e] = d2.argmin(dim=1)
        return res

    for _ in range(iters):
        a = assign(sub)
        sums = torch.zeros_like(cent).index_add_(0, a, sub)
        cnt = torch.bincount(a, minlength=n_parts).to(sub.dtype)
        nz = cnt > 0
        cent[nz] = sums[nz] / cnt[nz, None]
    return cent, assign(Xt)


def knn_partitioned(X: np.ndarray, K: int, n_parts: int, n_near: int = 2, device=None,
                    seed: int = 0, query_chunk: int = 2048) -> np.ndarray:
    """kNN restricted to each node's k-means partition plus its ``n_near``
    nearest partitions (by centroid distance). Self excluded."""
    dev = _dev(device)
    with torch.no_grad():
        Xt = torch.from_numpy(np.ascontiguousarray(X)).to(dev, torch.float32)
        n = Xt.shape[0]
        cent, assign = _kmeans(Xt, n_parts, seed, sample=min(n, 200 * n_parts))
        order = torch.argsort(assign)
        counts = torch.bincount(assign, minlength=n_parts)
        starts = torch.zeros(n_parts + 1, dtype=torch.int64, device=dev)
        starts[1:] = torch.cumsum(counts, 0)
        cn = _sqnorm(cent)
        cd = cn[:, None] + cn[None, :] - 2.0 * (cent @ cent.T)
        cd.fill_diagonal_(float("inf"))
        # candidate partitions by centroid distance; a pool takes the n_near
        # nearest and then more until it holds at least K + 1 points (tiny
        # partitions of skewed cluster sizes would otherwise pad their lists)
        near = torch.topk(cd, min(max(n_near, 32), n_parts - 1), dim=1, largest=False).indices if n_parts > 1 \
            else torch.zeros((1, 0), dtype=torch.int64, device=dev)
        xn = _sqnorm(Xt)
        out = torch.full((n, K), -1, dtype=torch.int64, device=dev)
        starts_h = starts.cpu().tolist()
        near_h = near.cpu().tolist()
        for p in range(n_parts):
            a, b = starts_h[p], starts_h[p + 1]
            if a == b:
                continue
            members = order[a:b]
            pool, size = [members], b - a
            for i, q in enumerate(near_h[p]):
                if i >= n_near and size >= K + 1:
                    break
                pool.append(order[starts_h[q]:starts_h[q + 1]])
                size += starts_h[q + 1] - starts_h[q]
            pool = torch.cat(pool)
            kk = min(K, pool.shape[0] - 1)
            P = Xt[pool]
            pn = xn[pool]
            for s in range(0, members.shape[0], query_chunk):
                e = min(members.shape[0], s + query_chunk)
                m = members[s:e]
                d2 = xn[m, None] + pn[None, :] - 2.0 * (Xt[m] @ P.T)
                d2[torch.arange(e - s, device=dev), torch.arange(s, e, device=dev)] = float("inf")
                _, idx = _topk_smallest(d2, kk)
                out[m, :kk] = pool[idx]
        # Rows shorter than K (tiny pools) are padded by repeating the last
        # neighbour; pruning deduplicates them away.
        bad = out < 0
        if bad.any():
            last = out[:, :1].expand_as(out)
            out = torch.where(bad, last, out)
        return out.cpu().numpy()


def prune_by_detours(knn: np.ndarray, degree: int, device=None, chunk: int = 2048) -> np.ndarray:
    """Rank-based detour pruning of kNN lists to a fixed out-degree.
    Returns uint32 n x degree."""
    dev = _dev(device)
    with torch.no_grad():
        N_all = torch.from_numpy(np.ascontiguousarray(knn)).to(dev, torch.int64)
        n, K = N_all.shape
        assert K >= degree, "kNN list shorter than the target degree"
        half = degree // 2
        a_idx = torch.arange(K, device=dev).repeat_interleave(K)
        c_idx = torch.arange(K, device=dev).repeat(K)
        ordered = torch.empty((n, K), dtype=torch.int64, device=dev)
        for s in range(0, n, chunk):
            e = min(n, s + chunk)
            N = N_all[s:e]
            B = e - s
            M = N_all[N.reshape(-1)].reshape(B, K * K)
            Ns, perm = N.sort(dim=1)
            pos = torch.searchsorted(Ns, M).clamp_(max=K - 1)
            found = Ns.gather(1, pos) == M
            rank = perm.gather(1, pos)
            ok = found & (a_idx[None, :] < rank) & (c_idx[None, :] < rank)
            det = torch.zeros((B, K), dtype=torch.int64, device=dev)
            det.scatter_add_(1, torch.where(ok, rank, torch.zeros_like(rank)), ok.to(torch.int64))
            key = det * K + torch.arange(K, device=dev)[None, :]
            ordered[s:e] = N.gather(1, torch.argsort(key, dim=1))
        fwd = ordered[:, :half]
        # reverse edges of the kept forward edges, ranked by the forward rank
        nr = degree - half
        src = torch.arange(n, device=dev).repeat_interleave(half)
        tgt = fwd.reshape(-1)
        rnk = torch.arange(half, device=dev).repeat(n)
        key = (tgt * K + rnk) * n + src
        o = torch.argsort(key)
        tgt_s, src_s = tgt[o], src[o]
        first = torch.ones_like(tgt_s, dtype=torch.bool)
        first[1:] = tgt_s[1:] != tgt_s[:-1]
        grp_start = torch.cummax(torch.where(first, torch.arange(tgt_s.shape[0], device=dev),
                                             torch.zeros_like(tgt_s)), 0).values
        slot = torch.arange(tgt_s.shape[0], device=dev) - grp_start
        keep = slot < nr
        rev = torch.full((n, nr), -1, dtype=torch.int64, device=dev)
        rev[tgt_s[keep], slot[keep]] = src_s[keep]
        cand = torch.cat([fwd, rev, ordered[:, half:]], dim=1)
        L = cand.shape[1]
        graph = torch.empty((n, degree), dtype=torch.int64, device=dev)
        posn = torch.arange(L, device=dev)
        for s in range(0, n, 65536):
            e = min(n, s + 65536)
            c = cand[s:e]
            vs, vi = torch.sort(c, dim=1, stable=True)
            dup = torch.zeros_like(vs, dtype=torch.bool)
            dup[:, 1:] = vs[:, 1:] == vs[:, :-1]
            selfloop = vs == torch.arange(s, e, device=dev)[:, None]
            removed = torch.zeros_like(dup)
            removed.scatter_(1, vi, dup | (vs < 0) | selfloop)
            k2 = removed.to(torch.int64) * L + posn[None, :]
            sel = torch.argsort(k2, dim=1)[:, :degree]
            g = c.gather(1, sel)
            nrem = (~removed).sum(dim=1)
            assert bool((nrem >= degree).all()), "not enough distinct neighbours to fill the degree"
            graph[s:e] = g
        return graph.cpu().numpy().astype(np.uint32)


def bridges(X: np.ndarray, n_parts: int, n_near: int = 2, n_random: int = 2, device=None,
            seed: int = 0, query_chunk: int = 4096) -> np.ndarray:
    """For every node: the nearest node in each of the ``n_near`` partitions
    nearest to its own k-means partition (by centroid distance), then
    ``n_random`` uniformly random nodes (seeded). Returns int64
    n x (n_near + n_random), -1 where a slot has no target."""
    dev = _dev(device)
    with torch.no_grad():
        Xt = torch.from_numpy(np.ascontiguousarray(X)).to(dev, torch.float32)
        n = Xt.shape[0]
        out = torch.full((n, n_near + n_random), -1, dtype=torch.int64, device=dev)
        if n_parts >= 2 and n_near > 0:
            cent, assign = _kmeans(Xt, n_parts, seed + 17, sample=min(n, 200 * n_parts))
            order = torch.argsort(assign)
            counts = torch.bincount(assign, minlength=n_parts)
            starts = torch.zeros(n_parts + 1, dtype=torch.int64, device=dev)
            starts[1:] = torch.cumsum(counts, 0)
            cn = _sqnorm(cent)
            cd = cn[:, None] + cn[None, :] - 2.0 * (cent @ cent.T)
            cd.fill_diagonal_(float("inf"))
            cd[:, counts == 0] = float("inf")
            near = torch.topk(cd, min(n_near, n_parts - 1), dim=1, largest=False).indices.cpu().tolist()
            xn = _sqnorm(Xt)
            starts_h = starts.cpu().tolist()
            for p in range(n_parts):
                a, b = starts_h[p], starts_h[p + 1]
                if a == b:
                    continue
                members = order[a:b]
                for slot, q in enumerate(near[p]):
                    pool = order[starts_h[q]:starts_h[q + 1]]
                    if pool.numel() == 0:
                        continue
                    P = Xt[pool]
                    pn = xn[pool]
                    for s in range(0, members.shape[0], query_chunk):
                        e = min(members.shape[0], s + query_chunk)
                        m = members[s:e]
                        out[m, slot] = pool[(pn[None, :] - 2.0 * (Xt[m] @ P.T)).argmin(dim=1)]
        res = out.cpu().numpy()
    if n_random > 0:
        rng = np.random.Generator(np.random.PCG64(seed + 29))
        r = rng.integers(0, n - 1, size=(n, n_random))
        r += r >= np.arange(n)[:, None]          # skip self
        res[:, n_near:] = r
    return res


def add_bridges(graph: np.ndarray, br: np.ndarray) -> np.ndarray:
    """Put the bridge targets in the last slots of each list (skipping
    targets already present and self); the displaced tail edges are the
    lowest-priority ones of the pruned order."""
    g = graph.astype(np.int64).copy()
    n, deg = g.shape
    nb = br.shape[1]
    if nb == 0:
        return graph
    for j in range(nb):
        slot = deg - nb + j
        t = br[:, j]
        present = (g[:, :slot] == t[:, None]).any(axis=1) | (t < 0) | (t == np.arange(n))
        g[~present, slot] = t[~present]
    # a bridge may duplicate an edge in a later bridge slot: rebuild such rows
    # from first occurrences, refilled from the pruned list
    out = g.copy()
    srt = np.sort(g, axis=1)
    orig = graph.astype(np.int64)
    for i in np.nonzero((srt[:, 1:] == srt[:, :-1]).any(axis=1))[0]:
        seen, row = set(), []
        for v in list(g[i]) + list(orig[i]):
            if v not in seen and v != i:
                seen.add(v)
                row.append(v)
            if len(row) == deg:
                break
        out[i] = row
    return out.astype(np.uint32)


def build_graph(X: np.ndarray, degree: int, knn_k: int, method: str = "exact",
                n_parts: int = 0, device=None, seed: int = 0, n_bridge: int = -1, n_near: int = 2,
                part_size: int = 1000) -> np.ndarray:
    """kNN lists of length ``knn_k`` (exact, or partitioned over each node's
    partition, of about ``part_size`` points, and its ``n_near`` nearest
    ones) pruned to ``degree``, with ``n_bridge`` bridge slots (default
    degree // 8; half to the nearest partitions, half to random ones)."""
    n = X.shape[0]
    parts = n_parts or max(1, n // part_size)
    if method == "exact" or n <= 20_000:
        knn = knn_exact(X, knn_k, device=device)
    else:
        knn = knn_partitioned(X, knn_k, parts, n_near=n_near, device=device, seed=seed)
    g = prune_by_detours(knn, degree, device=device)
    nb = degree // 8 if n_bridge < 0 else n_bridge
    if nb > 0 and n > 2 * degree:
        bparts = n_parts or max(2, n // 200 if n <= 20_000 else n // 1000)
        br = bridges(X, bparts, n_near=nb - nb // 2, n_random=nb // 2, device=device, seed=seed)
        g = add_bridges(g, br)
    return g


def ghost_sample(n: int, m: int, seed: int) -> np.ndarray:
    """A uniform sample of ``m`` distinct node ids (without replacement),
    returned in ascending order as uint32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ids = rng.choice(n, size=m, replace=False)
    return np.sort(ids).astype(np.uint32)
