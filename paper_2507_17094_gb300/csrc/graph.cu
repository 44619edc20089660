// Graph construction on the GPU (the build the paper times in Section 5.7,
// Fig. 16; the graph itself is an input of the search, Section 2.1):
//
//   ann_knn_exact   the K nearest other nodes of every node, by brute force:
//                   a block keeps 32 query rows and streams the candidates
//                   through shared memory in tiles of 64 rows; a warp owns 4
//                   queries and keeps each one's sorted (distance, id) list
//                   in shared memory, inserting the few tile candidates that
//                   beat its current K-th entry;
//   ann_graph_prune the detour-count pruning with reverse edges: one warp per
//                   node counts detours with a sorted (id, rank) table of its
//                   list in shared memory and orders the list by (detours,
//                   rank); the kept edges' reverse offers are bucketed by
//                   target (count, scan, scatter) and each target takes its
//                   smallest (position, source) offers; one warp per node
//                   assembles the row (kept, reverse, rest; repeats and the
//                   node itself dropped).
//
// Distances are squared L2 in FP32, one fused multiply-add per element in
// index order (the kNN lists rank by (distance, id)).
#include <algorithm>
#include <vector>

#include "ann_internal.cuh"

using namespace ann;

namespace {

constexpr int KQ = 32;          // query rows per block
constexpr int KC = 64;          // candidate rows per shared-memory tile
constexpr int KW = 8;           // warps per block (4 queries each)

__device__ __forceinline__ bool kless(float da, uint32_t ia, float db, uint32_t ib)
{
    return da < db || (da == db && ia < ib);
}

// Insert (d, id) into a warp's sorted list lst_d/lst_i of K entries if it
// beats the last one (all lanes call it with the same arguments).
__device__ __forceinline__ void list_insert(float *lst_d, uint32_t *lst_i, uint32_t K, float d, uint32_t id,
                                            uint32_t lane)
{
    if (!kless(d, id, lst_d[K - 1], lst_i[K - 1])) return;
    uint32_t pos = 0;
    for (uint32_t j = lane; j < K; j += 32) pos += kless(lst_d[j], lst_i[j], d, id) ? 1u : 0u;
    pos = __reduce_add_sync(0xffffffffu, pos);
    // shift [pos, K - 1) right by one, from the top (each lane one entry
    // per pass, read before any write of the pass)
    for (int32_t top = (int32_t)K - 2; top >= (int32_t)pos; top -= 32) {
        const int32_t j = top - (int32_t)lane;
        float vd = 0.0f;
        uint32_t vi = 0;
        const bool mine = j >= (int32_t)pos;
        if (mine) { vd = lst_d[j]; vi = lst_i[j]; }
        __syncwarp();
        if (mine) { lst_d[j + 1] = vd; lst_i[j + 1] = vi; }
        __syncwarp();
    }
    if (lane == 0) { lst_d[pos] = d; lst_i[pos] = id; }
    __syncwarp();
}

// Exact kNN: block b handles query rows [32 b, 32 b + 32); dynamic shared
// memory holds the 32 query rows, one tile of KC candidate rows (row stride
// d + 1 floats: lanes reading one element of 32 different rows hit 32
// banks) and the 32 lists of K entries.
__global__ void __launch_bounds__(KW * 32) knn_exact_kernel(const float *__restrict__ X, uint32_t n, uint32_t d,
                                                            uint32_t K, uint32_t *__restrict__ out)
{
    extern __shared__ __align__(16) uint8_t sm[];
    const uint32_t ds = d + 1;
    float *sq = reinterpret_cast<float *>(sm);                 // KQ x ds
    float *sc = sq + KQ * ds;                                  // KC x ds
    float *ld = sc + KC * ds;                                  // KQ x K
    uint32_t *li = reinterpret_cast<uint32_t *>(ld + KQ * K);  // KQ x K
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t q0 = blockIdx.x * KQ;
    for (uint32_t i = threadIdx.x; i < KQ * d; i += blockDim.x) {
        const uint32_t r = i / d, c = i % d;
        sq[r * ds + c] = q0 + r < n ? X[(size_t)(q0 + r) * d + c] : 0.0f;
    }
    for (uint32_t i = threadIdx.x; i < KQ * K; i += blockDim.x) {
        ld[i] = INFINITY;
        li[i] = ANN_INVALID_ID;
    }
    for (uint32_t c0 = 0; c0 < n; c0 += KC) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < KC * d; i += blockDim.x) {
            const uint32_t r = i / d, c = i % d;
            sc[r * ds + c] = c0 + r < n ? X[(size_t)(c0 + r) * d + c] : 0.0f;
        }
        __syncthreads();
        // this warp's 4 queries x the tile's 64 candidates: lane owns
        // candidates lane and lane + 32
        float acc[4][2];
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = 0.0f;
        const float *x0 = sc + lane * ds, *x1 = sc + (lane + 32) * ds;
        const float *qw = sq + (warp * 4) * ds;
#pragma unroll 2
        for (uint32_t i = 0; i < d; ++i) {
            const float xa = x0[i], xb = x1[i];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float qv = qw[a * ds + i];
                const float da = __fsub_rn(qv, xa), db = __fsub_rn(qv, xb);
                acc[a][0] = __fmaf_rn(da, da, acc[a][0]);
                acc[a][1] = __fmaf_rn(db, db, acc[a][1]);
            }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const uint32_t qi = q0 + warp * 4 + a;
            float *lda = ld + (warp * 4 + a) * K;
            uint32_t *lia = li + (warp * 4 + a) * K;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t cid = c0 + lane + 32 * h;
                const bool cand = qi < n && cid < n && cid != qi;
                const float dv = acc[a][h];
                uint32_t m = __ballot_sync(0xffffffffu, cand && kless(dv, cid, lda[K - 1], lia[K - 1]));
                while (m) {
                    const uint32_t src = __ffs(m) - 1;
                    m &= m - 1;
                    list_insert(lda, lia, K, __shfl_sync(0xffffffffu, dv, src),
                                __shfl_sync(0xffffffffu, cid, src), lane);
                }
            }
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < KQ * K; i += blockDim.x) {
        const uint32_t r = i / K;
        if (q0 + r < n) out[(size_t)(q0 + r) * K + (i % K)] = li[i];
    }
}

// ------------------------------------------------------------ pruning
// Detour counts and the (detours, rank) order of node u's list: warp per
// node, dynamic shared memory per warp: ids sorted by (id, rank) with their
// ranks (K x 8 bytes) and the counts (K x 4).
__global__ void detour_order_kernel(const uint32_t *__restrict__ knn, uint32_t n, uint32_t K,
                                    uint32_t *__restrict__ ordered)
{
    extern __shared__ __align__(16) uint8_t sm[];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t u = blockIdx.x * (blockDim.x >> 5) + warp;
    uint32_t *sid = reinterpret_cast<uint32_t *>(sm) + warp * 3 * K;   // sorted ids
    uint32_t *srk = sid + K;                                            // their ranks
    uint32_t *det = srk + K;
    if (u >= n) return;
    const uint32_t *N = knn + (size_t)u * K;
    // sort (id, rank) by rank counting (K <= ANN_MAX_DEGREE * 2)
    for (uint32_t r = lane; r < K; r += 32) {
        const uint32_t v = N[r];
        uint32_t pos = 0;
        for (uint32_t r2 = 0; r2 < K; ++r2) {
            const uint32_t w = N[r2];
            pos += (w < v || (w == v && r2 < r)) ? 1u : 0u;
        }
        sid[pos] = v;
        srk[pos] = r;
        det[r] = 0;
    }
    __syncwarp();
    for (uint32_t a = 0; a < K; ++a) {
        const uint32_t w = N[a];
        if (w == ANN_INVALID_ID || w >= n) continue;
        for (uint32_t c = lane; c < K; c += 32) {
            const uint32_t x = knn[(size_t)w * K + c];
            // lower bound of x among the sorted ids: its smallest rank
            uint32_t lo = 0, hi = K;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (sid[mid] < x) lo = mid + 1;
                else hi = mid;
            }
            if (lo < K && sid[lo] == x && x != ANN_INVALID_ID) {
                const uint32_t r = srk[lo];
                if (a < r && c < r) atomicAdd(&det[r], 1u);
            }
        }
    }
    __syncwarp();
    for (uint32_t r = lane; r < K; r += 32) {
        const uint32_t dr = det[r];
        uint32_t pos = 0;
        for (uint32_t r2 = 0; r2 < K; ++r2) {
            const uint32_t d2 = det[r2];
            pos += (d2 < dr || (d2 == dr && r2 < r)) ? 1u : 0u;
        }
        ordered[(size_t)u * K + pos] = N[r];
    }
}

// Reverse offers of the kept edges: count per target.
__global__ void offer_count_kernel(const uint32_t *__restrict__ ordered, uint32_t n, uint32_t K, uint32_t half,
                                   uint32_t *__restrict__ cnt)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= (uint64_t)n * half) return;
    const uint32_t w = (uint32_t)(i / half), p = (uint32_t)(i % half);
    const uint32_t v = ordered[(size_t)w * K + p];
    if (v < n) atomicAdd(&cnt[v], 1u);
}

// Exclusive scan of `cnt` (n) into off (n + 1): per-block scans, then a scan
// of the block sums (one block, looping), then the block offsets added.
__global__ void scan_block_kernel(const uint32_t *__restrict__ in, uint32_t n, uint32_t *__restrict__ out,
                                  uint32_t *__restrict__ block_sums)
{
    __shared__ uint32_t wsum[32];
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t v = i < n ? in[i] : 0u;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < (blockDim.x >> 5) ? wsum[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= (uint32_t)o) s += y;
        }
        wsum[lane] = s;
    }
    __syncthreads();
    const uint32_t incl = x + (warp ? wsum[warp - 1] : 0u);
    if (i < n) out[i] = incl - v;
    if (threadIdx.x == blockDim.x - 1) block_sums[blockIdx.x] = incl;
}

__global__ void scan_sums_kernel(uint32_t *__restrict__ sums, uint32_t nb, uint32_t *__restrict__ total)
{
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (uint32_t b = 0; b < nb; ++b) {
            const uint32_t v = sums[b];
            sums[b] = s;
            s += v;
        }
        *total = s;
    }
}

__global__ void scan_add_kernel(uint32_t *__restrict__ out, uint32_t n, const uint32_t *__restrict__ sums)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += sums[blockIdx.x];
}

// Offers bucketed by target: key (position p in the source's kept list,
// source w) as one 64-bit word (p high), at an atomically claimed slot.
__global__ void offer_scatter_kernel(const uint32_t *__restrict__ ordered, uint32_t n, uint32_t K, uint32_t half,
                                     const uint32_t *__restrict__ off, uint32_t *__restrict__ cursor,
                                     uint64_t *__restrict__ keys)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= (uint64_t)n * half) return;
    const uint32_t w = (uint32_t)(i / half), p = (uint32_t)(i % half);
    const uint32_t v = ordered[(size_t)w * K + p];
    if (v < n) keys[off[v] + atomicAdd(&cursor[v], 1u)] = ((uint64_t)p << 32) | w;
}

// Row assembly, warp per node v: its nr smallest offers (repeated warp
// minima over its bucket), then kept ++ reverse ++ rest with repeats and v
// dropped, first `degree` entries (INVALID-padded).
__global__ void assemble_kernel(const uint32_t *__restrict__ ordered, uint32_t n, uint32_t K, uint32_t half,
                                uint32_t degree, const uint32_t *__restrict__ off, const uint64_t *__restrict__ keys,
                                uint32_t *__restrict__ graph)
{
    extern __shared__ __align__(16) uint8_t sm[];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t v = blockIdx.x * (blockDim.x >> 5) + warp;
    const uint32_t L = K + (degree - half);
    uint32_t *cand = reinterpret_cast<uint32_t *>(sm) + warp * L;
    if (v >= n) return;
    const uint32_t nr = degree - half;
    for (uint32_t j = lane; j < half; j += 32) cand[j] = ordered[(size_t)v * K + j];
    const uint64_t *kv = keys + off[v];
    const uint32_t nk = off[v + 1] - off[v];
    uint64_t last = 0;
    bool have_last = false;
    uint32_t taken = 0;
    for (; taken < nr; ++taken) {
        uint64_t best = ~0ull;
        for (uint32_t j = lane; j < nk; j += 32) {
            const uint64_t k = kv[j];
            if ((!have_last || k > last) && k < best) best = k;
        }
        for (int o = 16; o; o >>= 1) {
            const uint64_t other = __shfl_xor_sync(0xffffffffu, best, o);
            best = other < best ? other : best;
        }
        if (best == ~0ull) break;
        if (lane == 0) cand[half + taken] = (uint32_t)best;
        last = best;
        have_last = true;
    }
    const uint32_t nrev = taken;
    for (uint32_t j = lane; j < K - half; j += 32) cand[half + nrev + j] = ordered[(size_t)v * K + half + j];
    __syncwarp();
    const uint32_t total = half + nrev + (K - half);
    uint32_t written = 0;
    for (uint32_t b = 0; b < total && written < degree; b += 32) {
        const uint32_t j = b + lane;
        bool keep = false;
        uint32_t x = ANN_INVALID_ID;
        if (j < total) {
            x = cand[j];
            keep = x < n && x != v;
            for (uint32_t t = 0; t < j && keep; ++t) keep = cand[t] != x;
        }
        const uint32_t m = __ballot_sync(0xffffffffu, keep);
        const uint32_t at = written + __popc(m & ((1u << lane) - 1u));
        if (keep && at < degree) graph[(size_t)v * degree + at] = x;
        written += __popc(m);
    }
    for (uint32_t j = written + lane; j < degree; j += 32) graph[(size_t)v * degree + j] = ANN_INVALID_ID;
}

int grid_for(uint64_t n, int threads) { return (int)std::max<uint64_t>(1, (n + threads - 1) / threads); }

}  // namespace

extern "C" {

ann_status ann_knn_exact(const float *X, uint64_t n, uint32_t dim, uint32_t K, uint32_t *ids, void *stream)
{
    if (!X || !ids || n < 2 || n > 0xFFFFFFFEull || dim == 0 || dim > ANN_MAX_DIM || K == 0 || K >= n ||
        K > 2 * ANN_MAX_DEGREE) {
        set_error("ann_knn_exact: need 2 <= n < 2^32 - 1, 1 <= dim <= %u, 1 <= K < n, K <= %u", ANN_MAX_DIM,
                  2 * ANN_MAX_DEGREE);
        return ANN_EINVAL;
    }
    const size_t smem = (size_t)(KQ + KC) * (dim + 1) * 4 + (size_t)KQ * K * 8;
    int dev = 0, optin = 0;
    ANN_CUDA(cudaGetDevice(&dev));
    ANN_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (smem > (size_t)optin) {
        set_error("ann_knn_exact: %zu bytes of shared memory needed (dim %u, K %u), %d available", smem, dim, K, optin);
        return ANN_EINVAL;
    }
    ANN_CUDA(cudaFuncSetAttribute(knn_exact_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    knn_exact_kernel<<<grid_for(n, KQ), KW * 32, smem, (cudaStream_t)stream>>>(X, (uint32_t)n, dim, K, ids);
    ANN_CUDA(cudaGetLastError());
    return ANN_OK;
}

ann_status ann_graph_prune(const uint32_t *knn, uint64_t n, uint32_t K, uint32_t degree, uint32_t *graph,
                           void *stream)
{
    if (!knn || !graph || n == 0 || n > 0xFFFFFFFEull || K == 0 || K > 2 * ANN_MAX_DEGREE || degree == 0 ||
        degree > K || degree > ANN_MAX_DEGREE) {
        set_error("ann_graph_prune: need n >= 1, 1 <= degree <= min(K, %u), K <= %u", ANN_MAX_DEGREE,
                  2 * ANN_MAX_DEGREE);
        return ANN_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t nn = (uint32_t)n, half = degree / 2;
    const uint32_t nb = (nn + 1023) / 1024;
    uint32_t *ordered = nullptr, *cnt = nullptr, *off = nullptr, *sums = nullptr, *cursor = nullptr;
    uint64_t *keys = nullptr;
    cudaError_t e = cudaMalloc(&ordered, (size_t)n * K * 4);
    if (e == cudaSuccess) e = cudaMalloc(&cnt, (size_t)n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&off, (size_t)(n + 1) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&sums, (size_t)nb * 4);
    if (e == cudaSuccess) e = cudaMalloc(&cursor, (size_t)n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&keys, (size_t)n * std::max(1u, half) * 8);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, (size_t)n * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, (size_t)n * 4, st);
    if (e == cudaSuccess) {
        const int wpb = 8;
        detour_order_kernel<<<grid_for(n, wpb), wpb * 32, (size_t)wpb * 3 * K * 4, st>>>(knn, nn, K, ordered);
        offer_count_kernel<<<grid_for((uint64_t)n * half, 256), 256, 0, st>>>(ordered, nn, K, half, cnt);
        scan_block_kernel<<<nb, 1024, 0, st>>>(cnt, nn, off, sums);
        scan_sums_kernel<<<1, 32, 0, st>>>(sums, nb, off + nn);
        scan_add_kernel<<<nb, 1024, 0, st>>>(off, nn, sums);
        offer_scatter_kernel<<<grid_for((uint64_t)n * half, 256), 256, 0, st>>>(ordered, nn, K, half, off, cursor,
                                                                                keys);
        const uint32_t L = K + (degree - half);
        assemble_kernel<<<grid_for(n, wpb), wpb * 32, (size_t)wpb * L * 4, st>>>(ordered, nn, K, half, degree, off,
                                                                               keys, graph);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    cudaFree(ordered);
    cudaFree(cnt);
    cudaFree(off);
    cudaFree(sums);
    cudaFree(cursor);
    cudaFree(keys);
    return e == cudaSuccess ? ANN_OK : cuda_fail(e, "ann_graph_prune");
}

}  // extern "C"
