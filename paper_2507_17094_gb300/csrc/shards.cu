// Pipelining-based path extension (Section 3.1.2, Eq. 3, Section 4) on one
// GPU: the shards are separate indexes in the same device memory, and what
// the paper sends from one GPU to the next is a device-local array here.
//
//   - links (Eq. 3): I(u) for every node u of shard i is the top-1 result of
//     searching shard (i + 1) mod N with u's FP32 vector as the query
//     (Section 4's construction), computed by the library's own search in
//     chunks of at most kLinkChunk nodes;
//   - search: the queries are split into N chunks; chunk c runs on its own
//     stream and visits shards c, c + 1, ... (mod N); between stages a small
//     kernel turns the best n_forward nodes z of the chunk's local result
//     into seeds I(z) of the next shard (entry ANN_ENTRY_GIVEN_BASE); the
//     stages of different chunks overlap on the GPU whenever they touch
//     different shards (a shard's own launches are ordered by its index);
//   - reduction: one thread per query merges the N sorted local lists, as
//     dataset ids, into the top k by (distance, id) (the paper does this on
//     the CPU).
#include <algorithm>
#include <vector>

#include "ann_internal.cuh"

using namespace ann;

namespace {

constexpr uint32_t kLinkChunk = 1u << 20;   // link queries per launch

struct GidTables {
    const uint32_t *g[ANN_MAX_SHARDS];
};

// seeds[r * F + j] = links[z] for the best F nodes z of row r's local result
// (ANN_INVALID_ID passes through).
__global__ void forward_kernel(const uint32_t *__restrict__ loc, uint32_t k, uint32_t rows, uint32_t F,
                               const uint32_t *__restrict__ links, uint64_t n_from, uint32_t *__restrict__ seeds)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= (uint64_t)rows * F) return;
    const uint64_t r = i / F, j = i % F;
    const uint32_t z = loc[r * k + j];
    seeds[i] = (z == ANN_INVALID_ID || z >= n_from) ? ANN_INVALID_ID : links[z];
}

// Query q of chunk c: stage t's list lies at loc + (t * nq + q) * k and holds
// local ids of shard (c + t) mod N, sorted by (distance, local id) -- the
// same order as by (distance, dataset id), since a shard's dataset ids
// ascend with its local ids. The N lists are merged head by head.
__global__ void reduce_kernel(const uint32_t *__restrict__ loc_ids, const float *__restrict__ loc_d, uint32_t nq,
                              uint32_t N, uint32_t k, GidTables gt, uint32_t *__restrict__ ids,
                              float *__restrict__ dists)
{
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    uint32_t c = 0;
    while (c + 1 < N && (uint64_t)(c + 1) * nq / N <= q) ++c;
    uint32_t head[ANN_MAX_SHARDS];
    for (uint32_t t = 0; t < N; ++t) head[t] = 0;
    for (uint32_t j = 0; j < k; ++j) {
        float bd = INFINITY;
        uint32_t bg = ANN_INVALID_ID, bt = N;
        for (uint32_t t = 0; t < N; ++t) {
            if (head[t] >= k) continue;
            const uint64_t at = ((uint64_t)t * nq + q) * k + head[t];
            const uint32_t li = loc_ids[at];
            if (li == ANN_INVALID_ID) continue;
            const float d = loc_d[at];
            const uint32_t g = gt.g[(c + t) % N][li];
            if (bt == N || d < bd || (d == bd && g < bg)) { bd = d; bg = g; bt = t; }
        }
        if (bt < N) ++head[bt];
        ids[(uint64_t)q * k + j] = bg;
        dists[(uint64_t)q * k + j] = bd;
    }
}

int grid_for(uint64_t n, int threads) { return (int)std::max<uint64_t>(1, (n + threads - 1) / threads); }

}  // namespace

struct ann_shards {
    int device = 0;
    uint32_t N = 0, dim = 0;
    std::vector<ann_index *> ix;
    std::vector<uint64_t> n;
    std::vector<uint32_t *> gids;    // device, n_i dataset ids of shard i
    std::vector<uint32_t *> links;   // device, n_i local ids in shard i + 1 (null until linked)
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    cudaEvent_t start = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
};

namespace {

void shards_release(ann_shards *s)
{
    for (auto p : s->gids) if (p) cudaFree(p);
    for (auto p : s->links) if (p) cudaFree(p);
    for (auto st : s->streams) if (st) cudaStreamDestroy(st);
    for (auto e : s->done) if (e) cudaEventDestroy(e);
    if (s->start) cudaEventDestroy(s->start);
    if (s->ws) cudaFree(s->ws);
}

ann_status grow_ws(ann_shards *s, size_t bytes, cudaStream_t st)
{
    if (bytes <= s->ws_bytes) return ANN_OK;
    if (s->ws) {
        ANN_CUDA(cudaStreamSynchronize(st));
        for (auto c : s->streams) ANN_CUDA(cudaStreamSynchronize(c));
        cudaFree(s->ws);
        s->ws = nullptr;
        s->ws_bytes = 0;
    }
    ANN_CUDA(cudaMalloc(&s->ws, bytes));
    s->ws_bytes = bytes;
    return ANN_OK;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" {

ann_status ann_shards_create(ann_index *const *shards, uint32_t n_shards, const uint32_t *const *global_ids,
                             ann_shards **out)
{
    if (!out) { set_error("ann_shards_create: out is NULL"); return ANN_EINVAL; }
    *out = nullptr;
    if (!shards || !global_ids || n_shards == 0 || n_shards > ANN_MAX_SHARDS) {
        set_error("ann_shards_create: need 1..%u shards and their global ids", ANN_MAX_SHARDS);
        return ANN_EINVAL;
    }
    for (uint32_t i = 0; i < n_shards; ++i) {
        if (!shards[i] || !global_ids[i]) { set_error("ann_shards_create: NULL shard %u", i); return ANN_EINVAL; }
        if (shards[i]->device != shards[0]->device || shards[i]->dim != shards[0]->dim ||
            shards[i]->storage != shards[0]->storage) {
            set_error("ann_shards_create: shards differ in device, dimension or storage");
            return ANN_EINVAL;
        }
    }
    int prev = -1;
    ann_status s = enter_device(shards[0]->device, &prev, "ann_shards_create");
    if (s != ANN_OK) return s;
    ann_shards *h = new ann_shards();
    h->device = shards[0]->device;
    h->N = n_shards;
    h->dim = shards[0]->dim;
    cudaError_t e = cudaSuccess;
    for (uint32_t i = 0; i < n_shards && e == cudaSuccess; ++i) {
        h->ix.push_back(shards[i]);
        h->n.push_back(shards[i]->n);
        uint32_t *g = nullptr;
        e = cudaMalloc(&g, shards[i]->n * 4);
        h->gids.push_back(g);
        h->links.push_back(nullptr);
        if (e == cudaSuccess) e = cudaMemcpy(g, global_ids[i], shards[i]->n * 4, cudaMemcpyHostToDevice);
        cudaStream_t st = nullptr;
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        h->streams.push_back(st);
        cudaEvent_t ev = nullptr;
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        h->done.push_back(ev);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->start, cudaEventDisableTiming);
    leave_device(h->device, prev);
    if (e != cudaSuccess) {
        shards_release(h);
        delete h;
        return cuda_fail(e, "ann_shards_create");
    }
    *out = h;
    return ANN_OK;
}

ann_status ann_shards_free(ann_shards *s)
{
    if (!s) return ANN_OK;
    int prev = -1;
    const bool switched = enter_device(s->device, &prev, "ann_shards_free") == ANN_OK;   // frees best-effort
    for (auto st : s->streams) if (st) cudaStreamSynchronize(st);
    shards_release(s);
    if (switched) leave_device(s->device, prev);
    delete s;
    return ANN_OK;
}

ann_status ann_shards_set_links(ann_shards *s, uint32_t shard, const uint32_t *links)
{
    if (!s || !links || shard >= s->N) { set_error("ann_shards_set_links: bad arguments"); return ANN_EINVAL; }
    const uint64_t n_next = s->n[(shard + 1) % s->N];
    for (uint64_t i = 0; i < s->n[shard]; ++i)
        if (links[i] >= n_next) {
            set_error("ann_shards_set_links: link %llu of shard %u is %u, beyond the next shard's %llu nodes",
                      (unsigned long long)i, shard, links[i], (unsigned long long)n_next);
            return ANN_EINVAL;
        }
    int prev = -1;
    ann_status st = enter_device(s->device, &prev, "ann_shards_set_links");
    if (st != ANN_OK) return st;
    cudaError_t e = cudaSuccess;
    if (!s->links[shard]) e = cudaMalloc(&s->links[shard], s->n[shard] * 4);
    if (e == cudaSuccess) e = cudaMemcpy(s->links[shard], links, s->n[shard] * 4, cudaMemcpyHostToDevice);
    leave_device(s->device, prev);
    return e == cudaSuccess ? ANN_OK : cuda_fail(e, "ann_shards_set_links");
}

ann_status ann_shards_get_links(const ann_shards *s, uint32_t shard, uint32_t *links)
{
    if (!s || !links || shard >= s->N || !s->links[shard]) {
        set_error("ann_shards_get_links: bad arguments or shard not linked");
        return ANN_EINVAL;
    }
    int prev = -1;
    ann_status st = enter_device(s->device, &prev, "ann_shards_get_links");
    if (st != ANN_OK) return st;
    cudaError_t e = cudaMemcpy(links, s->links[shard], s->n[shard] * 4, cudaMemcpyDeviceToHost);
    leave_device(s->device, prev);
    return e == cudaSuccess ? ANN_OK : cuda_fail(e, "ann_shards_get_links");
}

ann_status ann_shards_link(ann_shards *s, const ann_search_params *p, void *stream)
{
    if (!s || !p) { set_error("ann_shards_link: NULL argument"); return ANN_EINVAL; }
    if (p->entry > ANN_ENTRY_GHOST) {
        set_error("ann_shards_link: entry %u is not available for link searches (random or ghost only)", p->entry);
        return ANN_EINVAL;
    }
    int prev = -1;
    ann_status st = enter_device(s->device, &prev, "ann_shards_link");
    if (st != ANN_OK) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    const uint32_t d = s->dim;
    uint64_t most = 0;
    for (uint32_t i = 0; i < s->N; ++i) most = std::max(most, std::min<uint64_t>(s->n[i], kLinkChunk));
    // dense FP32 query copy + distances of one chunk
    st = grow_ws(s, up256(most * d * 4) + up256(most * 4), cs);
    for (uint32_t i = 0; i < s->N && st == ANN_OK; ++i) {
        ann_index *src = s->ix[i], *nxt = s->ix[(i + 1) % s->N];
        const void *x = src->storage == ANN_F32 ? src->codes : src->x32;
        const uint32_t stride = src->storage == ANN_F32 ? src->row_bytes : src->row32_bytes;
        if (!x) {
            set_error("ann_shards_link: shard %u keeps no FP32 vectors (create it with keep_fp32)", i);
            st = ANN_EINVAL;
            break;
        }
        cudaError_t e = cudaSuccess;
        if (!s->links[i]) e = cudaMalloc(&s->links[i], s->n[i] * 4);
        if (e != cudaSuccess) { st = cuda_fail(e, "ann_shards_link"); break; }
        float *q = static_cast<float *>(s->ws);
        float *dd = reinterpret_cast<float *>(static_cast<uint8_t *>(s->ws) + up256(most * d * 4));
        for (uint64_t lo = 0; lo < s->n[i] && st == ANN_OK; lo += kLinkChunk) {
            const uint64_t rows = std::min<uint64_t>(kLinkChunk, s->n[i] - lo);
            e = cudaMemcpy2DAsync(q, (size_t)d * 4, static_cast<const uint8_t *>(x) + lo * stride, stride,
                                  (size_t)d * 4, rows, cudaMemcpyDeviceToDevice, cs);
            if (e != cudaSuccess) { st = cuda_fail(e, "ann_shards_link copy"); break; }
            ann_search_params pl = *p;
            pl.k = 1;
            pl.qid_base = p->qid_base + lo;   // node u's stream is its local index
            st = search_launch(nxt, q, (uint32_t)rows, &pl, nullptr, 0, s->links[i] + lo, dd, nullptr, cs);
        }
    }
    if (st == ANN_OK) {
        cudaError_t e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) st = cuda_fail(e, "ann_shards_link");
    }
    leave_device(s->device, prev);
    return st;
}

ann_status ann_shards_search(ann_shards *s, const float *queries, uint32_t nq, const ann_search_params *p,
                             uint32_t n_forward, uint32_t *ids, float *dists, ann_query_stats *stats, void *stream)
{
    if (!s || !p) { set_error("ann_shards_search: NULL argument"); return ANN_EINVAL; }
    if (nq == 0) return ANN_OK;
    if (!queries || !ids || !dists) { set_error("ann_shards_search: NULL buffers"); return ANN_EINVAL; }
    if (p->entry > ANN_ENTRY_GHOST) {
        set_error("ann_shards_search: entry %u is not available (random or ghost staging start a chunk)", p->entry);
        return ANN_EINVAL;
    }
    if (n_forward > ANN_MAX_FORWARD || n_forward > p->k || p->k == 0) {
        set_error("ann_shards_search: need n_forward <= min(k, %u)", ANN_MAX_FORWARD);
        return ANN_EINVAL;
    }
    if (n_forward)
        for (uint32_t i = 0; i < s->N; ++i)
            if (!s->links[i]) { set_error("ann_shards_search: shard %u has no links", i); return ANN_EINVAL; }
    int prev = -1;
    ann_status st = enter_device(s->device, &prev, "ann_shards_search");
    if (st != ANN_OK) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    const uint32_t N = s->N, k = p->k, d = s->dim;
    const size_t list = (size_t)N * nq * k * 4;
    st = grow_ws(s, 2 * up256(list) + up256((size_t)nq * std::max(1u, n_forward) * 4), cs);
    if (st != ANN_OK) { leave_device(s->device, prev); return st; }
    uint32_t *loc_ids = static_cast<uint32_t *>(s->ws);
    float *loc_d = reinterpret_cast<float *>(static_cast<uint8_t *>(s->ws) + up256(list));
    uint32_t *seeds = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(s->ws) + 2 * up256(list));
    cudaError_t e = cudaEventRecord(s->start, cs);
    for (uint32_t c = 0; c < N && e == cudaSuccess; ++c) e = cudaStreamWaitEvent(s->streams[c], s->start, 0);
    if (e != cudaSuccess) st = cuda_fail(e, "ann_shards_search");
    for (uint32_t t = 0; t < N && st == ANN_OK; ++t) {
        for (uint32_t c = 0; c < N && st == ANN_OK; ++c) {
            const uint32_t lo = (uint32_t)((uint64_t)c * nq / N), hi = (uint32_t)((uint64_t)(c + 1) * nq / N);
            if (hi == lo) continue;
            const uint32_t sh = (c + t) % N, rows = hi - lo;
            cudaStream_t ss = s->streams[c];
            ann_search_params pt = *p;
            pt.qid_base = p->qid_base + lo;
            const uint32_t *given = nullptr;
            if (t > 0 && n_forward) {
                const uint32_t from = (sh + N - 1) % N;
                forward_kernel<<<grid_for((uint64_t)rows * n_forward, 256), 256, 0, ss>>>(
                    loc_ids + ((size_t)(t - 1) * nq + lo) * k, k, rows, n_forward, s->links[from], s->n[from],
                    seeds + (size_t)lo * n_forward);
                e = cudaGetLastError();
                if (e != cudaSuccess) { st = cuda_fail(e, "forward_kernel"); break; }
                pt.entry = ANN_ENTRY_GIVEN_BASE;
                given = seeds + (size_t)lo * n_forward;
            }
            st = search_launch(s->ix[sh], queries + (size_t)lo * d, rows, &pt, given, given ? n_forward : 0,
                               loc_ids + ((size_t)t * nq + lo) * k, loc_d + ((size_t)t * nq + lo) * k,
                               stats ? stats + (size_t)t * nq + lo : nullptr, ss);
        }
    }
    for (uint32_t c = 0; c < N && st == ANN_OK; ++c) {
        e = cudaEventRecord(s->done[c], s->streams[c]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, s->done[c], 0);
        if (e != cudaSuccess) st = cuda_fail(e, "ann_shards_search join");
    }
    if (st == ANN_OK) {
        GidTables gt{};
        for (uint32_t i = 0; i < N; ++i) gt.g[i] = s->gids[i];
        reduce_kernel<<<grid_for(nq, 128), 128, 0, cs>>>(loc_ids, loc_d, nq, N, k, gt, ids, dists);
        e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(e, "reduce_kernel");
    }
    leave_device(s->device, prev);
    return st;
}

}  // extern "C"
