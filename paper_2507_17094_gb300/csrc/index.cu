// Index construction and preprocessing kernels.
//
//   - low-precision codec: FP16 with a power-of-two per-vector scale, OCP FP8
//     E4M3 with scale max|x|/448 (round to nearest even, saturating);
//   - direction table (Section 3.3.2 (a), Section 4): per edge u->v one sign
//     bit per dimension, bit b of word w = [x_v[32w+b] > x_u[32w+b]], built
//     here with one warp per node and a ballot per 32 dimensions;
//   - the ghost shard's stored rows (Section 3.2.2), gathered contiguously so
//     ghost staging reads a small, L2-resident array.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "ann_internal.cuh"

namespace ann {

ann_status visited_pool_alloc(ann_visited_pool &vp, uint32_t slots, uint32_t bits)
{
    vp.slots = slots;
    vp.bits = bits;
    const size_t tab_bytes = ((size_t)slots << bits) * sizeof(uint32_t);
    cudaError_t e = cudaMalloc(&vp.tab, tab_bytes);
    if (e == cudaSuccess) e = cudaMemset(vp.tab, 0, tab_bytes);
    if (e != cudaSuccess) {
        visited_pool_free(vp);
        return cuda_fail(e, "visited tables");
    }
    return ANN_OK;
}

void visited_pool_free(ann_visited_pool &vp)
{
    if (vp.tab) cudaFree(vp.tab);
    vp = ann_visited_pool{};
}

// Visited-table slots of an index: 28 warps per SM, more than the search
// kernel's register budget lets run (6 blocks of 4 warps); a launch is also
// capped so that its resident warps never outnumber the slots.
uint32_t max_warp_slots(const ann_index *ix) { return (uint32_t)ix->num_sms * 7u * 4u; }

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

ann_status cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? ANN_ENOMEM : ANN_ECUDA;
}

ann_status enter_device(int dev, int *prev, const char *who)
{
    *prev = -1;
    if (cudaGetDevice(prev) != cudaSuccess) *prev = -1;
    if (*prev == dev) return ANN_OK;
    cudaError_t e = cudaSetDevice(dev);
    if (e != cudaSuccess) {
        set_error("%s: cannot make device %d current: %s", who, dev, cudaGetErrorString(e));
        return ANN_EDEVICE;
    }
    return ANN_OK;
}

void leave_device(int dev, int prev)
{
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
}

// Keeps the caller's current device and restores it on scope exit; `status`
// is ANN_EDEVICE when the index's device could not be made current.
struct DeviceGuard {
    int dev = 0, prev = -1;
    ann_status status = ANN_OK;
    DeviceGuard(int d, const char *who) : dev(d) { status = enter_device(d, &prev, who); }
    ~DeviceGuard()
    {
        if (status == ANN_OK) leave_device(dev, prev);
    }
};

}  // namespace ann

using namespace ann;

// ---------------------------------------------------------------- device
template <int ST>
__device__ __forceinline__ float stored_elem(const uint8_t *row, uint32_t i, float scale)
{
    if (ST == ANN_F32) return reinterpret_cast<const float *>(row)[i];
    if (ST == ANN_F16) return __fmul_rn(scale, __half2float(reinterpret_cast<const __half *>(row)[i]));
    __half_raw h = __nv_cvt_fp8_to_halfraw(static_cast<__nv_fp8_storage_t>(row[i]), __NV_E4M3);
    return __fmul_rn(scale, __half2float(__half(h)));
}

// One warp per row: scale from max|x| (a warp max is exact in any order),
// then the codes.
template <int ST>
__global__ void encode_kernel(const float *__restrict__ x, uint64_t n, uint32_t d, uint8_t *__restrict__ codes,
                              uint32_t code_stride, float *__restrict__ scales)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t r = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += warps) {
        const float *xr = x + r * d;
        uint8_t *cr = codes + r * code_stride;
        if (ST == ANN_F32) {
            for (uint32_t i = lane; i < d; i += 32) reinterpret_cast<float *>(cr)[i] = xr[i];
            continue;
        }
        float mx = 0.0f;
        for (uint32_t i = lane; i < d; i += 32) mx = fmaxf(mx, fabsf(xr[i]));
        for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (ST == ANN_F16) {
            float s = 1.0f, inv = 1.0f;
            if (mx > 0.0f) {
                uint32_t b = __float_as_uint(mx);
                uint32_t ex = b >> 23;
                int E = ex ? (int)ex - 127 : (31 - __clz(b & 0x7fffffu)) - 149;  // floor(log2 mx)
                int e = E - 14;
                if (e < -126) e = -126;
                s = __uint_as_float((uint32_t)(e + 127) << 23);
                inv = __uint_as_float((uint32_t)(127 - e) << 23);
            }
            if (lane == 0) scales[r] = s;
            for (uint32_t i = lane; i < d; i += 32)
                reinterpret_cast<__half *>(cr)[i] = __float2half_rn(__fmul_rn(xr[i], inv));
        } else {
            float s = mx > 0.0f ? __fdiv_rn(mx, 448.0f) : 1.0f;
            if (lane == 0) scales[r] = s;
            for (uint32_t i = lane; i < d; i += 32)
                cr[i] = (uint8_t)__nv_cvt_float_to_fp8(__fdiv_rn(xr[i], s), __NV_SATFINITE, __NV_E4M3);
        }
    }
}

// One warp per node u; word t of edge j is the ballot of
// [x_v[32t + lane] > x_u[32t + lane]] over the lanes (pad lanes vote 0).
template <int ST>
__global__ void dir_table_kernel(const uint8_t *__restrict__ codes, uint32_t code_stride,
                                 const float *__restrict__ scales, uint64_t n, uint32_t d,
                                 const uint32_t *__restrict__ graph, uint32_t deg, uint32_t graph_stride,
                                 uint32_t *__restrict__ dir, uint32_t dir_node_stride)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t w = (d + 31) / 32;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t u = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < n; u += warps) {
        const uint8_t *xu = codes + u * code_stride;
        const float su = scales ? scales[u] : 1.0f;
        for (uint32_t j = 0; j < deg; ++j) {
            const uint32_t v = graph[u * graph_stride + j];
            uint32_t *out = dir + u * dir_node_stride + (uint64_t)j * w;
            if (v == ANN_INVALID_ID) {
                for (uint32_t t = lane; t < w; t += 32) out[t] = 0;
                continue;
            }
            const uint8_t *xv = codes + (uint64_t)v * code_stride;
            const float sv = scales ? scales[v] : 1.0f;
            for (uint32_t t = 0; t < w; ++t) {
                const uint32_t i = 32 * t + lane;
                bool b = false;
                if (i < d) b = stored_elem<ST>(xv, i, sv) > stored_elem<ST>(xu, i, su);
                const uint32_t word = __ballot_sync(0xffffffffu, b);
                if (lane == 0) out[t] = word;
            }
        }
    }
}

// Copy rows ids[i] of (codes, scales) into dense ghost arrays.
__global__ void gather_rows_kernel(const uint8_t *__restrict__ codes, const float *__restrict__ scales,
                                   uint32_t row_bytes, const uint32_t *__restrict__ ids, uint32_t m,
                                   uint8_t *__restrict__ out, float *__restrict__ out_scales)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < m; r += warps) {
        const uint4 *src = reinterpret_cast<const uint4 *>(codes + (uint64_t)ids[r] * row_bytes);
        uint4 *dst = reinterpret_cast<uint4 *>(out + (uint64_t)r * row_bytes);
        for (uint32_t c = lane; c < row_bytes / 16; c += 32) dst[c] = src[c];
        if (lane == 0 && scales) out_scales[r] = scales[ids[r]];
    }
}

// Ghost index of each id by binary search over the ascending ghost ids;
// ANN_INVALID_ID where the id is not a ghost node.
__global__ void ghost_index_kernel(const uint32_t *__restrict__ ghost_ids, uint32_t m,
                                   const uint32_t *__restrict__ ids, uint32_t n, uint32_t *__restrict__ out)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t v = ids[i];
        uint32_t lo = 0, hi = m;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (ghost_ids[mid] < v) lo = mid + 1;
            else hi = mid;
        }
        out[i] = (lo < m && ghost_ids[lo] == v) ? lo : ANN_INVALID_ID;
    }
}

// ---------------------------------------------------------------- host
static int grid_for(uint64_t items, int warps_per_block, int num_sms)
{
    uint64_t blocks = (items + warps_per_block - 1) / warps_per_block;
    uint64_t cap = (uint64_t)num_sms * 16;
    return (int)(blocks < cap ? (blocks ? blocks : 1) : cap);
}

static int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

static ann_status launch_encode(const float *x, uint64_t n, uint32_t d, int storage, void *codes,
                                uint32_t code_stride, float *scales, cudaStream_t st)
{
    const int g = grid_for(n, 8, sm_count());
    switch (storage) {
    case ANN_F32: encode_kernel<ANN_F32><<<g, 256, 0, st>>>(x, n, d, (uint8_t *)codes, code_stride, scales); break;
    case ANN_F16: encode_kernel<ANN_F16><<<g, 256, 0, st>>>(x, n, d, (uint8_t *)codes, code_stride, scales); break;
    case ANN_E4M3: encode_kernel<ANN_E4M3><<<g, 256, 0, st>>>(x, n, d, (uint8_t *)codes, code_stride, scales); break;
    default: set_error("unknown storage %d", storage); return ANN_EINVAL;
    }
    ANN_CUDA(cudaGetLastError());
    return ANN_OK;
}

static ann_status launch_dir(const void *codes, uint32_t code_stride, const float *scales, int storage, uint64_t n,
                             uint32_t d, const uint32_t *graph, uint32_t deg, uint32_t graph_stride, uint32_t *dir,
                             uint32_t dir_node_stride, cudaStream_t st)
{
    const int g = grid_for(n, 8, sm_count());
    const uint8_t *c = (const uint8_t *)codes;
    switch (storage) {
    case ANN_F32:
        dir_table_kernel<ANN_F32><<<g, 256, 0, st>>>(c, code_stride, nullptr, n, d, graph, deg, graph_stride, dir,
                                                      dir_node_stride);
        break;
    case ANN_F16:
        dir_table_kernel<ANN_F16><<<g, 256, 0, st>>>(c, code_stride, scales, n, d, graph, deg, graph_stride, dir,
                                                      dir_node_stride);
        break;
    case ANN_E4M3:
        dir_table_kernel<ANN_E4M3><<<g, 256, 0, st>>>(c, code_stride, scales, n, d, graph, deg, graph_stride, dir,
                                                       dir_node_stride);
        break;
    default: set_error("unknown storage %d", storage); return ANN_EINVAL;
    }
    ANN_CUDA(cudaGetLastError());
    return ANN_OK;
}

extern "C" {

const char *ann_last_error(void) { return g_err; }

void ann_default_params(ann_search_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->k = 10;
    p->itopk = 64;
    p->search_width = 1;
    p->max_iters = 64;
    p->dgs_cooldown = 0.3f;
    p->ghost_max_iters = 16;
    p->ghost_max_iters_given = 4;
    p->ghost_search_width = 1;
}

ann_status ann_encode(const float *x, uint64_t n, uint32_t dim, ann_storage storage, void *codes, float *scales,
                      void *stream)
{
    if (!x || !codes || dim == 0 || dim > ANN_MAX_DIM || (storage != ANN_F32 && !scales)) {
        set_error("ann_encode: bad arguments");
        return ANN_EINVAL;
    }
    if (n == 0) return ANN_OK;
    const uint32_t eb = storage == ANN_F32 ? 4 : storage == ANN_F16 ? 2 : 1;
    return launch_encode(x, n, dim, storage, codes, dim * eb, scales, (cudaStream_t)stream);
}

ann_status ann_dir_table(const void *vectors, const float *scales, ann_storage storage, uint64_t n, uint32_t dim,
                         const uint32_t *graph, uint32_t degree, uint32_t *dir, void *stream)
{
    if (!vectors || !graph || !dir || dim == 0 || dim > ANN_MAX_DIM || degree == 0 || degree > ANN_MAX_DEGREE ||
        (storage != ANN_F32 && !scales)) {
        set_error("ann_dir_table: bad arguments");
        return ANN_EINVAL;
    }
    if (n == 0) return ANN_OK;
    const uint32_t eb = storage == ANN_F32 ? 4 : storage == ANN_F16 ? 2 : 1;
    const uint32_t w = (dim + 31) / 32;
    return launch_dir(vectors, dim * eb, storage == ANN_F32 ? nullptr : scales, storage, n, dim, graph, degree,
                      degree, dir, degree * w, (cudaStream_t)stream);
}

ann_status ann_index_free(ann_index *ix)
{
    if (!ix) return ANN_OK;
    DeviceGuard g(ix->device, "ann_index_free");   // frees best-effort even if the switch failed
    if (ix->busy) {
        cudaEventSynchronize(ix->busy);
        cudaEventDestroy(ix->busy);
    }
    void *ptrs[] = {ix->codes, ix->scales, ix->graph, ix->dir, ix->ghost_ids, ix->ghost_codes,
                    ix->ghost_scales, ix->ghost_graph, ix->d_counter, ix->d_error, ix->ws};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    visited_pool_free(ix->visited);
    if (ix->x32 && (void *)ix->x32 != ix->codes) cudaFree(ix->x32);
    delete ix;
    return ANN_OK;
}

ann_status ann_index_create(int device, ann_storage storage, uint64_t n, uint32_t dim, uint32_t degree,
                            const float *vectors, const uint32_t *graph, uint32_t n_ghost,
                            const uint32_t *ghost_ids, uint32_t ghost_degree, const uint32_t *ghost_graph,
                            uint32_t keep_fp32, uint32_t build_dir, ann_index **out)
{
    if (!out) { set_error("ann_index_create: out is NULL"); return ANN_EINVAL; }
    *out = nullptr;
    if (storage != ANN_F32 && storage != ANN_F16 && storage != ANN_E4M3) {
        set_error("ann_index_create: unknown storage %d", (int)storage);
        return ANN_EINVAL;
    }
    if (!vectors || !graph || n == 0 || n >= (1ull << 31) || dim == 0 || dim > ANN_MAX_DIM || degree == 0 ||
        degree > ANN_MAX_DEGREE) {
        set_error("ann_index_create: need n in [1, 2^31), dim in [1, %u], degree in [1, %u]", ANN_MAX_DIM,
                  ANN_MAX_DEGREE);
        return ANN_EINVAL;
    }
    if (n_ghost && (!ghost_ids || !ghost_graph || ghost_degree == 0 || ghost_degree > ANN_MAX_DEGREE ||
                    n_ghost > n)) {
        set_error("ann_index_create: ghost set needs ids, a graph and ghost_degree in [1, %u]", ANN_MAX_DEGREE);
        return ANN_EINVAL;
    }
    for (uint64_t i = 0; i < n * degree; ++i)
        if (graph[i] != ANN_INVALID_ID && graph[i] >= n) {
            set_error("ann_index_create: graph[%llu] = %u is not a node id", (unsigned long long)i, graph[i]);
            return ANN_EINVAL;
        }
    for (uint32_t i = 0; i < n_ghost; ++i)
        if (ghost_ids[i] >= n || (i && ghost_ids[i] <= ghost_ids[i - 1])) {
            set_error("ann_index_create: ghost ids must be distinct node ids in ascending order");
            return ANN_EINVAL;
        }
    for (uint64_t i = 0; i < (uint64_t)n_ghost * ghost_degree; ++i)
        if (ghost_graph[i] != ANN_INVALID_ID && ghost_graph[i] >= n_ghost) {
            set_error("ann_index_create: ghost_graph[%llu] is not a ghost index", (unsigned long long)i);
            return ANN_EINVAL;
        }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        set_error("ann_index_create: no CUDA device %d", device);
        return ANN_EDEVICE;
    }
    DeviceGuard guard(device, "ann_index_create");
    if (guard.status != ANN_OK) return guard.status;
    ann_index *ix = new ann_index();
    ix->device = device;
    ix->storage = storage;
    ix->n = n;
    ix->dim = dim;
    ix->degree = degree;
    ix->deg_pad = round_up(degree, 4);
    ix->words = (dim + 31) / 32;
    ix->elem_bytes = storage == ANN_F32 ? 4 : storage == ANN_F16 ? 2 : 1;
    ix->row_bytes = row_stride(dim * ix->elem_bytes);
    ix->row32_bytes = row_stride(dim * 4);
    cudaDeviceGetAttribute(&ix->num_sms, cudaDevAttrMultiProcessorCount, device);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    ix->smem_optin = (size_t)optin;

    auto fail = [&](ann_status s) { ann_index_free(ix); return s; };
#define ANN_TRY(call)                                                          \
    do {                                                                       \
        cudaError_t _e = (call);                                               \
        if (_e != cudaSuccess) return fail(cuda_fail(_e, #call));              \
    } while (0)

    ANN_TRY(cudaMalloc(&ix->codes, n * ix->row_bytes));
    if (storage != ANN_F32) ANN_TRY(cudaMalloc(&ix->scales, n * sizeof(float)));
    ANN_TRY(cudaMalloc(&ix->graph, n * ix->deg_pad * sizeof(uint32_t)));
    ANN_TRY(cudaMalloc(&ix->d_counter, 64));
    ANN_TRY(cudaMalloc(&ix->d_error, 64));
    ANN_TRY(cudaMemset(ix->d_error, 0, 64));
    ANN_TRY(cudaEventCreateWithFlags(&ix->busy, cudaEventDisableTiming));
    if (ann_status vs = visited_pool_alloc(ix->visited, max_warp_slots(ix), kVisitedBits); vs != ANN_OK)
        return fail(vs);

    // vectors: upload in chunks of FP32 rows, encode into the padded layout
    {
        const uint64_t chunk = 1u << 20;
        float *tmp = nullptr;
        ANN_TRY(cudaMalloc(&tmp, std::min<uint64_t>(chunk, n) * dim * sizeof(float)));
        for (uint64_t s = 0; s < n; s += chunk) {
            const uint64_t m = std::min<uint64_t>(chunk, n - s);
            cudaError_t e = cudaMemcpy(tmp, vectors + s * dim, m * dim * sizeof(float), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) { cudaFree(tmp); return fail(cuda_fail(e, "upload vectors")); }
            ann_status st = launch_encode(tmp, m, dim, storage, (uint8_t *)ix->codes + s * ix->row_bytes,
                                          ix->row_bytes, ix->scales ? ix->scales + s : nullptr, 0);
            if (st != ANN_OK) { cudaFree(tmp); return fail(st); }
        }
        cudaError_t e = cudaDeviceSynchronize();
        cudaFree(tmp);
        if (e != cudaSuccess) return fail(cuda_fail(e, "encode"));
    }
    if (storage == ANN_F32) {
        ix->x32 = (float *)ix->codes;
    } else if (keep_fp32) {
        ANN_TRY(cudaMalloc(&ix->x32, n * ix->row32_bytes));
        ANN_TRY(cudaMemcpy2D(ix->x32, ix->row32_bytes, vectors, dim * sizeof(float), dim * sizeof(float), n,
                             cudaMemcpyHostToDevice));
    }
    ANN_TRY(cudaMemset(ix->graph, 0xFF, n * ix->deg_pad * sizeof(uint32_t)));
    ANN_TRY(cudaMemcpy2D(ix->graph, ix->deg_pad * sizeof(uint32_t), graph, degree * sizeof(uint32_t),
                         degree * sizeof(uint32_t), n, cudaMemcpyHostToDevice));
    if (build_dir) {
        ANN_TRY(cudaMalloc(&ix->dir, n * ix->deg_pad * ix->words * sizeof(uint32_t)));
        ANN_TRY(cudaMemset(ix->dir, 0, n * ix->deg_pad * ix->words * sizeof(uint32_t)));
        ann_status st = launch_dir(ix->codes, ix->row_bytes, ix->scales, storage, n, dim, ix->graph, degree,
                                   ix->deg_pad, ix->dir, ix->deg_pad * ix->words, 0);
        if (st != ANN_OK) return fail(st);
    }
    if (n_ghost) {
        ix->n_ghost = n_ghost;
        ix->ghost_degree = ghost_degree;
        ix->gdeg_pad = round_up(ghost_degree, 4);
        ANN_TRY(cudaMalloc(&ix->ghost_ids, n_ghost * sizeof(uint32_t)));
        ANN_TRY(cudaMemcpy(ix->ghost_ids, ghost_ids, n_ghost * sizeof(uint32_t), cudaMemcpyHostToDevice));
        ANN_TRY(cudaMalloc(&ix->ghost_codes, (uint64_t)n_ghost * ix->row_bytes));
        if (ix->scales) ANN_TRY(cudaMalloc(&ix->ghost_scales, n_ghost * sizeof(float)));
        gather_rows_kernel<<<grid_for(n_ghost, 8, ix->num_sms), 256>>>(
            (const uint8_t *)ix->codes, ix->scales, ix->row_bytes, ix->ghost_ids, n_ghost,
            (uint8_t *)ix->ghost_codes, ix->ghost_scales);
        ANN_TRY(cudaGetLastError());
        ANN_TRY(cudaMalloc(&ix->ghost_graph, (uint64_t)n_ghost * ix->gdeg_pad * sizeof(uint32_t)));
        ANN_TRY(cudaMemset(ix->ghost_graph, 0xFF, (uint64_t)n_ghost * ix->gdeg_pad * sizeof(uint32_t)));
        ANN_TRY(cudaMemcpy2D(ix->ghost_graph, ix->gdeg_pad * sizeof(uint32_t), ghost_graph,
                             ghost_degree * sizeof(uint32_t), ghost_degree * sizeof(uint32_t), n_ghost,
                             cudaMemcpyHostToDevice));
    }
    ANN_TRY(cudaDeviceSynchronize());
#undef ANN_TRY
    *out = ix;
    return ANN_OK;
}

ann_status ann_index_load(const char *path, int device, ann_storage storage, uint32_t keep_fp32,
                          uint32_t build_dir, ann_index **out)
{
    if (!path || !out) { set_error("ann_index_load: NULL argument"); return ANN_EINVAL; }
    FILE *f = fopen(path, "rb");
    if (!f) { set_error("ann_index_load: cannot open %s", path); return ANN_EIO; }
    char magic[8];
    uint64_t n = 0;
    uint32_t hdr[4] = {0, 0, 0, 0};
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "ANNIDX01", 8) == 0 && fread(&n, 8, 1, f) == 1 &&
              fread(hdr, 4, 4, f) == 4;
    const uint32_t dim = hdr[0], degree = hdr[1], n_ghost = hdr[2], gdeg = hdr[3];
    ok = ok && n > 0 && dim > 0 && dim <= ANN_MAX_DIM && degree > 0 && degree <= ANN_MAX_DEGREE &&
         n_ghost <= n && gdeg <= ANN_MAX_DEGREE;
    std::vector<float> X;
    std::vector<uint32_t> G, S, GG;
    if (ok) {
        try {
            X.resize(n * dim);
            G.resize(n * degree);
            S.resize(n_ghost);
            GG.resize((uint64_t)n_ghost * gdeg);
        } catch (...) {
            fclose(f);
            set_error("ann_index_load: out of host memory");
            return ANN_ENOMEM;
        }
        ok = fread(X.data(), 4, X.size(), f) == X.size() && fread(G.data(), 4, G.size(), f) == G.size() &&
             fread(S.data(), 4, S.size(), f) == S.size() && fread(GG.data(), 4, GG.size(), f) == GG.size();
    }
    fclose(f);
    if (!ok) { set_error("ann_index_load: %s is not a valid index file", path); return ANN_EIO; }
    return ann_index_create(device, storage, n, dim, degree, X.data(), G.data(), n_ghost,
                            n_ghost ? S.data() : nullptr, gdeg, n_ghost ? GG.data() : nullptr, keep_fp32,
                            build_dir, out);
}

ann_status ann_index_info(const ann_index *ix, uint64_t *n, uint32_t *dim, uint32_t *degree, uint32_t *storage,
                          uint32_t *n_ghost, uint32_t *ghost_degree)
{
    if (!ix) { set_error("ann_index_info: NULL index"); return ANN_EINVAL; }
    if (n) *n = ix->n;
    if (dim) *dim = ix->dim;
    if (degree) *degree = ix->degree;
    if (storage) *storage = (uint32_t)ix->storage;
    if (n_ghost) *n_ghost = ix->n_ghost;
    if (ghost_degree) *ghost_degree = ix->ghost_degree;
    return ANN_OK;
}

ann_status ann_index_export(const ann_index *ix, int which, void *dst, uint64_t bytes)
{
    if (!ix || !dst) { set_error("ann_index_export: NULL argument"); return ANN_EINVAL; }
    DeviceGuard g(ix->device, "ann_index_export");
    if (g.status != ANN_OK) return g.status;
    const uint64_t row = (uint64_t)ix->dim * ix->elem_bytes;
    const void *src = nullptr;
    uint64_t rows = 0, pitch = 0, width = 0;
    switch (which) {
    case 0: src = ix->codes; rows = ix->n; pitch = ix->row_bytes; width = row; break;
    case 1: src = ix->scales; rows = 1; width = pitch = ix->n * 4; break;
    case 2:
        src = ix->dir; rows = ix->n; pitch = (uint64_t)ix->deg_pad * ix->words * 4;
        width = (uint64_t)ix->degree * ix->words * 4; break;
    case 3: src = ix->ghost_codes; rows = ix->n_ghost; pitch = ix->row_bytes; width = row; break;
    case 4: src = ix->ghost_scales; rows = 1; width = pitch = (uint64_t)ix->n_ghost * 4; break;
    default: break;
    }
    if (!src || rows * width != bytes) {
        set_error("ann_index_export: array %d absent or size %llu != %llu", which, (unsigned long long)bytes,
                  (unsigned long long)(rows * width));
        return ANN_EINVAL;
    }
    ANN_CUDA(cudaMemcpy2D(dst, width, src, pitch, width, rows, cudaMemcpyDeviceToHost));
    return ANN_OK;
}

ann_status ann_ghost_index_of(const ann_index *ix, const uint32_t *ids, uint32_t n, uint32_t *out, void *stream)
{
    if (!ix || (n && (!ids || !out))) { set_error("ann_ghost_index_of: NULL argument"); return ANN_EINVAL; }
    if (!ix->n_ghost) { set_error("ann_ghost_index_of: the index has no ghost set"); return ANN_EINVAL; }
    if (n == 0) return ANN_OK;
    DeviceGuard g(ix->device, "ann_ghost_index_of");
    if (g.status != ANN_OK) return g.status;
    ghost_index_kernel<<<(int)std::min<uint64_t>((n + 255) / 256, (uint64_t)ix->num_sms * 8), 256, 0,
                         (cudaStream_t)stream>>>(ix->ghost_ids, ix->n_ghost, ids, n, out);
    ANN_CUDA(cudaGetLastError());
    return ANN_OK;
}

// One warp waits, at most `cycles`, for a phase of an mbarrier that no copy
// and no thread completes: the bounded wait must run out and record
// ANN_DEV_TIMEOUT in *err, and the kernel then returns normally.
__global__ void timeout_probe_kernel(int *err, long long cycles)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    fence_mbar_init();
    __syncwarp();
    (void)__all_sync(0xffffffffu, mbar_wait_bounded(&bar, 0, err, cycles));
}

ann_status ann_selftest_timeout(ann_index *ix)
{
    if (!ix) { set_error("ann_selftest_timeout: NULL index"); return ANN_EINVAL; }
    DeviceGuard g(ix->device, "ann_selftest_timeout");
    if (g.status != ANN_OK) return g.status;
    ANN_CUDA(cudaDeviceSynchronize());
    timeout_probe_kernel<<<1, 32>>>(ix->d_error, 2000000ll);   // about 1 ms at 2 GHz
    ANN_CUDA(cudaGetLastError());
    const ann_status s = ann_sync(ix, nullptr);
    if (s == ANN_ETIMEOUT) return ANN_OK;
    if (s == ANN_OK) set_error("ann_selftest_timeout: the expired wait was not reported");
    return s == ANN_OK ? ANN_EDEVICE : s;
}

ann_status ann_sync(ann_index *ix, void *stream)
{
    if (!ix) { set_error("ann_sync: NULL index"); return ANN_EINVAL; }
    DeviceGuard g(ix->device, "ann_sync");
    if (g.status != ANN_OK) return g.status;
    ANN_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int err = 0;
    ANN_CUDA(cudaMemcpy(&err, ix->d_error, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        ANN_CUDA(cudaMemset(ix->d_error, 0, sizeof(int)));
        set_error("a bounded device wait ran out (code %d)", err);
        return ANN_ETIMEOUT;
    }
    return ANN_OK;
}

}  // extern "C"
