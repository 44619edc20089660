// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <string>

#include "ann.h"

#define ANN_DEV_OK 0
#define ANN_DEV_TIMEOUT 1

// Device-side bound on any wait (an mbarrier phase, a flag): about one second
// at the GB300's clock. On expiry the waiter records ANN_DEV_TIMEOUT in the
// error word and gives up instead of spinning forever.
#define ANN_WAIT_LIMIT_CYCLES (2000000000ll)

// Per-warp visited tables in global memory: one table of 2^bits uint32
// entries (id + 1, 0 = empty) per resident-warp slot; a warp zeroes its table
// at the start of each query.
struct ann_visited_pool {
    uint32_t *tab = nullptr;     // slots x 2^bits
    uint32_t slots = 0, bits = 0;
};

struct ann_index {
    int device = 0;
    int storage = ANN_F32;
    uint64_t n = 0;
    uint32_t dim = 0, degree = 0, deg_pad = 0, words = 0;
    uint32_t elem_bytes = 4;     // bytes per stored element
    uint32_t row_bytes = 0;      // device row stride of the stored codes (multiple of 16)
    uint32_t row32_bytes = 0;    // device row stride of the FP32 originals (multiple of 16)
    void *codes = nullptr;       // n x row_bytes
    float *scales = nullptr;     // n (FP16 / E4M3)
    float *x32 = nullptr;        // n x row32_bytes (FP32 originals, optional)
    uint32_t *graph = nullptr;   // n x deg_pad
    uint32_t *dir = nullptr;     // n x deg_pad x words (optional)
    uint32_t n_ghost = 0, ghost_degree = 0, gdeg_pad = 0;
    uint32_t *ghost_ids = nullptr;     // n_ghost ascending
    void *ghost_codes = nullptr;       // n_ghost x row_bytes
    float *ghost_scales = nullptr;     // n_ghost
    uint32_t *ghost_graph = nullptr;   // n_ghost x gdeg_pad
    uint32_t *d_counter = nullptr;     // work counter for the persistent search kernel
    int *d_error = nullptr;            // device error word
    void *ws = nullptr;                // ann_search_host workspace
    size_t ws_bytes = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    ann_visited_pool visited;          // visited tables of ann_search launches
    cudaEvent_t busy = nullptr;        // completes when this index's last search does
    cudaStream_t busy_stream = nullptr;
    bool busy_set = false;
};

namespace ann {

void set_error(const char *fmt, ...);
ann_status cuda_fail(cudaError_t e, const char *what);

#define ANN_CUDA(call)                                              \
    do {                                                            \
        cudaError_t _e = (call);                                    \
        if (_e != cudaSuccess) return ::ann::cuda_fail(_e, #call);  \
    } while (0)

inline uint32_t round_up(uint32_t x, uint32_t m) { return (x + m - 1) / m * m; }

// Make `dev` current for an entry point, remembering the caller's device in
// *prev (-1 if it could not be read). Returns ANN_EDEVICE, with the message
// set, when the switch fails: the entry point must then return without
// touching device state, since another device would be current.
ann_status enter_device(int dev, int *prev, const char *who);
// Restore the caller's device after enter_device.
void leave_device(int dev, int prev);

// Per-query search parameters (derived from ann_search_params).
struct QParams {
    uint32_t k, L, W, T, m, n_keep, it_cool, reexpand, entry, Lg, Tg, Tg_given, g, rerank, n_given, Wg;
    uint64_t seed, qid_base;
    uint32_t min_match;   // > 0: DGS keeps the neighbours scoring >= min_match (not the top n_keep)
    float judge;          // > 0: given ghost seeds whose ghost result is farther continue to Tg
};
static_assert(sizeof(QParams) <= 96, "the serve kernel keeps a request's QParams in 96 bytes of shared memory");

// One request in the serving ring (device memory).
struct ServeReq {
    QParams qp;
    uint32_t nq, slot0, done, flag;
};

// The serving ring as the serve kernel sees it.
struct ServeRing {
    const float *queries;            // cap x dim
    const uint32_t *seeds;           // cap x P (learned entry) or NULL
    uint32_t P;
    uint32_t *ids;                   // cap x kmax
    float *dists;                    // cap x kmax
    const uint32_t *slot_req;        // cap: request-ring index of each slot
    ServeReq *reqs;
    unsigned long long *head;        // next query to take
    const unsigned long long *tail;  // queries published
    volatile uint32_t *flags;        // host-mapped completion flags
    uint32_t cap, kmax, per_warp;
};

// Visited tables for `slots` warps, 2^bits entries each; zeroed.
// visited_pool_free releases them.
ann_status visited_pool_alloc(ann_visited_pool &vp, uint32_t slots, uint32_t bits);
void visited_pool_free(ann_visited_pool &vp);
// Warp slots that one launch of the search or serve kernel can occupy.
uint32_t max_warp_slots(const ann_index *ix);
constexpr uint32_t kVisitedBits = 12;   // 4,096 entries (16 KB) per warp

// Validate `p` against the index and derive the per-query parameters.
ann_status derive_qparams(const ann_index *ix, const ann_search_params *p, uint32_t n_given, QParams *out);

// A serve-kernel launch plan sized for the largest parameters `maxp`
// (opaque; free with serve_plan_free).
// The plan owns visited tables for `n_streams` concurrent launches.
ann_status serve_plan(ann_index *ix, const ann_search_params *maxp, uint32_t n_given_max, uint32_t n_streams,
                      void **plan);
void serve_plan_free(void *plan);
// Launch a serve kernel with capacity for at least `queries` queries on
// `stream`, the plan's concurrent-launch slot `stream_index`.
ann_status serve_launch(void *plan, const ServeRing &ring, uint32_t queries, cudaStream_t stream,
                        uint32_t stream_index);

// The search launch (search.cu) with the index's own work counter and error
// word (ann_search after its device switch).
ann_status search_launch(ann_index *ix, const float *queries, uint32_t nq, const ann_search_params *p,
                         const uint32_t *given, uint32_t n_given, uint32_t *ids, float *dists,
                         ann_query_stats *stats, cudaStream_t stream);

// The search launch (search.cu) with caller-chosen device scratch: the work
// counter (zeroed on `stream` before the launch) and the error word. With
// `prof` (one row of ANN_PROFILE_STAGES x ANN_PROFILE_PHASES counters per
// visited-table slot) the profiling build of the kernel runs instead.
ann_status search_launch_ex(ann_index *ix, const float *queries, uint32_t nq, const ann_search_params *p,
                            const uint32_t *given, uint32_t n_given, uint32_t *ids, float *dists,
                            ann_query_stats *stats, cudaStream_t stream, uint32_t *counter, int *err,
                            unsigned long long *prof = nullptr);

// Device row stride for `bytes` of payload: a multiple of 16 bytes (the
// bulk-copy granule).
inline uint32_t row_stride(uint32_t bytes) { return round_up(bytes, 16); }

// Shared-memory row stride for staged rows: a multiple of 16 bytes whose
// word count is 4 mod 8, so 8 lanes reading 16 bytes each from 8 different
// rows hit 8 different 4-bank groups.
inline uint32_t smem_row_stride(uint32_t bytes)
{
    uint32_t w = round_up(bytes, 16) / 4;
    while (w % 8 != 4) w += 4;
    return w * 4;
}

}  // namespace ann

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make an mbarrier initialisation (and prior generic-proxy shared-memory
// writes) visible to the async proxy that bulk copies complete through.
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// One bounded test of phase `parity`: the thread may be suspended until the
// phase completes or about 0.1 ms pass (the suspend-time hint), so a waiting
// warp takes no issue slots from the others.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(100000u)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of `bar` to complete, at most `limit` cycles.
// Returns false (and records a timeout in *err) if it did not.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *err,
                                                  long long limit = ANN_WAIT_LIMIT_CYCLES)
{
    if (mbar_try_wait(bar, parity)) return true;
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) {
            atomicExch(err, ANN_DEV_TIMEOUT);
            return false;
        }
    }
    return true;
}

// One-dimensional bulk copy global -> this CTA's shared memory through the
// TMA engine; completion is counted in bytes on `bar`. dst, src and bytes
// must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
