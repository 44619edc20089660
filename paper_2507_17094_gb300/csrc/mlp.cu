// Learned entry (not in the paper): an MLP that maps a query to logits over
// the ghost set (Section 3.2.2), trained on the method's own ghost-staging
// results, whose top-P ghost nodes seed the ghost stage.
//
// Dense contractions run on the 5th-generation tensor cores: one GEMM kernel
// computes C = A * B^T with A (M x K) and B (N x K) both K-major BF16 in
// global memory, FP32 accumulation in tensor memory:
//   - TMA 2-D loads (128-byte swizzle) fill a 4-stage shared-memory ring,
//     one elected thread issues them; full/empty mbarriers link the stages;
//   - one elected thread issues tcgen05.mma (M 128, N 128, K 16 per
//     instruction) reading both operands from shared memory by descriptor;
//     tcgen05.commit frees a stage when the MMAs reading it are done;
//   - the accumulator (128 lanes x 128 columns) is read back with
//     tcgen05.ld by all four warps for the epilogue: plain FP32, bias,
//     bias + ReLU to BF16, or a fused top-P + online-softmax reduction so
//     inference never writes the (queries x ghosts) logits.
// Every mbarrier wait is bounded; on expiry the kernel records a timeout in
// the error word, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ann_internal.cuh"

using namespace ann;

namespace {

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 4;
constexpr int TILE_A = BM * BK * 2;
constexpr int TILE_B = BN * BK * 2;
constexpr int GEMM_STAGE_BYTES = STAGES * (TILE_A + TILE_B);
// top-P epilogue: each of the 8 x 32 epilogue threads parks a 32-logit chunk
// here (stride 33 floats: conflict-free) while it inserts the chunk's
// candidates one per step
constexpr int XS_STRIDE = 33;
constexpr int GEMM_XS_BYTES = 8 * 32 * XS_STRIDE * 4;
constexpr int GEMM_SMEM = GEMM_STAGE_BYTES + 256 + GEMM_XS_BYTES + 1024;
// Resident-A variant (fused top-P logits, K <= RES_K): a CTA keeps its row
// block's whole A (128 x K, as RES_K / BK swizzled 128 x BK tiles) in shared
// memory while B streams through a ring of RES_STAGES tiles, so the L2 ->
// shared-memory stream per tile halves (A is read once per row block).
constexpr int RES_K = 512;
constexpr int RES_STAGES = 4;
constexpr int RES_A_BYTES = (RES_K / BK) * TILE_A;
constexpr int RES_SMEM = RES_A_BYTES + RES_STAGES * TILE_B + 256 + GEMM_XS_BYTES + 1024;
static_assert(RES_SMEM <= 232448, "resident-A GEMM exceeds the shared memory of a CTA");
constexpr int TOPP = 8;   // top-P of the fused inference epilogue

enum { EPI_F32 = 0, EPI_BIAS_F32 = 1, EPI_BIAS_RELU_BF16 = 2, EPI_TOPP = 3 };

struct EpiArgs {
    float *c;                 // FP32 output, row stride ldc
    __nv_bfloat16 *cb;        // BF16 output, row stride ldc
    const float *bias;        // per output column
    uint32_t ldc;
    float *part;              // top-P partials: per (row, column tile) TOPP values, TOPP ids, max, sum
    uint32_t ntiles;
    int *err;
};

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major operand in the 128-byte swizzle
// layout TMA writes: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);        // start address
    d |= (uint64_t)1 << 16;                           // leading byte offset (unused in this layout)
    d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                           // descriptor version of this architecture
    d |= (uint64_t)2 << 61;                           // swizzle: 128 bytes
    return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, both K-major, M 128, N BN.
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t m, uint32_t n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// Two 32-column accumulator loads in flight together and one wait: the
// second statement waits for both and names the first load's registers as
// its operands, so no use of them can move above the wait.
__device__ __forceinline__ void tmem_ld32x2(uint32_t taddr0, uint32_t taddr1, float (&v0)[32], float (&v1)[32])
{
    uint32_t r[32], s[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr0));
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%64];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(s[7]), "=r"(s[8]), "=r"(s[9]), "=r"(s[10]), "=r"(s[11]), "=r"(s[12]), "=r"(s[13]), "=r"(s[14]), "=r"(s[15]), "=r"(s[16]), "=r"(s[17]), "=r"(s[18]), "=r"(s[19]), "=r"(s[20]), "=r"(s[21]), "=r"(s[22]), "=r"(s[23]), "=r"(s[24]), "=r"(s[25]), "=r"(s[26]), "=r"(s[27]), "=r"(s[28]), "=r"(s[29]), "=r"(s[30]), "=r"(s[31]),
          "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
        : "r"(taddr1)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        v0[i] = __uint_as_float(r[i]);
        v1[i] = __uint_as_float(s[i]);
    }
}

// Cluster helpers (the multicast logits kernel runs in clusters of two CTAs).
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// A 2-D TMA load whose data, and the completion of its bytes, land at the
// same shared-memory offsets in every CTA of `mask` within the cluster.
__device__ __forceinline__ void tma_load_2d_mc(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar,
                                               uint16_t mask)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1, "
        "{%2, %3}], [%4], %5;" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar)), "h"(mask)
        : "memory");
}

// tcgen05.commit arriving on the barrier at the same offset in every CTA of `mask`.
__device__ __forceinline__ void mma_commit_mc(uint64_t *bar, uint16_t mask)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_addr(bar)),
        "h"(mask)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// 2^x by the hardware approximation (MUFU): the softmax sum only decides the
// confidence fallback, relative error ~2^-22 is ample.
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ bool better(float va, uint32_t ia, float vb, uint32_t ib)
{
    return va > vb || (va == vb && ia < ib);
}

// max(a, b, c) in one instruction (the three-input form of max.f32)
__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// ------------------------------------------------------------------ GEMM
// Persistent and warp-specialised: CTA b walks the contiguous tile range
// [b * per, (b + 1) * per) in row-block-major order (per = ceil(tiles /
// grid)), so a CTA stays on one row block for many consecutive column tiles.
// Warp 0 streams A/B tiles with TMA into the stage ring, warp 1 issues the
// MMAs into one of two tensor-memory accumulators, warps 2-9 run the
// epilogue of the previous tile from the other accumulator (two warps per
// 32-lane quarter of the accumulator, one per half of the columns), so
// loads, MMAs and epilogues of consecutive tiles overlap.
constexpr int EPI_WARPS = 8;
constexpr int GEMM_THREADS = 64 + 32 * EPI_WARPS;

// Per-thread state of the fused top-P epilogue: the TOPP best (logit,
// column) pairs and the online-softmax (max, sum) of the columns seen.
struct TopP {
    float tv[TOPP];
    uint32_t ti[TOPP];
    float mx, sm;
    __device__ void reset()
    {
#pragma unroll
        for (int p = 0; p < TOPP; ++p) { tv[p] = -INFINITY; ti[p] = 0xFFFFFFFFu; }
        mx = -INFINITY;
        sm = 0.0f;
    }
};

// The bias of columns nb..nb+31 (0 past N; none for the plain FP32 store).
template <int EPI>
__device__ __forceinline__ void load_bias32(const EpiArgs &e, uint32_t nb, uint32_t N, float (&bias)[32])
{
    if (EPI == EPI_F32) return;
    if (nb + 32 <= N) {
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
            const float4 b4 = __ldg(reinterpret_cast<const float4 *>(e.bias + nb + j));
            bias[j] = b4.x; bias[j + 1] = b4.y; bias[j + 2] = b4.z; bias[j + 3] = b4.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) bias[j] = nb + j < N ? __ldg(e.bias + nb + j) : 0.0f;
    }
}

// One 32-column chunk of a row (accumulator values v, the columns' bias) for
// columns nb..nb+31, stored (the top-P epilogue is topp_pair).
template <int EPI>
__device__ __forceinline__ void epilogue_chunk(const float (&v)[32], const float (&bias)[32], uint32_t m, uint32_t M,
                                               uint32_t nb, uint32_t N, const EpiArgs &e)
{
    const bool full = nb + 32 <= N;
    if (EPI == EPI_F32 || EPI == EPI_BIAS_F32) {
        if (m >= M) return;
        float *out = e.c + (size_t)m * e.ldc + nb;
        if (full && (e.ldc % 4) == 0) {
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
                float4 o;
                o.x = v[j] + (EPI == EPI_BIAS_F32 ? bias[j] : 0.0f);
                o.y = v[j + 1] + (EPI == EPI_BIAS_F32 ? bias[j + 1] : 0.0f);
                o.z = v[j + 2] + (EPI == EPI_BIAS_F32 ? bias[j + 2] : 0.0f);
                o.w = v[j + 3] + (EPI == EPI_BIAS_F32 ? bias[j + 3] : 0.0f);
                *reinterpret_cast<float4 *>(out + j) = o;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (nb + j < N) out[j] = v[j] + (EPI == EPI_BIAS_F32 ? bias[j] : 0.0f);
        }
    } else if (EPI == EPI_BIAS_RELU_BF16) {
        if (m >= M) return;
        __nv_bfloat16 *out = e.cb + (size_t)m * e.ldc + nb;
        if (full && (e.ldc % 8) == 0) {
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
                uint4 o;
                __nv_bfloat162 h[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    h[k] = __floats2bfloat162_rn(fmaxf(v[j + 2 * k] + bias[j + 2 * k], 0.0f),
                                                 fmaxf(v[j + 2 * k + 1] + bias[j + 2 * k + 1], 0.0f));
                o.x = *reinterpret_cast<uint32_t *>(&h[0]);
                o.y = *reinterpret_cast<uint32_t *>(&h[1]);
                o.z = *reinterpret_cast<uint32_t *>(&h[2]);
                o.w = *reinterpret_cast<uint32_t *>(&h[3]);
                *reinterpret_cast<uint4 *>(out + j) = o;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (nb + j < N) out[j] = __float2bfloat16_rn(fmaxf(v[j] + bias[j], 0.0f));
        }
    }
}

// The logits of a 32-column chunk above the thread's current P-th best
// (bits of pend; their values parked in xs) enter its top-P one per step,
// all lanes inserting together. Columns reach a thread in increasing order,
// so every entry holds a smaller column and wins a tie: a new logit goes
// behind all entries >= it, each slot decided from the old values (no chain
// of swaps).
__device__ __forceinline__ void topp_insert(TopP &tp, const float *xs, uint32_t pend, uint32_t nb)
{
    while (__any_sync(0xffffffffu, pend != 0)) {
        if (pend) {
            const uint32_t j = __ffs(pend) - 1;
            pend &= pend - 1;
            const float xv = xs[j];
            if (xv > tp.tv[TOPP - 1]) {
                const uint32_t col = nb + j;
#pragma unroll
                for (int p = TOPP - 1; p > 0; --p) {
                    const bool before_prev = xv > tp.tv[p - 1];
                    const bool before_cur = xv > tp.tv[p];
                    tp.tv[p] = before_prev ? tp.tv[p - 1] : (before_cur ? xv : tp.tv[p]);
                    tp.ti[p] = before_prev ? tp.ti[p - 1] : (before_cur ? col : tp.ti[p]);
                }
                if (xv > tp.tv[0]) {
                    tp.tv[0] = xv;
                    tp.ti[0] = col;
                }
            }
        }
    }
}

// The fused top-P epilogue on a thread's 64 columns of a tile (accumulator
// chunks v0, v1; columns nb..nb+63; rows m >= M take part in the warp's
// collectives with no effect): the logits' max and exp-sum by trees over
// all 64 (three-input max, packed FP32 adds and multiply-adds) and one
// online-softmax combine; then each chunk's logits above the thread's P-th
// best enter its top-P. Most chunks hold none: the 64 columns' max says so
// without a per-column test.
__device__ __forceinline__ void topp_pair(const float (&v0)[32], const float (&v1)[32], const float (&b0)[32],
                                          const float (&b1)[32], uint32_t m, uint32_t M, uint32_t nb, uint32_t N,
                                          TopP &tp, float *xs)
{
    constexpr float kLog2e = 1.4426950408889634f;
    float x[64];
    if (nb + 64 <= N && m < M) {
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
            const float2 r0 = __fadd2_rn(make_float2(v0[j], v0[j + 1]), make_float2(b0[j], b0[j + 1]));
            const float2 r1 = __fadd2_rn(make_float2(v1[j], v1[j + 1]), make_float2(b1[j], b1[j + 1]));
            x[j] = r0.x;
            x[j + 1] = r0.y;
            x[32 + j] = r1.x;
            x[32 + j + 1] = r1.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            x[j] = (m < M && nb + j < N) ? v0[j] + b0[j] : -INFINITY;
            x[32 + j] = (m < M && nb + 32 + j < N) ? v1[j] + b1[j] : -INFINITY;
        }
    }
    float t[22];
#pragma unroll
    for (int j = 0; j < 21; ++j) t[j] = fmax3(x[3 * j], x[3 * j + 1], x[3 * j + 2]);
    t[21] = x[63];
#pragma unroll
    for (int j = 0; j < 7; ++j) t[j] = fmax3(t[3 * j], t[3 * j + 1], t[3 * j + 2]);
    t[7] = t[21];
    const float cm = fmax3(fmax3(t[0], t[1], t[2]), fmax3(t[3], t[4], t[5]), fmaxf(t[6], t[7]));
    if (cm > -INFINITY) {
        const float off = -cm * kLog2e;
        float2 e[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const float2 a = __ffma2_rn(make_float2(x[2 * j], x[2 * j + 1]), make_float2(kLog2e, kLog2e),
                                        make_float2(off, off));
            e[j] = make_float2(ex2_approx(a.x), ex2_approx(a.y));
        }
#pragma unroll
        for (int w = 16; w; w >>= 1)
#pragma unroll
            for (int j = 0; j < w; ++j) e[j] = __fadd2_rn(e[j], e[j + w]);
        const float cs = e[0].x + e[0].y;
        if (cm > tp.mx) {
            tp.sm = tp.sm * ex2_approx((tp.mx - cm) * kLog2e) + cs;
            tp.mx = cm;
        } else {
            tp.sm += cs * ex2_approx((cm - tp.mx) * kLog2e);
        }
    }
    uint32_t pend0 = 0, pend1 = 0;
    const float th = tp.tv[TOPP - 1];
    if (cm > th) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            pend0 |= (x[j] > th ? 1u : 0u) << j;
            pend1 |= (x[32 + j] > th ? 1u : 0u) << j;
        }
    }
    if (__any_sync(0xffffffffu, pend0 != 0)) {
        if (pend0) {
#pragma unroll
            for (int j = 0; j < 32; ++j) xs[j] = x[j];
        }
        __syncwarp();
        topp_insert(tp, xs, pend0, nb);
        __syncwarp();
    }
    if (__any_sync(0xffffffffu, pend1 != 0)) {
        if (pend1) {
#pragma unroll
            for (int j = 0; j < 32; ++j) xs[j] = x[32 + j];
        }
        __syncwarp();
        topp_insert(tp, xs, pend1, nb + 32);
        __syncwarp();
    }
}

// Top-P partial record of (row m, CTA segment slot): TOPP logits, TOPP
// columns, max, exp-sum.
__device__ __forceinline__ void topp_flush(const EpiArgs &e, const TopP &tp, uint32_t m, uint32_t slot)
{
    float *o = e.part + ((size_t)m * e.ntiles + slot) * (2 * TOPP + 2);
#pragma unroll
    for (int p = 0; p < TOPP; ++p) {
        o[p] = tp.tv[p];
        o[TOPP + p] = __uint_as_float(tp.ti[p]);
    }
    o[2 * TOPP] = tp.mx;
    o[2 * TOPP + 1] = tp.sm;
}

// MODE 0: the ring of (A, B) tiles; 1: resident A; 2: resident A, and the
// CTAs run in clusters of two on the two row blocks of a pair, loading half
// of each B tile each and multicasting it to both (B is read from L2 once
// per pair instead of once per CTA).
template <int EPI, int MODE = 0>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, uint32_t M,
                uint32_t N, uint32_t K, EpiArgs e)
{
    constexpr bool RESA = MODE >= 1, MC = MODE == 2;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t pad = (1024u - (smem_addr(smem_raw) & 1023u)) & 1023u;
    uint8_t *smem = smem_raw + pad;
    // ring layout: STAGES x (A tile, B tile); resident-A layout: the row
    // block's A tiles, then RES_STAGES B tiles
    constexpr int NST = RESA ? RES_STAGES : STAGES;
    constexpr int BAR_OFF = RESA ? RES_A_BYTES + RES_STAGES * TILE_B : GEMM_STAGE_BYTES;
    uint8_t *sA = smem;
    uint8_t *sB = smem + (RESA ? RES_A_BYTES : STAGES * TILE_A);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + BAR_OFF);
    uint64_t *empty = full + NST;
    uint64_t *acc_full = empty + NST;        // [2]: MMA -> epilogue
    uint64_t *acc_empty = acc_full + 2;      // [2]: epilogue -> MMA
    uint64_t *a_full = acc_empty + 2;        // resident A loaded
    uint64_t *a_empty = a_full + 1;          // resident A no longer read
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(a_empty + 1);
    float *xs_all = reinterpret_cast<float *>(smem + BAR_OFF + 256);
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t nkb = (K + BK - 1) / BK;
    const uint32_t n_tiles = (N + BN - 1) / BN, m_tiles = (M + BM - 1) / BM;
    // work units: tiles, or with clusters (row-block pair, column tile);
    // unit t covers row block rb(t) = row unit (t / n_tiles), or with
    // clusters row block 2 (t / n_tiles) + the CTA's rank in its pair
    const uint32_t crank = MC ? cluster_rank() : 0u;
    const uint32_t units = MC ? gridDim.x / 2 : gridDim.x, me = MC ? blockIdx.x / 2 : blockIdx.x;
    const uint32_t tiles = n_tiles * (MC ? (m_tiles + 1) / 2 : m_tiles);
    const uint32_t per = (tiles + units - 1) / units;
    const uint32_t t_begin = min(tiles, me * per), t_end = min(tiles, t_begin + per);
    auto rb_of_unit = [&](uint32_t u) { return MC ? 2 * u + crank : u; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], MC ? 2 : 1);   // with clusters, both CTAs' MMAs free a stage
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], EPI_WARPS);
        }
        mbar_init(a_full, 1);
        mbar_init(a_empty, 1);
        fence_mbar_init();
    }
    // both CTAs' barriers exist before either multicasts into the other
    if (MC) cluster_sync_all();
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"((uint32_t)(2 * BN))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && RESA) {
        if (lane == 0) {
            // A once per row block (after the MMAs on the previous one are
            // done), then the B tiles of each of the block's column tiles
            uint32_t it = 0, loads = 0, cur_u = 0xFFFFFFFFu;
            bool ok = true;
            for (uint32_t t = t_begin; t < t_end && ok; ++t) {
                const uint32_t u = t / n_tiles, n0 = (t % n_tiles) * BN;
                if (u != cur_u) {
                    if (loads > 0 && !(ok = mbar_wait_bounded(a_empty, (loads - 1) & 1, e.err))) break;
                    mbar_arrive_expect_tx(a_full, nkb * TILE_A);
                    for (uint32_t kb = 0; kb < nkb; ++kb)
                        tma_load_2d(sA + kb * TILE_A, &tA, (int)(kb * BK), (int)(rb_of_unit(u) * BM), a_full);
                    cur_u = u;
                    ++loads;
                }
                for (uint32_t kb = 0; kb < nkb; ++kb, ++it) {
                    const uint32_t s = it % NST, ph = (it / NST) & 1;
                    if (!(ok = mbar_wait_bounded(&empty[s], ph ^ 1, e.err))) break;
                    mbar_arrive_expect_tx(&full[s], TILE_B);
                    if (MC)   // this CTA's half of the B tile (64 rows), to both CTAs
                        tma_load_2d_mc(sB + s * TILE_B + crank * (TILE_B / 2), &tB, (int)(kb * BK),
                                       (int)(n0 + crank * (BN / 2)), &full[s], (uint16_t)3);
                    else
                        tma_load_2d(sB + s * TILE_B, &tB, (int)(kb * BK), (int)n0, &full[s]);
                }
            }
        }
    } else if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (uint32_t t = t_begin; t < t_end && ok; ++t) {
                const uint32_t m0 = (t / n_tiles) * BM, n0 = (t % n_tiles) * BN;
                for (uint32_t kb = 0; kb < nkb; ++kb, ++it) {
                    const uint32_t s = it % STAGES, ph = (it / STAGES) & 1;
                    if (!(ok = mbar_wait_bounded(&empty[s], ph ^ 1, e.err))) break;
                    mbar_arrive_expect_tx(&full[s], TILE_A + TILE_B);
                    tma_load_2d(sA + s * TILE_A, &tA, (int)(kb * BK), (int)m0, &full[s]);
                    tma_load_2d(sB + s * TILE_B, &tB, (int)(kb * BK), (int)n0, &full[s]);
                }
            }
        }
    } else if (warp == 1 && RESA) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(BM, BN);
            uint32_t it = 0, tc = 0, loads = 0, cur_u = 0xFFFFFFFFu;
            bool ok = true;
            for (uint32_t t = t_begin; t < t_end && ok; ++t, ++tc) {
                const uint32_t u = t / n_tiles;
                if (u != cur_u) {
                    if (!(ok = mbar_wait_bounded(a_full, loads & 1, e.err))) break;
                    cur_u = u;
                    ++loads;
                }
                const uint32_t buf = tc & 1, use = tc >> 1;
                if (!(ok = mbar_wait_bounded(&acc_empty[buf], (use & 1) ^ 1, e.err))) break;
                tc_fence_after();
                const uint32_t acc = tmem + buf * BN;
                for (uint32_t kb = 0; kb < nkb; ++kb, ++it) {
                    const uint32_t s = it % NST, ph = (it / NST) & 1;
                    if (!(ok = mbar_wait_bounded(&full[s], ph, e.err))) break;
                    tc_fence_after();
                    const uint32_t a0 = smem_addr(sA + kb * TILE_A), b0 = smem_addr(sB + s * TILE_B);
#pragma unroll
                    for (uint32_t k = 0; k < BK / 16; ++k)
                        mma_bf16(acc, desc_sw128(a0 + k * 32), desc_sw128(b0 + k * 32), idesc, (kb | k) != 0);
                    if (MC) mma_commit_mc(&empty[s], (uint16_t)3);   // frees the stage in both CTAs
                    else mma_commit(&empty[s]);
                }
                mma_commit(&acc_full[buf]);
                // the last tile of this row block: A may be replaced once
                // these MMAs are done
                if (t + 1 < t_end && (t + 1) / n_tiles != u) mma_commit(a_empty);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(BM, BN);
            uint32_t it = 0, tc = 0;
            bool ok = true;
            for (uint32_t t = t_begin; t < t_end && ok; ++t, ++tc) {
                const uint32_t buf = tc & 1, use = tc >> 1;
                if (!(ok = mbar_wait_bounded(&acc_empty[buf], (use & 1) ^ 1, e.err))) break;
                tc_fence_after();
                const uint32_t acc = tmem + buf * BN;
                for (uint32_t kb = 0; kb < nkb; ++kb, ++it) {
                    const uint32_t s = it % STAGES, ph = (it / STAGES) & 1;
                    if (!(ok = mbar_wait_bounded(&full[s], ph, e.err))) break;
                    tc_fence_after();
                    const uint32_t a0 = smem_addr(sA + s * TILE_A), b0 = smem_addr(sB + s * TILE_B);
#pragma unroll
                    for (uint32_t k = 0; k < BK / 16; ++k)
                        mma_bf16(acc, desc_sw128(a0 + k * 32), desc_sw128(b0 + k * 32), idesc, (kb | k) != 0);
                    mma_commit(&empty[s]);
                }
                mma_commit(&acc_full[buf]);
            }
        }
    } else {
        // epilogue warps 2..9: warp w reads accumulator lanes 32 * (w % 4) ..
        // + 31 (its quarter) and columns 64 * h .. + 63 of each tile
        const uint32_t q = warp & 3, h = (warp - 2) >> 2;
        uint32_t tc = 0, cur_u = 0xFFFFFFFFu;
        TopP tp;
        tp.reset();
        for (uint32_t t = t_begin; t < t_end; ++t, ++tc) {
            const uint32_t buf = tc & 1, use = tc >> 1;
            const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&acc_full[buf], use & 1, e.err));
            if (!ok) break;
            tc_fence_after();
            const uint32_t u = t / n_tiles, n0 = (t % n_tiles) * BN;
            const uint32_t m = rb_of_unit(u) * BM + q * 32 + lane;
            if (EPI == EPI_TOPP && u != cur_u) {
                // a new row block: the previous one's partial is complete
                if (cur_u != 0xFFFFFFFFu) {
                    const uint32_t pm = rb_of_unit(cur_u) * BM + q * 32 + lane;
                    if (pm < M) topp_flush(e, tp, pm, (me - (cur_u * n_tiles) / per) * 2 + h);
                }
                tp.reset();
                cur_u = u;
            }
            // the warp's two 32-column chunks of the tile in one round of
            // accumulator loads; the accumulator is released to the MMA
            // warp before the epilogue arithmetic
            // (the chunks' bias loads are in flight meanwhile)
            static_assert(BN / 2 == 64, "two 32-column chunks per epilogue warp and tile");
            const uint32_t nb = n0 + h * (BN / 2);
            float v0[32], v1[32], bias0[32], bias1[32];
            load_bias32<EPI>(e, nb, N, bias0);
            load_bias32<EPI>(e, nb + 32, N, bias1);
            __syncwarp();
            const uint32_t ta = tmem + buf * BN + ((q * 32u) << 16) + h * (BN / 2);
            tmem_ld32x2(ta, ta + 32, v0, v1);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
            if (EPI == EPI_TOPP) {
                topp_pair(v0, v1, bias0, bias1, m, M, nb, N, tp, xs_all + (threadIdx.x - 64) * XS_STRIDE);
            } else {
                epilogue_chunk<EPI>(v0, bias0, m, M, nb, N, e);
                epilogue_chunk<EPI>(v1, bias1, m, M, nb + 32, N, e);
            }
        }
        if (EPI == EPI_TOPP && cur_u != 0xFFFFFFFFu) {
            const uint32_t pm = rb_of_unit(cur_u) * BM + q * 32 + lane;
            if (pm < M) topp_flush(e, tp, pm, (me - (cur_u * n_tiles) / per) * 2 + h);
        }
    }
    tc_fence_before();
    __syncthreads();
    // no CTA leaves while its pair may still multicast into it or arrive on
    // its barriers
    if (MC) cluster_sync_all();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * BN))
                     : "memory");
    }
}

// ------------------------------------------------------------------ helpers
__global__ void to_bf16_kernel(const float *__restrict__ x, __nv_bfloat16 *__restrict__ y, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// Queries (rows x d) to the first GEMM's BF16 operand, standardised per
// dimension on the way: (x - mean) * inv_std, each step rounded in FP32
// (mean 0 and inv_std 1, the defaults, leave x unchanged).
__global__ void input_bf16_kernel(const float *__restrict__ x, const float *__restrict__ mean,
                                  const float *__restrict__ inv_std, __nv_bfloat16 *__restrict__ y, size_t rows,
                                  uint32_t d)
{
    const size_t n = rows * d;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t c = (uint32_t)(i % d);
        y[i] = __float2bfloat16_rn(__fmul_rn(__fsub_rn(x[i], mean[c]), inv_std[c]));
    }
}

// out (C x R) = in (R x C)^T, BF16, 32 x 32 tiles through shared memory
__global__ void transpose_bf16_kernel(const __nv_bfloat16 *__restrict__ in, __nv_bfloat16 *__restrict__ out,
                                      uint32_t R, uint32_t C)
{
    __shared__ __nv_bfloat16 t[32][33];
    const uint32_t c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (uint32_t i = threadIdx.y; i < 32; i += blockDim.y) {
        const uint32_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < R && c < C) t[i][threadIdx.x] = in[(size_t)r * C + c];
    }
    __syncthreads();
    for (uint32_t i = threadIdx.y; i < 32; i += blockDim.y) {
        const uint32_t c = c0 + i, r = r0 + threadIdx.x;
        if (r < R && c < C) out[(size_t)c * R + r] = t[threadIdx.x][i];
    }
}

// g' = g * [mask > 0] (mask optional), as BF16 (optional) and BF16^T (optional)
__global__ void post_grad_kernel(const float *__restrict__ g, const __nv_bfloat16 *__restrict__ mask,
                                 float *__restrict__ gm, __nv_bfloat16 *__restrict__ gb,
                                 __nv_bfloat16 *__restrict__ gT, uint32_t R, uint32_t C)
{
    __shared__ __nv_bfloat16 t[32][33];
    const uint32_t c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (uint32_t i = threadIdx.y; i < 32; i += blockDim.y) {
        const uint32_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < R && c < C) {
            const size_t at = (size_t)r * C + c;
            float v = g[at];
            if (mask && !(__bfloat162float(mask[at]) > 0.0f)) v = 0.0f;
            if (gm) gm[at] = v;
            const __nv_bfloat16 b = __float2bfloat16_rn(v);
            if (gb) gb[at] = b;
            t[i][threadIdx.x] = b;
        }
    }
    if (!gT) return;
    __syncthreads();
    for (uint32_t i = threadIdx.y; i < 32; i += blockDim.y) {
        const uint32_t c = c0 + i, r = r0 + threadIdx.x;
        if (r < R && c < C) gT[(size_t)c * R + r] = t[threadIdx.x][i];
    }
}

// Column sums of an R x C FP32 matrix, rows in order (deterministic).
__global__ void colsum_kernel(const float *__restrict__ g, float *__restrict__ out, uint32_t R, uint32_t C)
{
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float s = 0.0f;
    for (uint32_t r = 0; r < R; ++r) s += g[(size_t)r * C + c];
    out[c] = s;
}

// Row-wise softmax cross-entropy over z (B x N): z <- (softmax(z) - onehot(y)) / B,
// loss += mean_i(logsumexp(z_i) - z_i[y_i]). One warp per row.
__global__ void softmax_ce_kernel(float *__restrict__ z, const uint32_t *__restrict__ y, uint32_t B, uint32_t N,
                                  float *__restrict__ loss)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= B) return;
    float *zr = z + (size_t)r * N;
    float mx = -INFINITY;
    for (uint32_t c = lane; c < N; c += 32) mx = fmaxf(mx, zr[c]);
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float s = 0.0f;
    for (uint32_t c = lane; c < N; c += 32) s += expf(zr[c] - mx);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float lse = mx + logf(s);
    const uint32_t yr = y[r];
    const float zy = zr[yr];
    const float inv = 1.0f / (float)B;
    for (uint32_t c = lane; c < N; c += 32) zr[c] = (expf(zr[c] - lse) - (c == yr ? 1.0f : 0.0f)) * inv;
    if (lane == 0) atomicAdd(loss, (lse - zy) * inv);
}

struct AdamHP {
    float lr, b1, b2, eps, wd, c1, c2;
};

// AdamW (decoupled weight decay) on FP32 masters; refreshes the BF16 copy.
__global__ void adamw_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                             float *__restrict__ v, __nv_bfloat16 *__restrict__ wb, size_t n, AdamHP h)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = h.b1 * m[i] + (1.0f - h.b1) * gi;
        const float vi = h.b2 * v[i] + (1.0f - h.b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - h.lr * ((mi / h.c1) / (sqrtf(vi / h.c2) + h.eps) + h.wd * w[i]);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16_rn(wi);
    }
}

// Merge the per-tile top-P partials of each row; seeds = ghost ids of the
// top P (ties: smaller id), pmax = the largest softmax probability; a row
// with pmax < tau gets ANN_INVALID_ID as its first seed (fall back to
// random ghost seeds). One warp per row: each lane merges its slots (each
// read in one round of 8-byte loads) into a sorted top-P list, then P
// rounds of a warp-wide maximum over the lists' heads take the row's top P
// in order (the slots cover disjoint columns, so ids are distinct).
__global__ void topp_merge_kernel(const float *__restrict__ part, uint32_t M, uint32_t ntiles, uint32_t P,
                                  float tau, uint32_t *__restrict__ seeds, float *__restrict__ pmax)
{
    constexpr int SLOT = 2 * TOPP + 2;
    __shared__ float sv[4][32 * TOPP];
    __shared__ uint32_t si[4][32 * TOPP];
    const uint32_t lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const uint32_t r = blockIdx.x * 4 + wl;
    if (r >= M) return;
    float tv[TOPP];
    uint32_t ti[TOPP];
#pragma unroll
    for (int p = 0; p < TOPP; ++p) { tv[p] = -INFINITY; ti[p] = 0xFFFFFFFFu; }
    float mx = -INFINITY, sm = 0.0f;
    for (uint32_t t = lane; t < ntiles; t += 32) {
        const float2 *o2 = reinterpret_cast<const float2 *>(part + ((size_t)r * ntiles + t) * SLOT);
        float o[SLOT];
#pragma unroll
        for (int k = 0; k < SLOT / 2; ++k) {
            const float2 a = __ldg(o2 + k);
            o[2 * k] = a.x;
            o[2 * k + 1] = a.y;
        }
        const float tm = o[2 * TOPP], ts = o[2 * TOPP + 1];
        if (ts > 0.0f) {
            if (tm > mx) { sm = sm * __expf(mx - tm) + ts; mx = tm; }
            else sm += ts * __expf(tm - mx);
        }
#pragma unroll
        for (int p = 0; p < TOPP; ++p) {
            const float x = o[p];
            const uint32_t n = __float_as_uint(o[TOPP + p]);
            if (n == 0xFFFFFFFFu || !better(x, n, tv[TOPP - 1], ti[TOPP - 1])) continue;
            tv[TOPP - 1] = x;
            ti[TOPP - 1] = n;
#pragma unroll
            for (int q = TOPP - 1; q > 0; --q)
                if (better(tv[q], ti[q], tv[q - 1], ti[q - 1])) {
                    const float a = tv[q]; tv[q] = tv[q - 1]; tv[q - 1] = a;
                    const uint32_t u = ti[q]; ti[q] = ti[q - 1]; ti[q - 1] = u;
                }
        }
    }
    // softmax normaliser across lanes
    float gm = mx;
    for (int o = 16; o; o >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, o));
    float gs = (sm > 0.0f) ? sm * __expf(mx - gm) : 0.0f;
    for (int o = 16; o; o >>= 1) gs += __shfl_xor_sync(0xffffffffu, gs, o);
    // top-P across lanes: P rounds of the best head (every lane ends each
    // butterfly with the same winner; the lane holding it advances)
#pragma unroll
    for (int p = 0; p < TOPP; ++p) {
        sv[wl][lane * TOPP + p] = tv[p];
        si[wl][lane * TOPP + p] = ti[p];
    }
    __syncwarp();
    uint32_t hp = 0;
    for (uint32_t k = 0; k < P; ++k) {
        const uint32_t id = hp < TOPP ? si[wl][lane * TOPP + hp] : 0xFFFFFFFFu;
        const float v = hp < TOPP ? sv[wl][lane * TOPP + hp] : -INFINITY;
        float bv = v;
        uint32_t bid = id;
        for (int o = 16; o; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const uint32_t oid = __shfl_xor_sync(0xffffffffu, bid, o);
            if (oid != 0xFFFFFFFFu && (bid == 0xFFFFFFFFu || better(ov, oid, bv, bid))) {
                bv = ov;
                bid = oid;
            }
        }
        if (bid == 0xFFFFFFFFu) break;   // no entries left (the same in every lane)
        if (id == bid) ++hp;
        if (lane == 0) seeds[(size_t)r * P + k] = bid;
    }
    __syncwarp();
    const float pm = gs > 0.0f ? 1.0f / gs : 0.0f;
    if (lane == 0) {
        if (pmax) pmax[r] = pm;
        if (pm < tau) seeds[(size_t)r * P] = ANN_INVALID_ID;
    }
}

// Rows perm[0, n) of x (and their labels) into contiguous batch buffers.
__global__ void gather_batch_kernel(const float *__restrict__ x, const uint32_t *__restrict__ y,
                                    const uint32_t *__restrict__ perm, uint32_t n, uint32_t d,
                                    float *__restrict__ xb, uint32_t *__restrict__ yb)
{
    const uint32_t r = blockIdx.x;
    if (r >= n) return;
    const uint32_t src = perm[r];
    for (uint32_t c = threadIdx.x; c < d; c += blockDim.x) xb[(size_t)r * d + c] = x[(size_t)src * d + c];
    if (threadIdx.x == 0) yb[r] = y[src];
}

__global__ void accumulate_kernel(float *__restrict__ acc, const float *__restrict__ v, float w)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *acc += w * *v;
}

// ---------------------------------------------------------- input statistics
// Column sums of an n x d row-major FP32 matrix, in FP64, by row chunks: the
// block of chunk `blockIdx.x` and columns `blockIdx.y * blockDim.x + tid`
// adds its rows in row order (a warp reads consecutive columns of one row,
// so every load is coalesced) and writes one partial per (chunk, column).
// With `mean`, it sums the squared deviations (x - mean)^2 instead. The
// partials are added in chunk order by col_finish_kernel, so the result does
// not depend on scheduling.
__global__ void col_partial_kernel(const float *__restrict__ x, uint32_t n, uint32_t d, uint32_t rows_per_chunk,
                                   const double *__restrict__ mean, double *__restrict__ partial)
{
    const uint32_t c = blockIdx.y * blockDim.x + threadIdx.x;
    if (c >= d) return;
    const uint64_t r0 = (uint64_t)blockIdx.x * rows_per_chunk;
    const uint64_t r1 = (r0 + rows_per_chunk < (uint64_t)n) ? r0 + rows_per_chunk : (uint64_t)n;
    const double mu = mean ? mean[c] : 0.0;
    double s = 0.0;
    for (uint64_t r = r0; r < r1; ++r) {
        const double v = (double)x[r * d + c];
        if (mean) {
            const double t = __dsub_rn(v, mu);
            s = __dadd_rn(s, __dmul_rn(t, t));
        } else {
            s = __dadd_rn(s, v);
        }
    }
    partial[(size_t)blockIdx.x * d + c] = s;
}

// out[c] = (sum of the chunk partials of column c, in chunk order) / n.
__global__ void col_finish_kernel(const double *__restrict__ partial, uint32_t chunks, uint32_t d, uint32_t n,
                                  double *__restrict__ out)
{
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d) return;
    double s = 0.0;
    for (uint32_t k = 0; k < chunks; ++k) s = __dadd_rn(s, partial[(size_t)k * d + c]);
    out[c] = __ddiv_rn(s, (double)n);
}

// Standardisation from the FP64 mean and variance (one block): std = sqrt(var),
// the floor 1e-6 * max(largest std, 1e-30) keeps constant dimensions finite,
// inv_std = 1 / max(std, floor); both rounded once to FP32.
__global__ void norm_finish_kernel(const double *__restrict__ mean, const double *__restrict__ var, uint32_t d,
                                   float *__restrict__ mean_out, float *__restrict__ inv_std_out)
{
    __shared__ double red[32];
    double mx = 0.0;
    for (uint32_t c = threadIdx.x; c < d; c += blockDim.x) mx = fmax(mx, __dsqrt_rn(var[c]));
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        mx = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (threadIdx.x == 0) red[0] = mx;
    }
    __syncthreads();
    const double fl = 1e-6 * fmax(red[0], 1e-30);
    for (uint32_t c = threadIdx.x; c < d; c += blockDim.x) {
        mean_out[c] = __double2float_rn(mean[c]);
        inv_std_out[c] = __double2float_rn(__ddiv_rn(1.0, fmax(__dsqrt_rn(var[c]), fl)));
    }
}

// ---------------------------------------------------------- rank selection
// A total order on FP32 values as unsigned keys: negative values flip all
// bits, non-negative ones set the sign bit.
__device__ __forceinline__ uint32_t order_key(float f)
{
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// The value of 0-based rank `rank` among v[0..n) in ascending order (one
// block). The key is found bit by bit from the most significant: a bit is
// set when fewer than rank + 1 keys lie below the candidate, so the result is
// the largest key with at most `rank` keys below it -- the rank-th smallest.
__global__ void select_rank_kernel(const float *__restrict__ v, uint32_t n, uint32_t rank, float *__restrict__ out)
{
    __shared__ uint32_t red[32];
    __shared__ uint32_t total;
    uint32_t key = 0;
    for (int b = 31; b >= 0; --b) {
        const uint32_t t = key | (1u << b);
        uint32_t c = 0;
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) c += order_key(v[i]) < t ? 1u : 0u;
        c = __reduce_add_sync(0xffffffffu, c);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x < 32) {
            c = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0u;
            c = __reduce_add_sync(0xffffffffu, c);
            if (threadIdx.x == 0) total = c;
        }
        __syncthreads();
        if (total <= rank) key = t;
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = __uint_as_float((key & 0x80000000u) ? (key & 0x7FFFFFFFu) : ~key);
}

bool env_flag(const char *name, bool dflt)
{
    const char *v = getenv(name);
    return v ? atoi(v) != 0 : dflt;
}

uint64_t mix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

// ------------------------------------------------------------------ host side
struct ann_mlp {
    int device = 0;
    uint32_t d = 0, h1 = 0, h2 = 0, out = 0, maxb = 0;
    float *W[3] = {}, *b[3] = {}, *mW[3] = {}, *vW[3] = {}, *mb[3] = {}, *vb[3] = {}, *gW[3] = {}, *gb[3] = {};
    __nv_bfloat16 *Wb[3] = {}, *WT[3] = {};
    __nv_bfloat16 *xb = nullptr, *xT = nullptr, *h1b = nullptr, *h1T = nullptr, *h2b = nullptr, *h2T = nullptr;
    __nv_bfloat16 *dzb = nullptr, *dzT = nullptr, *da2b = nullptr, *da2T = nullptr, *da1T = nullptr;
    float *z = nullptr, *dh = nullptr, *dm = nullptr, *loss = nullptr, *part = nullptr;
    float *xbat = nullptr, *epoch_loss = nullptr;
    float *mean = nullptr, *inv_std = nullptr;   // input standardisation (in_dim each)
    uint32_t *ybat = nullptr, *perm = nullptr;
    size_t perm_cap = 0;
    uint32_t train_cap = 0;
    size_t part_cap = 0;
    uint32_t step = 0;
    int *d_error = nullptr;
    int num_sms = 0;
};

namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

ann_status get_encoder()
{
    if (g_encode) return ANN_OK;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return ANN_ECUDA;
    }
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return ANN_OK;
}

// Tensor map of a row-major BF16 matrix (rows x K, row stride K elements),
// box BK x box_rows, 128-byte swizzle; out-of-range elements read as zero.
ann_status make_map(CUtensorMap *map, const void *ptr, uint32_t rows, uint32_t K, uint32_t box_rows = 128)
{
    ann_status s = get_encoder();
    if (s != ANN_OK) return s;
    const cuuint64_t dims[2] = {K, rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {BK, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d) for %u x %u", (int)r, rows, K);
        return ANN_ECUDA;
    }
    return ANN_OK;
}

// Which GEMM variant runs: the fused top-P logits with K <= RES_K keep A
// resident (ANN_GEMM_RESIDENT_A=0 turns that off); ANN_GEMM_MULTICAST=1
// runs them in clusters of two CTAs that share each B tile by multicast
// (measured no faster: the L2 reads of B are not what bounds the kernel);
// everything else streams both operands.
int gemm_mode(int epi, uint32_t K)
{
    static const bool res_on = env_flag("ANN_GEMM_RESIDENT_A", true);
    static const bool mc_on = env_flag("ANN_GEMM_MULTICAST", false);
    if (epi != EPI_TOPP || K > (uint32_t)RES_K || !res_on) return 0;
    return mc_on ? 2 : 1;
}

// Work units of a launch (tiles, or with clusters row-block pairs x column
// tiles) and the persistent grid: one CTA per SM (pairs of CTAs with
// clusters), fewer if there is less work.
uint32_t gemm_units(uint32_t M, uint32_t N, int mode)
{
    const uint32_t n_tiles = (N + BN - 1) / BN, m_tiles = (M + BM - 1) / BM;
    return n_tiles * (mode == 2 ? (m_tiles + 1) / 2 : m_tiles);
}

// Clusters of two that can be resident at once (SMs pair up within a GPC,
// so this can be below half the SM count); queried once.
uint32_t pair_slots(uint32_t sms);

uint32_t gemm_grid(uint32_t M, uint32_t N, uint32_t sms, int mode = 0)
{
    const uint32_t units = gemm_units(M, N, mode);
    return mode == 2 ? 2 * std::max(1u, std::min(units, pair_slots(sms))) : std::max(1u, std::min(units, sms));
}

// Top-P partial slots per row: two column halves times the largest number
// of CTAs (pairs, with clusters) whose contiguous unit ranges meet one row
// unit.
uint32_t topp_slots(uint32_t M, uint32_t N, uint32_t sms, int mode)
{
    const uint32_t n_tiles = (N + BN - 1) / BN;
    const uint32_t units = gemm_units(M, N, mode), row_units = units / n_tiles;
    const uint32_t ctas = mode == 2 ? gemm_grid(M, N, sms, mode) / 2 : gemm_grid(M, N, sms, mode);
    const uint32_t per = (units + ctas - 1) / ctas;
    uint32_t smax = 1;
    for (uint32_t u = 0; u < row_units; ++u)
        smax = std::max(smax, ((u + 1) * n_tiles - 1) / per - (u * n_tiles) / per + 1);
    return 2 * smax;
}

uint32_t pair_slots(uint32_t sms)
{
    static uint32_t cached = 0;
    if (!cached) {
        cudaFuncSetAttribute(gemm_kernel<EPI_TOPP, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, RES_SMEM);
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(sms);
        cfg.blockDim = dim3(GEMM_THREADS);
        cfg.dynamicSmemBytes = RES_SMEM;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, gemm_kernel<EPI_TOPP, 2>, &cfg) != cudaSuccess || n <= 0)
            n = (int)(sms / 2);
        cudaGetLastError();
        cached = (uint32_t)std::min<int>(n, (int)(sms / 2));
    }
    return cached;
}

template <int EPI>
ann_status gemm(const __nv_bfloat16 *A, const __nv_bfloat16 *B, uint32_t M, uint32_t N, uint32_t K, EpiArgs e,
                cudaStream_t st)
{
    if (M == 0 || N == 0) return ANN_OK;
    if (K % 8) {
        set_error("gemm: K = %u must be a multiple of 8", K);
        return ANN_EINVAL;
    }
    const int mode = gemm_mode(EPI, K);
    CUtensorMap ta, tb;
    ann_status s = make_map(&ta, A, M, K);
    if (s == ANN_OK) s = make_map(&tb, B, N, K, mode == 2 ? BN / 2 : 128);
    if (s != ANN_OK) return s;
    static bool attr[3] = {false, false, false};
    if (!attr[mode]) {
        if (mode == 0)
            ANN_CUDA(cudaFuncSetAttribute(gemm_kernel<EPI, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM));
        else if (mode == 1)
            ANN_CUDA(cudaFuncSetAttribute(gemm_kernel<EPI, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, RES_SMEM));
        else
            ANN_CUDA(cudaFuncSetAttribute(gemm_kernel<EPI, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, RES_SMEM));
        attr[mode] = true;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t grid = gemm_grid(M, N, (uint32_t)sms, mode);
    if (mode == 0) {
        gemm_kernel<EPI, 0><<<grid, GEMM_THREADS, GEMM_SMEM, st>>>(ta, tb, M, N, K, e);
    } else if (mode == 1) {
        gemm_kernel<EPI, 1><<<grid, GEMM_THREADS, RES_SMEM, st>>>(ta, tb, M, N, K, e);
    } else {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(GEMM_THREADS);
        cfg.dynamicSmemBytes = RES_SMEM;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        ANN_CUDA(cudaLaunchKernelEx(&cfg, gemm_kernel<EPI, 2>, ta, tb, M, N, K, e));
    }
    ANN_CUDA(cudaGetLastError());
    return ANN_OK;
}

int grid1d(size_t n, int num_sms) { return (int)std::min<size_t>((n + 255) / 256, (size_t)num_sms * 8); }

ann_status transpose(const __nv_bfloat16 *in, __nv_bfloat16 *out, uint32_t R, uint32_t C, cudaStream_t st)
{
    dim3 grid((C + 31) / 32, (R + 31) / 32), block(32, 8);
    transpose_bf16_kernel<<<grid, block, 0, st>>>(in, out, R, C);
    ANN_CUDA(cudaGetLastError());
    return ANN_OK;
}

// Training-only buffers for batches of up to train_cap rows (grown once).
ann_status ensure_train_buffers(ann_mlp *m, uint32_t n)
{
    if (n <= m->train_cap) return ANN_OK;
    __nv_bfloat16 **bf[] = {&m->xT, &m->h1T, &m->h2T, &m->dzb, &m->dzT, &m->da2b, &m->da2T, &m->da1T};
    float **fp[] = {&m->z, &m->dh, &m->dm, &m->xbat};
    for (auto p : bf) if (*p) { cudaFree(*p); *p = nullptr; }
    for (auto p : fp) if (*p) { cudaFree(*p); *p = nullptr; }
    if (m->ybat) { cudaFree(m->ybat); m->ybat = nullptr; }
    m->train_cap = 0;
    const size_t B = n;
    cudaError_t e = cudaSuccess;
    auto al = [&](void **p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
    al((void **)&m->xT, B * m->d * 2);
    al((void **)&m->h1T, B * m->h1 * 2);
    al((void **)&m->h2T, B * m->h2 * 2);
    al((void **)&m->dzb, B * m->out * 2);
    al((void **)&m->dzT, B * m->out * 2);
    al((void **)&m->da2b, B * m->h2 * 2);
    al((void **)&m->da2T, B * m->h2 * 2);
    al((void **)&m->da1T, B * m->h1 * 2);
    al((void **)&m->z, B * m->out * 4);
    al((void **)&m->dh, B * std::max(m->h1, m->h2) * 4);
    al((void **)&m->dm, B * std::max(m->h1, m->h2) * 4);
    al((void **)&m->xbat, B * m->d * 4);
    al((void **)&m->ybat, B * 4);
    if (e != cudaSuccess) return cuda_fail(e, "MLP training buffers");
    m->train_cap = n;
    return ANN_OK;
}

ann_status forward(ann_mlp *m, const float *x, uint32_t n, cudaStream_t st, int logits_epi, float *logits,
                   float *part, uint32_t ntiles)
{
    input_bf16_kernel<<<grid1d((size_t)n * m->d, m->num_sms), 256, 0, st>>>(x, m->mean, m->inv_std, m->xb, n, m->d);
    ANN_CUDA(cudaGetLastError());
    EpiArgs e{};
    e.err = m->d_error;
    e.bias = m->b[0]; e.cb = m->h1b; e.ldc = m->h1;
    ann_status s = gemm<EPI_BIAS_RELU_BF16>(m->xb, m->Wb[0], n, m->h1, m->d, e, st);
    if (s != ANN_OK) return s;
    e.bias = m->b[1]; e.cb = m->h2b; e.ldc = m->h2;
    s = gemm<EPI_BIAS_RELU_BF16>(m->h1b, m->Wb[1], n, m->h2, m->h1, e, st);
    if (s != ANN_OK) return s;
    e.bias = m->b[2]; e.cb = nullptr;
    if (logits_epi == EPI_BIAS_F32) {
        e.c = logits; e.ldc = m->out;
        return gemm<EPI_BIAS_F32>(m->h2b, m->Wb[2], n, m->out, m->h2, e, st);
    }
    e.part = part; e.ntiles = ntiles;
    return gemm<EPI_TOPP>(m->h2b, m->Wb[2], n, m->out, m->h2, e, st);
}

void mlp_free_all(ann_mlp *m)
{
    for (int l = 0; l < 3; ++l) {
        void *p[] = {m->W[l], m->b[l], m->mW[l], m->vW[l], m->mb[l], m->vb[l], m->gW[l], m->gb[l], m->Wb[l], m->WT[l]};
        for (void *x : p) if (x) cudaFree(x);
    }
    void *q[] = {m->xb, m->xT, m->h1b, m->h1T, m->h2b, m->h2T, m->dzb, m->dzT, m->da2b, m->da2T, m->da1T,
                 m->z, m->dh, m->dm, m->loss, m->part, m->d_error, m->xbat, m->ybat, m->perm, m->epoch_loss,
                 m->mean, m->inv_std};
    for (void *x : q) if (x) cudaFree(x);
}

}  // namespace

extern "C" {

ann_status ann_mlp_create(int device, uint32_t in_dim, uint32_t hidden1, uint32_t hidden2, uint32_t out_dim,
                          uint32_t max_batch, ann_mlp **out)
{
    if (!out) { set_error("ann_mlp_create: out is NULL"); return ANN_EINVAL; }
    *out = nullptr;
    if (!in_dim || !hidden1 || !hidden2 || !out_dim || !max_batch || in_dim % 8 || hidden1 % 8 || hidden2 % 8 ||
        out_dim % 8 || max_batch % 8) {
        set_error("ann_mlp_create: sizes must be positive multiples of 8");
        return ANN_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        set_error("ann_mlp_create: no CUDA device %d", device);
        return ANN_EDEVICE;
    }
    int prev = -1;
    {
        const ann_status ds = enter_device(device, &prev, "ann_mlp_create");
        if (ds != ANN_OK) return ds;
    }
    ann_mlp *m = new ann_mlp();
    m->device = device;
    m->d = in_dim; m->h1 = hidden1; m->h2 = hidden2; m->out = out_dim; m->maxb = max_batch;
    cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, device);
    const uint32_t rows[3] = {hidden1, hidden2, out_dim}, cols[3] = {in_dim, hidden1, hidden2};
    cudaError_t e = cudaSuccess;
    auto al = [&](void **p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes); };
    for (int l = 0; l < 3; ++l) {
        const size_t nw = (size_t)rows[l] * cols[l];
        al((void **)&m->W[l], nw * 4); al((void **)&m->mW[l], nw * 4); al((void **)&m->vW[l], nw * 4);
        al((void **)&m->gW[l], nw * 4); al((void **)&m->Wb[l], nw * 2); al((void **)&m->WT[l], nw * 2);
        al((void **)&m->b[l], rows[l] * 4); al((void **)&m->mb[l], rows[l] * 4); al((void **)&m->vb[l], rows[l] * 4);
        al((void **)&m->gb[l], rows[l] * 4);
    }
    // activations of the forward pass, for up to max_batch rows; the
    // training-only buffers are allocated on the first training step
    const size_t B = max_batch;
    al((void **)&m->xb, B * in_dim * 2);
    al((void **)&m->h1b, B * hidden1 * 2);
    al((void **)&m->h2b, B * hidden2 * 2);
    al((void **)&m->loss, 64);
    al((void **)&m->d_error, 64);
    al((void **)&m->epoch_loss, 4096 * 4);
    al((void **)&m->mean, (size_t)in_dim * 4);
    al((void **)&m->inv_std, (size_t)in_dim * 4);
    if (e == cudaSuccess) {
        const std::vector<float> ones(in_dim, 1.0f);
        e = cudaMemcpy(m->inv_std, ones.data(), (size_t)in_dim * 4, cudaMemcpyHostToDevice);
    }
    leave_device(device, prev);
    if (e != cudaSuccess) {
        mlp_free_all(m);
        delete m;
        return cuda_fail(e, "ann_mlp_create");
    }
    *out = m;
    return ANN_OK;
}

ann_status ann_mlp_free(ann_mlp *m)
{
    if (!m) return ANN_OK;
    int prev = -1;
    const bool switched = enter_device(m->device, &prev, "ann_mlp_free") == ANN_OK;   // frees best-effort
    mlp_free_all(m);
    if (switched) leave_device(m->device, prev);
    delete m;
    return ANN_OK;
}

// Host FP32 parameters in; resets the optimizer state and step count.
ann_status ann_mlp_set_params(ann_mlp *m, const float *W1, const float *b1, const float *W2, const float *b2,
                              const float *W3, const float *b3)
{
    if (!m || !W1 || !b1 || !W2 || !b2 || !W3 || !b3) { set_error("ann_mlp_set_params: NULL argument"); return ANN_EINVAL; }
    int prev = -1;
    {
        const ann_status ds = enter_device(m->device, &prev, "ann_mlp_set_params");
        if (ds != ANN_OK) return ds;
    }
    const float *Ws[3] = {W1, W2, W3}, *bs[3] = {b1, b2, b3};
    const uint32_t rows[3] = {m->h1, m->h2, m->out}, cols[3] = {m->d, m->h1, m->h2};
    ann_status s = ANN_OK;
    for (int l = 0; l < 3 && s == ANN_OK; ++l) {
        const size_t nw = (size_t)rows[l] * cols[l];
        cudaError_t e = cudaMemcpy(m->W[l], Ws[l], nw * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(m->b[l], bs[l], rows[l] * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(m->mW[l], 0, nw * 4);
        if (e == cudaSuccess) e = cudaMemset(m->vW[l], 0, nw * 4);
        if (e == cudaSuccess) e = cudaMemset(m->mb[l], 0, rows[l] * 4);
        if (e == cudaSuccess) e = cudaMemset(m->vb[l], 0, rows[l] * 4);
        if (e != cudaSuccess) { s = cuda_fail(e, "ann_mlp_set_params"); break; }
        to_bf16_kernel<<<grid1d(nw, m->num_sms), 256>>>(m->W[l], m->Wb[l], nw);
        if (l > 0) s = transpose(m->Wb[l], m->WT[l], rows[l], cols[l], 0);
    }
    m->step = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (s == ANN_OK && e != cudaSuccess) s = cuda_fail(e, "ann_mlp_set_params");
    leave_device(m->device, prev);
    return s;
}

// Host copies of the FP32 parameters (which = 0) or of the last step's
// gradients (which = 1), each pointer NULL to skip.
ann_status ann_mlp_get(const ann_mlp *m, int which, float *W1, float *b1, float *W2, float *b2, float *W3, float *b3)
{
    if (!m || (which != 0 && which != 1)) { set_error("ann_mlp_get: bad arguments"); return ANN_EINVAL; }
    int prev = -1;
    {
        const ann_status ds = enter_device(m->device, &prev, "ann_mlp_get");
        if (ds != ANN_OK) return ds;
    }
    float *Ws[3] = {W1, W2, W3}, *bs[3] = {b1, b2, b3};
    const uint32_t rows[3] = {m->h1, m->h2, m->out}, cols[3] = {m->d, m->h1, m->h2};
    ann_status s = ANN_OK;
    cudaDeviceSynchronize();
    for (int l = 0; l < 3; ++l) {
        cudaError_t e = cudaSuccess;
        if (Ws[l]) e = cudaMemcpy(Ws[l], which ? m->gW[l] : m->W[l], (size_t)rows[l] * cols[l] * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && bs[l]) e = cudaMemcpy(bs[l], which ? m->gb[l] : m->b[l], rows[l] * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { s = cuda_fail(e, "ann_mlp_get"); break; }
    }
    leave_device(m->device, prev);
    return s;
}

// Per-dimension input standardisation (host arrays of in_dim floats; both
// NULL restores the identity: mean 0, inv_std 1).
ann_status ann_mlp_set_input_norm(ann_mlp *m, const float *mean, const float *inv_std)
{
    if (!m || (!mean) != (!inv_std)) { set_error("ann_mlp_set_input_norm: bad arguments"); return ANN_EINVAL; }
    std::vector<float> mu(m->d, 0.0f), is(m->d, 1.0f);
    if (mean) {
        for (uint32_t i = 0; i < m->d; ++i) {
            if (!std::isfinite(mean[i]) || !std::isfinite(inv_std[i])) {
                set_error("ann_mlp_set_input_norm: non-finite value at %u", i);
                return ANN_EINVAL;
            }
            mu[i] = mean[i];
            is[i] = inv_std[i];
        }
    }
    int prev = -1;
    {
        const ann_status ds = enter_device(m->device, &prev, "ann_mlp_set_input_norm");
        if (ds != ANN_OK) return ds;
    }
    cudaError_t e = cudaMemcpy(m->mean, mu.data(), (size_t)m->d * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->inv_std, is.data(), (size_t)m->d * 4, cudaMemcpyHostToDevice);
    leave_device(m->device, prev);
    return e == cudaSuccess ? ANN_OK : cuda_fail(e, "ann_mlp_set_input_norm");
}

// Standardisation statistics of n device queries (n x in_dim FP32): per
// dimension the mean and 1 / std (population std, FP64 on the device), with
// std floored at 1e-6 of the largest; installed as the input standardisation.
// Synchronous on `stream`.
ann_status ann_mlp_fit_input_norm(ann_mlp *m, const float *x, uint32_t n, void *stream)
{
    if (!m || !x || n == 0) { set_error("ann_mlp_fit_input_norm: NULL argument or no rows"); return ANN_EINVAL; }
    int prev = -1;
    {
        const ann_status ds = enter_device(m->device, &prev, "ann_mlp_fit_input_norm");
        if (ds != ANN_OK) return ds;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t d = m->d, rows_per_chunk = 512;
    const uint32_t chunks = (n + rows_per_chunk - 1) / rows_per_chunk;
    double *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, ((size_t)chunks * d + 2 * (size_t)d) * sizeof(double));
    if (e == cudaSuccess) {
        double *partial = buf, *mean = buf + (size_t)chunks * d, *var = mean + d;
        const dim3 grid(chunks, (d + 127) / 128);
        col_partial_kernel<<<grid, 128, 0, st>>>(x, n, d, rows_per_chunk, nullptr, partial);
        col_finish_kernel<<<(d + 127) / 128, 128, 0, st>>>(partial, chunks, d, n, mean);
        col_partial_kernel<<<grid, 128, 0, st>>>(x, n, d, rows_per_chunk, mean, partial);
        col_finish_kernel<<<(d + 127) / 128, 128, 0, st>>>(partial, chunks, d, n, var);
        norm_finish_kernel<<<1, 1024, 0, st>>>(mean, var, d, m->mean, m->inv_std);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(buf);
    }
    leave_device(m->device, prev);
    return e == cudaSuccess ? ANN_OK : cuda_fail(e, "ann_mlp_fit_input_norm");
}

// The confidence threshold tau: the value of 0-based rank
// floor(min(fallback, 1) * (n - 1)) among the n device values pmax in
// ascending order (numpy's "lower" quantile); 0 when fallback <= 0 or n = 0.
// Written to *tau on the host (synchronous on `stream`).
ann_status ann_mlp_confidence_threshold(ann_mlp *m, const float *pmax, uint32_t n, double fallback, float *tau,
                                        void *stream)
{
    if (!m || !tau || (n && !pmax) || !(fallback == fallback)) {
        set_error("ann_mlp_confidence_threshold: NULL argument or NaN fallback");
        return ANN_EINVAL;
    }
    *tau = 0.0f;
    if (n == 0 || fallback <= 0.0) return ANN_OK;
    const double q = fallback < 1.0 ? fallback : 1.0;
    const uint32_t rank = (uint32_t)std::floor(q * (double)(n - 1));
    int prev = -1;
    {
        const ann_status ds = enter_device(m->device, &prev, "ann_mlp_confidence_threshold");
        if (ds != ANN_OK) return ds;
    }
    cudaStream_t st = (cudaStream_t)stream;
    float *dv = nullptr;
    cudaError_t e = cudaMalloc(&dv, 16);
    if (e == cudaSuccess) {
        select_rank_kernel<<<1, 1024, 0, st>>>(pmax, n, rank, dv);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(tau, dv, sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(dv);
    }
    leave_device(m->device, prev);
    return e == cudaSuccess ? ANN_OK : cuda_fail(e, "ann_mlp_confidence_threshold");
}

// Host copies of the input standardisation (in_dim floats each).
ann_status ann_mlp_get_input_norm(const ann_mlp *m, float *mean, float *inv_std)
{
    if (!m || !mean || !inv_std) { set_error("ann_mlp_get_input_norm: NULL argument"); return ANN_EINVAL; }
    int prev = -1;
    {
        const ann_status ds = enter_device(m->device, &prev, "ann_mlp_get_input_norm");
        if (ds != ANN_OK) return ds;
    }
    cudaError_t e = cudaMemcpy(mean, m->mean, (size_t)m->d * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(inv_std, m->inv_std, (size_t)m->d * 4, cudaMemcpyDeviceToHost);
    leave_device(m->device, prev);
    return e == cudaSuccess ? ANN_OK : cuda_fail(e, "ann_mlp_get_input_norm");
}

// Logits z = MLP(x) (device x: n x in_dim FP32; device logits: n x out_dim).
ann_status ann_mlp_forward(ann_mlp *m, const float *x, uint32_t n, float *logits, void *stream)
{
    if (!m || !x || !logits) { set_error("ann_mlp_forward: NULL argument"); return ANN_EINVAL; }
    if (n > m->maxb) { set_error("ann_mlp_forward: n = %u > max_batch %u", n, m->maxb); return ANN_EINVAL; }
    if (n == 0) return ANN_OK;
    int prev = -1;
    {
        const ann_status ds = enter_device(m->device, &prev, "ann_mlp_forward");
        if (ds != ANN_OK) return ds;
    }
    ann_status s = forward(m, x, n, (cudaStream_t)stream, EPI_BIAS_F32, logits, nullptr, 0);
    leave_device(m->device, prev);
    return s;
}

// One AdamW step on a minibatch (device x: n x in_dim, labels: n ghost
// indices < out_dim); writes the mean loss of the batch to *loss_out (device,
// may be NULL). Gradients stay available to ann_mlp_get(which = 1).
ann_status ann_mlp_train_step(ann_mlp *m, const float *x, const uint32_t *labels, uint32_t n, float lr, float beta1,
                              float beta2, float eps, float weight_decay, float *loss_out, void *stream)
{
    if (!m || !x || !labels) { set_error("ann_mlp_train_step: NULL argument"); return ANN_EINVAL; }
    if (n == 0 || n > m->maxb || n % 8) {
        set_error("ann_mlp_train_step: batch %u must be a positive multiple of 8 <= %u", n, m->maxb);
        return ANN_EINVAL;
    }
    int prev = -1;
    {
        const ann_status ds = enter_device(m->device, &prev, "ann_mlp_train_step");
        if (ds != ANN_OK) return ds;
    }
    cudaStream_t st = (cudaStream_t)stream;
    ann_status s = ensure_train_buffers(m, n);
    auto chk = [&]() { cudaError_t e = cudaGetLastError(); if (e != cudaSuccess && s == ANN_OK) s = cuda_fail(e, "ann_mlp_train_step"); };
    if (s == ANN_OK && cudaMemsetAsync(m->loss, 0, 4, st) != cudaSuccess) s = ANN_ECUDA;
    if (s == ANN_OK) s = forward(m, x, n, st, EPI_BIAS_F32, m->z, nullptr, 0);
    const dim3 tb(32, 8);
    EpiArgs e{};
    e.err = m->d_error;
    if (s == ANN_OK) {
        softmax_ce_kernel<<<(n + 7) / 8, 256, 0, st>>>(m->z, labels, n, m->out, m->loss);
        chk();
        post_grad_kernel<<<dim3((m->out + 31) / 32, (n + 31) / 32), tb, 0, st>>>(m->z, nullptr, nullptr, m->dzb, m->dzT, n, m->out);
        chk();
        colsum_kernel<<<(m->out + 255) / 256, 256, 0, st>>>(m->z, m->gb[2], n, m->out);
        chk();
    }
    if (s == ANN_OK) s = transpose(m->h2b, m->h2T, n, m->h2, st);
    e.c = m->gW[2]; e.ldc = m->h2;
    if (s == ANN_OK) s = gemm<EPI_F32>(m->dzT, m->h2T, m->out, m->h2, n, e, st);
    e.c = m->dh; e.ldc = m->h2;
    if (s == ANN_OK) s = gemm<EPI_F32>(m->dzb, m->WT[2], n, m->h2, m->out, e, st);
    if (s == ANN_OK) {
        post_grad_kernel<<<dim3((m->h2 + 31) / 32, (n + 31) / 32), tb, 0, st>>>(m->dh, m->h2b, m->dm, m->da2b, m->da2T, n, m->h2);
        chk();
        colsum_kernel<<<(m->h2 + 255) / 256, 256, 0, st>>>(m->dm, m->gb[1], n, m->h2);
        chk();
    }
    if (s == ANN_OK) s = transpose(m->h1b, m->h1T, n, m->h1, st);
    e.c = m->gW[1]; e.ldc = m->h1;
    if (s == ANN_OK) s = gemm<EPI_F32>(m->da2T, m->h1T, m->h2, m->h1, n, e, st);
    e.c = m->dh; e.ldc = m->h1;
    if (s == ANN_OK) s = gemm<EPI_F32>(m->da2b, m->WT[1], n, m->h1, m->h2, e, st);
    if (s == ANN_OK) {
        post_grad_kernel<<<dim3((m->h1 + 31) / 32, (n + 31) / 32), tb, 0, st>>>(m->dh, m->h1b, m->dm, nullptr, m->da1T, n, m->h1);
        chk();
        colsum_kernel<<<(m->h1 + 255) / 256, 256, 0, st>>>(m->dm, m->gb[0], n, m->h1);
        chk();
    }
    if (s == ANN_OK) s = transpose(m->xb, m->xT, n, m->d, st);
    e.c = m->gW[0]; e.ldc = m->d;
    if (s == ANN_OK) s = gemm<EPI_F32>(m->da1T, m->xT, m->h1, m->d, n, e, st);
    if (s == ANN_OK) {
        m->step++;
        AdamHP h{lr, beta1, beta2, eps, weight_decay, (float)(1.0 - std::pow((double)beta1, (double)m->step)),
                 (float)(1.0 - std::pow((double)beta2, (double)m->step))};
        const uint32_t rows[3] = {m->h1, m->h2, m->out}, cols[3] = {m->d, m->h1, m->h2};
        for (int l = 0; l < 3; ++l) {
            const size_t nw = (size_t)rows[l] * cols[l];
            adamw_kernel<<<grid1d(nw, m->num_sms), 256, 0, st>>>(m->W[l], m->gW[l], m->mW[l], m->vW[l], m->Wb[l], nw, h);
            adamw_kernel<<<grid1d(rows[l], m->num_sms), 256, 0, st>>>(m->b[l], m->gb[l], m->mb[l], m->vb[l], nullptr, rows[l], h);
            chk();
            if (l > 0 && s == ANN_OK) s = transpose(m->Wb[l], m->WT[l], rows[l], cols[l], st);
        }
    }
    if (s == ANN_OK && loss_out) {
        cudaError_t ce = cudaMemcpyAsync(loss_out, m->loss, 4, cudaMemcpyDeviceToDevice, st);
        if (ce != cudaSuccess) s = cuda_fail(ce, "ann_mlp_train_step loss");
    }
    leave_device(m->device, prev);
    return s;
}

// Entry prediction (fused): the top-P ghost indices per query by logit
// (ties: smaller index), and the largest softmax probability; a query whose
// probability is below tau gets ANN_INVALID_ID as its first seed, which
// ann_search treats as "fall back to random ghost seeds". P <= 8.
ann_status ann_mlp_predict(ann_mlp *m, const float *x, uint32_t n, uint32_t P, float tau, uint32_t *seeds,
                           float *pmax, void *stream)
{
    if (!m || !x || !seeds || P == 0 || P > TOPP || P > m->out) {
        set_error("ann_mlp_predict: bad arguments (1 <= P <= %d)", TOPP);
        return ANN_EINVAL;
    }
    if (n == 0) return ANN_OK;
    int prev = -1;
    {
        const ann_status ds = enter_device(m->device, &prev, "ann_mlp_predict");
        if (ds != ANN_OK) return ds;
    }
    cudaStream_t st = (cudaStream_t)stream;
    ann_status s = ANN_OK;
    for (uint32_t r0 = 0; r0 < n && s == ANN_OK; r0 += m->maxb) {
        const uint32_t rows = std::min(m->maxb, n - r0);
        const uint32_t ntiles = topp_slots(rows, m->out, (uint32_t)m->num_sms, gemm_mode(EPI_TOPP, m->h2));
        const size_t need = (size_t)rows * ntiles * (2 * TOPP + 2) * 4;
        if (need > m->part_cap) {
            if (m->part) cudaFree(m->part);
            m->part = nullptr;
            m->part_cap = 0;
            cudaError_t e = cudaMalloc(&m->part, need);
            if (e != cudaSuccess) { s = cuda_fail(e, "ann_mlp_predict"); break; }
            m->part_cap = need;
        }
        // slots no CTA writes read as empty (ids 0xFFFFFFFF, exp-sum NaN)
        if (cudaError_t me = cudaMemsetAsync(m->part, 0xFF, need, st); me != cudaSuccess)
            s = cuda_fail(me, "ann_mlp_predict");
        if (s == ANN_OK) s = forward(m, x + (size_t)r0 * m->d, rows, st, EPI_TOPP, nullptr, m->part, ntiles);
        if (s == ANN_OK) {
            topp_merge_kernel<<<(rows + 3) / 4, 128, 0, st>>>(m->part, rows, ntiles, P, tau, seeds + (size_t)r0 * P,
                                                               pmax ? pmax + r0 : nullptr);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) s = cuda_fail(e, "topp_merge_kernel");
        }
    }
    leave_device(m->device, prev);
    return s;
}

// Epochs of minibatch AdamW over (x, labels) (device, n rows): each epoch
// visits the rows in a fresh order (Fisher-Yates driven by splitmix64 of
// (seed, epoch)), in batches of `batch` rows (a multiple of 8); a final
// partial batch is cut down to a multiple of 8. epoch_loss (host, `epochs`
// floats, may be NULL) receives each epoch's mean batch loss. Synchronous.
ann_status ann_mlp_train_epochs(ann_mlp *m, const float *x, const uint32_t *labels, uint32_t n, uint32_t batch,
                                uint32_t epochs, float lr, float beta1, float beta2, float eps, float weight_decay,
                                uint64_t seed, float *epoch_loss, void *stream)
{
    if (!m || !x || !labels || batch == 0 || batch % 8 || batch > m->maxb || epochs > 4096 || n < 8) {
        set_error("ann_mlp_train_epochs: bad arguments (batch a multiple of 8 <= max_batch, n >= 8, epochs <= 4096)");
        return ANN_EINVAL;
    }
    int prev = -1;
    {
        const ann_status ds = enter_device(m->device, &prev, "ann_mlp_train_epochs");
        if (ds != ANN_OK) return ds;
    }
    cudaStream_t st = (cudaStream_t)stream;
    ann_status s = ANN_OK;
    if (n > m->perm_cap) {
        if (m->perm) cudaFree(m->perm);
        m->perm = nullptr;
        m->perm_cap = 0;
        cudaError_t e = cudaMalloc(&m->perm, (size_t)n * 4);
        if (e != cudaSuccess) s = cuda_fail(e, "ann_mlp_train_epochs");
        else m->perm_cap = n;
    }
    if (s == ANN_OK) s = ensure_train_buffers(m, batch);
    std::vector<uint32_t> perm(n);
    if (s == ANN_OK && cudaMemsetAsync(m->epoch_loss, 0, (size_t)epochs * 4, st) != cudaSuccess) s = ANN_ECUDA;
    for (uint32_t ep = 0; ep < epochs && s == ANN_OK; ++ep) {
        for (uint32_t i = 0; i < n; ++i) perm[i] = i;
        const uint64_t key = mix64(seed ^ mix64(ep));
        for (uint32_t i = n - 1; i > 0; --i) {
            const uint32_t j = (uint32_t)(mix64(key ^ i) % (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        cudaError_t e = cudaMemcpyAsync(m->perm, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // perm is reused next epoch
        if (e != cudaSuccess) { s = cuda_fail(e, "ann_mlp_train_epochs"); break; }
        uint32_t steps = 0;
        for (uint32_t b0 = 0; b0 + 8 <= n; b0 += batch) ++steps;
        for (uint32_t b0 = 0; b0 + 8 <= n && s == ANN_OK; b0 += batch) {
            uint32_t rows = std::min(batch, n - b0) & ~7u;
            gather_batch_kernel<<<rows, 128, 0, st>>>(x, labels, m->perm + b0, rows, m->d, m->xbat, m->ybat);
            e = cudaGetLastError();
            if (e != cudaSuccess) { s = cuda_fail(e, "gather_batch_kernel"); break; }
            s = ann_mlp_train_step(m, m->xbat, m->ybat, rows, lr, beta1, beta2, eps, weight_decay, nullptr, stream);
            if (s == ANN_OK) accumulate_kernel<<<1, 32, 0, st>>>(m->epoch_loss + ep, m->loss, 1.0f / (float)steps);
        }
    }
    if (s == ANN_OK && epoch_loss) {
        cudaError_t e = cudaMemcpyAsync(epoch_loss, m->epoch_loss, (size_t)epochs * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(e, "ann_mlp_train_epochs");
    }
    leave_device(m->device, prev);
    return s;
}

// Synchronise `stream` and report (then clear) the MLP's device error word.
ann_status ann_mlp_sync(ann_mlp *m, void *stream)
{
    if (!m) { set_error("ann_mlp_sync: NULL"); return ANN_EINVAL; }
    int prev = -1;
    {
        const ann_status ds = enter_device(m->device, &prev, "ann_mlp_sync");
        if (ds != ANN_OK) return ds;
    }
    ann_status s = ANN_OK;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, m->d_error, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) s = cuda_fail(e, "ann_mlp_sync");
    else if (err) {
        cudaMemset(m->d_error, 0, 4);
        set_error("a bounded device wait ran out in an MLP kernel");
        s = ANN_ETIMEOUT;
    }
    leave_device(m->device, prev);
    return s;
}


// Parameter file: magic, four uint32 sizes, then W1 b1 W2 b2 W3 b3 and the
// input standardisation (mean, inv_std) as FP32;
// both hosts this builds for are little-endian, so the bytes go out as they are.
// Parameter files: "ANNMLP01" (parameters and input standardisation) and
// "ANNMLP02" (the same, then the AdamW state: the step count and the first
// and second moments of every parameter array). Saving writes version 02.
static const char kMlpMagic1[8] = {'A', 'N', 'N', 'M', 'L', 'P', '0', '1'};
static const char kMlpMagic2[8] = {'A', 'N', 'N', 'M', 'L', 'P', '0', '2'};

namespace {

// Copy one device array to the host (or the host to the device).
bool copy_d2h(std::vector<float> &h, const float *d, size_t n)
{
    h.resize(n);
    return cudaMemcpy(h.data(), d, n * 4, cudaMemcpyDeviceToHost) == cudaSuccess;
}

bool copy_h2d(float *d, const std::vector<float> &h)
{
    return cudaMemcpy(d, h.data(), h.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess;
}

}  // namespace

ann_status ann_mlp_save(const ann_mlp *m, const char *path)
{
    if (!m || !path) { set_error("ann_mlp_save: NULL argument"); return ANN_EINVAL; }
    const uint32_t dims[4] = {m->d, m->h1, m->h2, m->out};
    std::vector<float> W[3], b[3];
    const uint32_t rows[3] = {m->h1, m->h2, m->out}, cols[3] = {m->d, m->h1, m->h2};
    for (int l = 0; l < 3; ++l) { W[l].resize((size_t)rows[l] * cols[l]); b[l].resize(rows[l]); }
    ann_status s = ann_mlp_get(m, 0, W[0].data(), b[0].data(), W[1].data(), b[1].data(), W[2].data(), b[2].data());
    std::vector<float> mu(m->d), is(m->d);
    if (s == ANN_OK) s = ann_mlp_get_input_norm(m, mu.data(), is.data());
    if (s != ANN_OK) return s;
    // optimizer moments, in the order mW, vW, mb, vb per layer
    std::vector<float> opt[12];
    {
        int prev = -1;
        const ann_status ds = enter_device(m->device, &prev, "ann_mlp_save");
        if (ds != ANN_OK) return ds;
        bool ok = true;
        for (int l = 0; l < 3 && ok; ++l) {
            const size_t nw = (size_t)rows[l] * cols[l];
            ok = copy_d2h(opt[4 * l], m->mW[l], nw) && copy_d2h(opt[4 * l + 1], m->vW[l], nw) &&
                 copy_d2h(opt[4 * l + 2], m->mb[l], rows[l]) && copy_d2h(opt[4 * l + 3], m->vb[l], rows[l]);
        }
        leave_device(m->device, prev);
        if (!ok) { set_error("ann_mlp_save: reading the optimizer state failed"); return ANN_ECUDA; }
    }
    FILE *f = std::fopen(path, "wb");
    if (!f) { set_error("ann_mlp_save: cannot open %s", path); return ANN_EIO; }
    bool ok = std::fwrite(kMlpMagic2, 1, 8, f) == 8 && std::fwrite(dims, 4, 4, f) == 4;
    for (int l = 0; l < 3 && ok; ++l)
        ok = std::fwrite(W[l].data(), 4, W[l].size(), f) == W[l].size() &&
             std::fwrite(b[l].data(), 4, b[l].size(), f) == b[l].size();
    ok = ok && std::fwrite(mu.data(), 4, m->d, f) == m->d && std::fwrite(is.data(), 4, m->d, f) == m->d;
    const uint32_t step = m->step;
    ok = ok && std::fwrite(&step, 4, 1, f) == 1;
    for (int i = 0; i < 12 && ok; ++i) ok = std::fwrite(opt[i].data(), 4, opt[i].size(), f) == opt[i].size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) { set_error("ann_mlp_save: write to %s failed", path); return ANN_EIO; }
    return ANN_OK;
}

ann_status ann_mlp_load(const char *path, int device, uint32_t max_batch, ann_mlp **out)
{
    if (!path || !out) { set_error("ann_mlp_load: NULL argument"); return ANN_EINVAL; }
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) { set_error("ann_mlp_load: cannot open %s", path); return ANN_EIO; }
    char magic[8];
    uint32_t dims[4];
    if (std::fread(magic, 1, 8, f) != 8 || std::fread(dims, 4, 4, f) != 4) {
        std::fclose(f);
        set_error("ann_mlp_load: %s is too short", path);
        return ANN_EIO;
    }
    const bool v2 = std::memcmp(magic, kMlpMagic2, 8) == 0;
    if (!v2 && std::memcmp(magic, kMlpMagic1, 8) != 0) {
        std::fclose(f);
        set_error("ann_mlp_load: %s is not an MLP parameter file", path);
        return ANN_EINVAL;
    }
    for (uint32_t v : dims)
        if (!v || v % 8 || v > (1u << 24)) {
            std::fclose(f);
            set_error("ann_mlp_load: %s has invalid sizes", path);
            return ANN_EINVAL;
        }
    const uint32_t rows[3] = {dims[1], dims[2], dims[3]}, cols[3] = {dims[0], dims[1], dims[2]};
    std::vector<float> W[3], b[3];
    bool ok = true;
    for (int l = 0; l < 3 && ok; ++l) {
        W[l].resize((size_t)rows[l] * cols[l]);
        b[l].resize(rows[l]);
        ok = std::fread(W[l].data(), 4, W[l].size(), f) == W[l].size() &&
             std::fread(b[l].data(), 4, b[l].size(), f) == b[l].size();
    }
    std::vector<float> mu(dims[0]), is(dims[0]);
    ok = ok && std::fread(mu.data(), 4, dims[0], f) == dims[0] && std::fread(is.data(), 4, dims[0], f) == dims[0];
    uint32_t step = 0;
    std::vector<float> opt[12];
    if (v2 && ok) {
        ok = std::fread(&step, 4, 1, f) == 1;
        for (int l = 0; l < 3 && ok; ++l) {
            const size_t sz[4] = {(size_t)rows[l] * cols[l], (size_t)rows[l] * cols[l], rows[l], rows[l]};
            for (int j = 0; j < 4 && ok; ++j) {
                opt[4 * l + j].resize(sz[j]);
                ok = std::fread(opt[4 * l + j].data(), 4, sz[j], f) == sz[j];
            }
        }
    }
    std::fclose(f);
    if (!ok) { set_error("ann_mlp_load: %s is too short", path); return ANN_EIO; }
    ann_mlp *m = nullptr;
    ann_status s = ann_mlp_create(device, dims[0], dims[1], dims[2], dims[3], max_batch, &m);
    if (s == ANN_OK) s = ann_mlp_set_params(m, W[0].data(), b[0].data(), W[1].data(), b[1].data(), W[2].data(), b[2].data());
    if (s == ANN_OK) s = ann_mlp_set_input_norm(m, mu.data(), is.data());
    if (s == ANN_OK && v2) {
        // set_params zeroed the moments and the step: restore the saved ones
        int prev = -1;
        s = enter_device(device, &prev, "ann_mlp_load");
        if (s == ANN_OK) {
            bool ok2 = true;
            for (int l = 0; l < 3 && ok2; ++l)
                ok2 = copy_h2d(m->mW[l], opt[4 * l]) && copy_h2d(m->vW[l], opt[4 * l + 1]) &&
                      copy_h2d(m->mb[l], opt[4 * l + 2]) && copy_h2d(m->vb[l], opt[4 * l + 3]);
            leave_device(device, prev);
            if (!ok2) s = cuda_fail(cudaGetLastError(), "ann_mlp_load: restoring the optimizer state");
            m->step = step;
        }
    }
    if (s != ANN_OK) { ann_mlp_free(m); return s; }
    *out = m;
    return ANN_OK;
}

}  // extern "C"
