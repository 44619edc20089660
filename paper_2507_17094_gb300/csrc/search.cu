// Batched graph beam search on sm_103a (Section 2.2 Steps 1-4), with ghost
// staging (Section 3.2.2) and direction-guided selection (Section 3.3.2).
//
// Design (GB300-first, not the paper's 32-thread-block CAGRA kernel):
//   - persistent CTAs of 4 warps; each warp owns one query at a time and pulls
//     the next query index from a device counter, so long and short searches
//     balance across the 152 SMs;
//   - per warp, a small shared-memory region (about 9.5 KB for itopk 32 on
//     96-d FP32) holds the query, the priority queue, the candidate list, the
//     parents' adjacency / direction / vector rows and 16 staged rows, so 24
//     warps share an SM and hide each other's memory latency;
//   - the visited set of each warp is a 4,096-entry table in global memory
//     (L2-resident, 16 KB per warp), probed with one atomicCAS per lane; the
//     ghost stage of a small ghost set uses an exact shared-memory bitmap;
//   - every random global read (adjacency rows, direction rows, vector rows,
//     FP32 rerank rows) is a 1-D TMA bulk copy into shared memory completing
//     on the warp's mbarrier: one instruction per row, all rows of a round in
//     flight together;
//   - distances are computed by a lane pair per row from shared memory, one
//     fused multiply-add per element into four interleaved partial sums, the
//     same FP32 operations as the reference definition, so they agree bit
//     for bit;
//   - DGS needs the query's sign bits relative to each parent; they are
//     recomputed from the parent's row, which arrives in the same bulk-copy
//     round as its adjacency and direction rows (one ballot per 32 dims);
//   - DGS keeps its top n neighbours by a ballot radix select of the score
//     threshold, not by sorting;
//   - the merge works in place: candidates no better than the queue's last
//     entry are dropped first, each survivor's slot is its rank among the
//     candidates plus its insertion point in the queue, and only queue
//     entries behind the first insertion point move;
//   - the hot loop is kept small: with 24 warps per SM at different points
//     of an iteration the kernel is bound by instruction fetch (instruction
//     requests to the GPC cache near 80% of peak), so seeding shares the
//     iteration's code and loops with run-time trip counts are not unrolled
//     ("#pragma unroll 1"; measured +7% on the 1M x 96 workload).
//
// Visited set: open addressing with linear probing over entries id + 1 (0 =
// empty) in the warp's table in global memory, zeroed at the start of each
// query (and at the switch from the ghost to the base graph). A lane claims
// an empty slot with atomicCAS; slots only ever change from empty to an id,
// so a probe run never moves and a lookup that reaches an empty slot has
// proved the id absent (concurrent lanes inserting the same id: one CAS wins,
// the other then finds it). The table is exact between resets. It is reset (and refilled with the
// queue's ids) only when it would pass half full. Forgetting a node that is no
// longer in the queue cannot change the result: its key is larger than the
// queue's current l-th key (which only decreases), so re-evaluating it rejects
// it again. Results therefore equal those of an exact visited set; only the
// work counters can grow (counted in hash_resets).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "ann_internal.cuh"

using namespace ann;

namespace {

constexpr uint32_t kUnexpanded = 0, kPartial = 1, kExpanded = 2;
constexpr uint64_t kGhostTag = 0x67686F7374ull;
constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr uint32_t kMaxDegWords = ANN_MAX_DEGREE / 32;
// Resident 4-warp blocks per SM the register allocation is sized for.
#ifndef ANN_SEARCH_BLOCKS_PER_SM
#define ANN_SEARCH_BLOCKS_PER_SM 6
#endif
constexpr int kSearchBlocksPerSm = ANN_SEARCH_BLOCKS_PER_SM;

// Entries that run the ghost stage first.
__host__ __device__ __forceinline__ bool ghost_entry(uint32_t e)
{
    return e == ANN_ENTRY_GHOST || e == ANN_ENTRY_GIVEN_GHOST;
}
// Entries that read a row of caller-given seeds.
__host__ __device__ __forceinline__ bool given_entry(uint32_t e)
{
    return e == ANN_ENTRY_GIVEN_GHOST || e == ANN_ENTRY_GIVEN_BASE;
}

struct View {
    const uint8_t *codes;
    const float *scales;   // nullptr for FP32
    uint32_t row_bytes;
    const uint32_t *graph;
    uint32_t deg, deg_pad;
    const uint32_t *dir;   // nullptr: no DGS on this graph
    uint32_t n;
};

struct Layout {  // byte offsets inside one warp's shared-memory region
    uint32_t q, bd, bi, bs, cd, ci, cs, adj, dir, prow, par, stage, bar, qp, total;
};

// Ghost sets up to this many nodes get an exact shared-memory bitmap as the
// ghost stage's visited set (2 KB per warp at most).
constexpr uint32_t kGhostBitmapMax = 16384;

struct Args {
    View base, ghost;
    const uint32_t *ghost_ids;
    const uint8_t *x32;
    uint32_t row32_bytes;
    const float *queries;
    uint32_t nq, d, w;
    const uint32_t *given;
    uint32_t *out_ids;
    float *out_dists;
    ann_query_stats *stats;
    QParams qp;
    uint32_t *counter;
    int *err;
    Layout lay;
    uint32_t cap_cand, stage_rows, stage_stride, prow_bytes;
    // the rerank's FP32 rows in the same staging area: rows per round, stride
    uint32_t rr_rows, rr_stride;
    // visited tables: slot_base + warp slot selects one table of 2^vbits
    // entries (tables 2^vstride_bits entries apart)
    uint32_t *vtab;
    uint32_t vbits, vstride_bits, slot_base;
    uint32_t gbm_words;   // > 0: the ghost stage's visited set is a bitmap of this many words
    uint32_t lpr;         // lanes per staged row in the distance step: 2, or 4 for wide rows
    // profile build only: per warp slot, ANN_PROFILE_STAGES x ANN_PROFILE_PHASES
    // cycle counters (slot_base + warp slot selects a row)
    unsigned long long *prof;
};

// Phases of the per-phase clock profile (ann_search_profile); a stage is the
// ghost stage, the base stage, or the rerank and output.
enum Phase : uint32_t { PH_SELECT = 0, PH_DGS, PH_VISIT, PH_GATHER, PH_DIST, PH_MERGE, PH_OTHER };
enum ProfStage : uint32_t { PS_GHOST = 0, PS_BASE, PS_FINISH };
static_assert(PH_OTHER < ANN_PROFILE_PHASES && PS_FINISH < ANN_PROFILE_STAGES, "profile table too small");

__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// (da, ia) < (db, ib) in (distance, id) order. Distances are squared L2,
// never negative nor NaN, and non-negative floats order as their bit
// patterns do, so the key compares as one 64-bit integer (bits, id): two
// integer compares instead of three float and integer ones.
__device__ __forceinline__ bool key_less(float da, uint32_t ia, float db, uint32_t ib)
{
    return (((uint64_t)__float_as_uint(da) << 32) | ia) < (((uint64_t)__float_as_uint(db) << 32) | ib);
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// One element: df = q - x, acc += df * df with a single rounding.
__device__ __forceinline__ void step(float qv, float xv, float &acc)
{
    const float df = __fsub_rn(qv, xv);
    acc = __fmaf_rn(df, df, acc);
}

// Stored value of element i (decoded to FP32).
template <int ST>
__device__ __forceinline__ float stored_elem(const uint8_t *row, uint32_t i, float scale)
{
    if (ST == ANN_F32) return reinterpret_cast<const float *>(row)[i];
    if (ST == ANN_F16) return __fmul_rn(scale, __half2float(reinterpret_cast<const __half *>(row)[i]));
    const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)row[i], __NV_E4M3);
    return __fmul_rn(scale, __half2float(__half(h)));
}

// One element of the distance: acc += (q - stored)^2, the difference
// rounded once. An FP16 row's scale is a power of two, so its stored value
// s * h is exact in FP32 (for every row whose largest |x| is at least 2^-88,
// where s * h stays a normal number) and q - s * h is one fused multiply-add,
// equal to the rounded difference of q and the stored value; E4M3 scales are
// not powers of two, so that stored value is rounded first.
template <int ST>
__device__ __forceinline__ void elem_step(float qv, const uint8_t *row, uint32_t i, float scale, float &acc)
{
    if (ST == ANN_F16) {
        const float df = __fmaf_rn(-scale, __half2float(reinterpret_cast<const __half *>(row)[i]), qv);
        acc = __fmaf_rn(df, df, acc);
    } else {
        step(qv, stored_elem<ST>(row, i, scale), acc);
    }
}

// rn(y - x) and rn(acc + df * df) for two elements at once with the packed
// FP32 pipe: fma(x, -1, y) rounds y - x once, so both results equal the
// scalar __fsub_rn / __fmaf_rn of each component.
__device__ __forceinline__ void step2(float2 y, float2 x, float2 &acc)
{
    const float2 df = __ffma2_rn(x, make_float2(-1.0f, -1.0f), y);
    acc = __ffma2_rn(df, df, acc);
}

// Half of the squared L2 between a staged row and the query (both in
// shared memory). The distance keeps four partial sums, element i (in index
// order) fused into sum i mod 4, and is (s0 + s1) + (s2 + s3); half h of the
// lane pair of a row computes s_{2h} + s_{2h+1}, so one more add of the two
// halves gives the distance and each lane does half the elements. The two
// sums of a lane are one float2, updated with packed FP32 instructions. The
// loops unroll by two only: with 24 warps per SM spread over the whole
// iteration, the kernel is bound by instruction fetch, and the compiler's
// deeper unrolling cost 6% of throughput (measured on the 1M x 96 workload).
template <int ST>
__device__ __forceinline__ float row_dist_half(const uint8_t *row, const float *q, float scale, uint32_t d,
                                               uint32_t h)
{
    float2 s = make_float2(0.0f, 0.0f);  // s_{2h}, s_{2h+1}
    const float2 sc = make_float2(scale, scale), nsc = make_float2(-scale, -scale);
    uint32_t i = 0;
    if (ST == ANN_F32) {
#pragma unroll 2
        for (; i + 4 <= d; i += 4) {
            const float2 x = *reinterpret_cast<const float2 *>(row + (size_t)(i + 2 * h) * 4);
            const float2 y = *reinterpret_cast<const float2 *>(q + i + 2 * h);
            step2(y, x, s);
        }
    } else if (ST == ANN_F16) {
#pragma unroll 2
        for (; i + 8 <= d; i += 8) {
#pragma unroll
            for (uint32_t g = 0; g < 2; ++g) {
                const uint32_t e = i + 4 * g + 2 * h;
                const __half2 hv = *reinterpret_cast<const __half2 *>(row + (size_t)e * 2);
                const float2 y = *reinterpret_cast<const float2 *>(q + e);
                // y - s h in one rounding (s h is exact: s is a power of two)
                const float2 df = __ffma2_rn(nsc, __half22float2(hv), y);
                s = __ffma2_rn(df, df, s);
            }
        }
    } else {
#pragma unroll 2
        for (; i + 16 <= d; i += 16) {
            const uint4 raw = *reinterpret_cast<const uint4 *>(row + i);
            const uint32_t wds[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
            for (uint32_t g = 0; g < 4; ++g) {
                const __half2_raw pr =
                    __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)((wds[g] >> (16 * h)) & 0xffffu), __NV_E4M3);
                const float2 y = *reinterpret_cast<const float2 *>(q + i + 4 * g + 2 * h);
                step2(y, __fmul2_rn(sc, __half22float2(__half2(pr))), s);
            }
        }
    }
    // tail (d not a multiple of the vector width); i is a multiple of 4 here
    #pragma unroll 1
    for (; i < d; i += 4) {
        if (i + 2 * h < d) elem_step<ST>(q[i + 2 * h], row, i + 2 * h, scale, s.x);
        if (i + 2 * h + 1 < d) elem_step<ST>(q[i + 2 * h + 1], row, i + 2 * h + 1, scale, s.y);
    }
    return __fadd_rn(s.x, s.y);
}

// One of the four partial sums of the squared L2 between a staged row and
// the query: lane j of a row's four lanes runs sum j (elements i = j, j + 4,
// ... in index order, one fused multiply-add each), so the four lanes
// together do the work of one row with the same operations as the
// definition. Used for wide rows, where a round stages at most 8 rows.
template <int ST>
__device__ __forceinline__ float row_dist_quarter(const uint8_t *row, const float *q, float scale, uint32_t d,
                                                  uint32_t j)
{
    float s = 0.0f;
#pragma unroll 4
    for (uint32_t i = j; i < d; i += 4) elem_step<ST>(q[i], row, i, scale, s);
    return s;
}

template <int ST, bool PROF = false, int LPR = 2>
struct WarpSearch {
    const Args &a;
    uint8_t *base;
    uint32_t lane;
    uint32_t cnt = 0, phase = 0, hash_count = 0;
    bool failed = false;
    uint64_t qid = 0;
    ann_query_stats st;
    uint32_t *vt;        // this warp's visited table
    bool gbm = false;    // the visited set is the ghost bitmap (ghost stage, small ghost sets)
    // profile build: this warp slot's counters, the stage being timed and the
    // clock at the last phase boundary (lane 0)
    unsigned long long *pacc = nullptr;
    uint32_t pstage = 0;
    long long pt = 0;

    __device__ WarpSearch(const Args &args, uint8_t *b, uint32_t slot)
        : a(args), base(b), lane(threadIdx.x & 31), vt(args.vtab + ((size_t)slot << args.vstride_bits))
    {
        if (PROF) pacc = args.prof + (size_t)slot * (ANN_PROFILE_STAGES * ANN_PROFILE_PHASES);
    }

    // Profile build: charge the cycles since the last boundary to phase ph
    // of the current stage (a fire-and-forget add to this slot's counter).
    __device__ __forceinline__ void mark(uint32_t ph)
    {
        if (PROF && lane == 0) {
            const long long t = clock64();
            atomicAdd(pacc + pstage * ANN_PROFILE_PHASES + ph, (unsigned long long)(t - pt));
            pt = t;
        }
    }

    // shared-memory arrays of this warp
    __device__ __forceinline__ float *q() const { return reinterpret_cast<float *>(base + a.lay.q); }
    __device__ __forceinline__ float *bd() const { return reinterpret_cast<float *>(base + a.lay.bd); }
    __device__ __forceinline__ uint32_t *bi() const { return reinterpret_cast<uint32_t *>(base + a.lay.bi); }
    __device__ __forceinline__ uint8_t *bs() const { return base + a.lay.bs; }
    __device__ __forceinline__ float *cd() const { return reinterpret_cast<float *>(base + a.lay.cd); }
    __device__ __forceinline__ uint32_t *ci() const { return reinterpret_cast<uint32_t *>(base + a.lay.ci); }
    __device__ __forceinline__ uint32_t *cs() const { return reinterpret_cast<uint32_t *>(base + a.lay.cs); }
    __device__ __forceinline__ uint32_t *adj() const { return reinterpret_cast<uint32_t *>(base + a.lay.adj); }
    __device__ __forceinline__ uint32_t *dirs() const { return reinterpret_cast<uint32_t *>(base + a.lay.dir); }
    __device__ __forceinline__ uint8_t *prow() const { return base + a.lay.prow; }
    __device__ __forceinline__ uint32_t *par() const { return reinterpret_cast<uint32_t *>(base + a.lay.par); }
    __device__ __forceinline__ uint8_t *stage() const { return base + a.lay.stage; }
    __device__ __forceinline__ uint64_t *bar() const { return reinterpret_cast<uint64_t *>(base + a.lay.bar); }
    // two words beside the mbarrier (its 16-byte slot): the ghost judge
    __device__ __forceinline__ uint32_t *judge() const { return reinterpret_cast<uint32_t *>(base + a.lay.bar + 8); }

    // ---------------------------------------------------------- visited set
    __device__ __forceinline__ uint32_t *gbits() const { return reinterpret_cast<uint32_t *>(base + a.lay.dir); }
    __device__ __forceinline__ uint32_t hash_home(uint32_t v) const { return (v * 2654435761u) >> (32 - a.vbits); }

    // The rest of a test-and-insert of entry want (id + 1) whose first probe,
    // a CAS of slot s from empty, returned old: true if the id was new.
    __device__ bool hash_finish(uint32_t s, uint32_t want, uint32_t old)
    {
        const uint32_t mask = (1u << a.vbits) - 1;
        #pragma unroll 1
        for (uint32_t probe = 0; probe <= mask; ++probe) {
            if (old == 0) return true;        // claimed an empty slot
            if (old == want) return false;    // found it
            s = (s + 1) & mask;
            old = atomicCAS(vt + s, 0u, want);
        }
        return true;  // unreachable: the table is never more than half full
    }

    // Test-and-insert: true if v was not in the set (and is now).
    __device__ bool hash_insert(uint32_t v)
    {
        if (gbm) {
            const uint32_t bit = 1u << (v & 31);
            return (atomicOr(gbits() + (v >> 5), bit) & bit) == 0;
        }
        const uint32_t s = hash_home(v);
        return hash_finish(s, v + 1, atomicCAS(vt + s, 0u, v + 1));
    }

    // Start an empty set: zero the bitmap or the warp's table.
    __device__ void hash_clear()
    {
        if (gbm) {
            #pragma unroll 1
            for (uint32_t i = lane; i < a.gbm_words; i += 32) gbits()[i] = 0;
            __syncwarp();
            hash_count = 0;
            return;
        }
        const uint32_t H = 1u << a.vbits;
        uint4 *t4 = reinterpret_cast<uint4 *>(vt);
        #pragma unroll 1
        for (uint32_t i = lane; i < H / 4; i += 32) t4[i] = make_uint4(0, 0, 0, 0);
        __threadfence_block();
        __syncwarp();   // the lanes' zeroing precedes any lane's probes
        hash_count = 0;
    }

    // Forget everything but the queue (why this cannot change the result is
    // in the file comment).
    __device__ void hash_reset()
    {
        hash_clear();
        #pragma unroll 1
        for (uint32_t i = lane; i < cnt; i += 32) hash_insert(bi()[i]);
        __syncwarp();
        hash_count = cnt;
        st.hash_resets++;
    }

    __device__ __forceinline__ void hash_make_room(uint32_t incoming)
    {
        if (!gbm && hash_count + incoming > (1u << (a.vbits - 1))) hash_reset();
    }

    // ------------------------------------------------ bulk copies + waiting
    // Every lane waits; the outcome is made warp-uniform so the warp's later
    // collectives never see a partial warp.
    __device__ bool wait_copies()
    {
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar(), phase, a.err));
        phase ^= 1;
        if (!ok) {
            failed = true;
            mbar_wait_bounded(bar(), phase ^ 1, a.err);  // let copies in flight land
            __syncwarp();
        }
        return ok;
    }

    // ----------------------------------------------------- evaluate rows
    // Distances of rows ids[0, n) of `codes` into out[0, n), R (<= 32 / LPR)
    // rows of `stride` bytes per bulk-copy round; lanes LPR r .. LPR r + LPR
    // - 1 compute row r (a lane pair, or four lanes for wide rows).
    template <int RST>
    __device__ bool evaluate(const uint8_t *codes, const float *scales, uint32_t row_bytes, const uint32_t *ids,
                             uint32_t n, float *out, uint32_t R, uint32_t stride)
    {
        #pragma unroll 1
        for (uint32_t b0 = 0; b0 < n; b0 += R) {
            const uint32_t rows = min(R, n - b0);
            float scale = 1.0f;
            if (lane == 0) {
                fence_proxy_async();
                mbar_arrive_expect_tx(bar(), rows * row_bytes);
            }
            __syncwarp();
            if (lane < rows) {
                const uint32_t v = ids[b0 + lane];
                bulk_g2s(stage() + lane * stride, codes + (uint64_t)v * row_bytes, row_bytes, bar());
                if (RST != ANN_F32) scale = __ldg(scales + v);
            }
            if (!wait_copies()) return false;
            mark(PH_GATHER);
            const uint32_t r = lane / LPR;
            const float rs = __shfl_sync(0xffffffffu, scale, r);
            float part = 0.0f;
            if (LPR == 2) {
                if (r < rows) part = row_dist_half<RST>(stage() + r * stride, q(), rs, a.d, lane & 1);
            } else {
                // sum j of the row, then (s0 + s1) and (s2 + s3) on lane pairs
                if (r < rows) part = row_dist_quarter<RST>(stage() + r * stride, q(), rs, a.d, lane & 3);
                part = __fadd_rn(part, __shfl_xor_sync(0xffffffffu, part, 1));
            }
            const float other = __shfl_xor_sync(0xffffffffu, part, LPR / 2);
            if (r < rows && (lane & (LPR - 1)) == 0) out[b0 + r] = __fadd_rn(part, other);
            __syncwarp();
            mark(PH_DIST);
        }
        return true;
    }

    // --------------------------------------------------------------- merge
    // In-place merge of candidates [0, nc) into the queue, keeping the first
    // lcap entries by (dist, id). New entries are UNEXPANDED.
    __device__ void merge(uint32_t nc, uint32_t lcap)
    {
        float *qd = bd();
        uint32_t *qi = bi();
        uint8_t *qs = bs();
        float *kd = cd();
        uint32_t *kid = ci();
        uint32_t *ks = cs();
        // 1. drop candidates no better than the last entry of a full queue
        if (cnt == lcap && nc) {
            const float wd = qd[cnt - 1];
            const uint32_t wi = qi[cnt - 1];
            uint32_t kept = 0;
            #pragma unroll 1
            for (uint32_t b = 0; b < nc; b += 32) {
                const uint32_t c = b + lane;
                float dd = 0.0f;
                uint32_t id = 0;
                bool keep = false;
                if (c < nc) {
                    dd = kd[c];
                    id = kid[c];
                    keep = key_less(dd, id, wd, wi);
                }
                const uint32_t m = __ballot_sync(0xffffffffu, keep);
                __syncwarp();
                if (keep) {
                    const uint32_t at = kept + __popc(m & lanemask_lt());
                    kd[at] = dd;
                    kid[at] = id;
                }
                kept += __popc(m);
                __syncwarp();
            }
            nc = kept;
        }
        if (nc == 0) return;
        // 2. insertion point in the queue and rank among the candidates (the
        //    counting loop unrolls by two only, to keep the kernel's code
        //    small: it is bound by instruction fetch). lr[rank] = insertion
        //    point, in the staging area (free between gathers): candidate
        //    keys are distinct, so ranks are a permutation, and a larger key
        //    never has a smaller insertion point, so lr is non-decreasing.
        uint32_t *lr = reinterpret_cast<uint32_t *>(stage());
        uint32_t min_lb = 0xffffffffu;
        #pragma unroll 1
        for (uint32_t c = lane; c < nc; c += 32) {
            const float dd = kd[c];
            const uint32_t id = kid[c];
            uint32_t r = 0;
#pragma unroll 2
            for (uint32_t c2 = 0; c2 < nc; ++c2) r += key_less(kd[c2], kid[c2], dd, id);
            uint32_t lo = 0, hi = cnt;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (key_less(qd[mid], qi[mid], dd, id)) lo = mid + 1;
                else hi = mid;
            }
            ks[c] = lo | (r << 16);
            lr[r] = lo;
            min_lb = min(min_lb, lo);
        }
        for (int o = 16; o; o >>= 1) min_lb = min(min_lb, __shfl_xor_sync(0xffffffffu, min_lb, o));
        __syncwarp();
        // 3. shift queue entries [min_lb, cnt) by the number of candidates
        //    inserted before them (those whose insertion point is <= the
        //    entry's slot: a binary search of lr), last chunk first (in place)
        if (cnt > min_lb) {
            #pragma unroll 1
            for (int32_t top = (int32_t)cnt - 1; top >= (int32_t)min_lb; top -= 32) {
                const int32_t b = top - (int32_t)lane;
                float dd = 0.0f;
                uint32_t id = 0, s = 0, shift = 0;
                const bool mine = b >= (int32_t)min_lb;
                if (mine) {
                    dd = qd[b];
                    id = qi[b];
                    s = qs[b];
                    uint32_t hi = nc;
                    while (shift < hi) {
                        const uint32_t mid = (shift + hi) >> 1;
                        if (lr[mid] <= (uint32_t)b) shift = mid + 1;
                        else hi = mid;
                    }
                }
                __syncwarp();
                if (mine && (uint32_t)b + shift < lcap) {
                    qd[b + shift] = dd;
                    qi[b + shift] = id;
                    qs[b + shift] = (uint8_t)s;
                }
                __syncwarp();
            }
        }
        // 4. candidates into their slots
        #pragma unroll 1
        for (uint32_t c = lane; c < nc; c += 32) {
            const uint32_t pos = (ks[c] & 0xffffu) + (ks[c] >> 16);
            if (pos < lcap) {
                qd[pos] = kd[c];
                qi[pos] = kid[c];
                qs[pos] = kUnexpanded;
            }
        }
        cnt = min(lcap, cnt + nc);
        __syncwarp();
    }

    // Collect the kept neighbours of parent pi in slots lane + 32 (r0 + r),
    // r < NW (bit r0 + r of km), that are new to the visited set. The first
    // probes of a lane's NW slots are issued before any result is examined,
    // so their latencies overlap. Returns the warp's new candidate count.
    template <uint32_t NW>
    __device__ uint32_t collect_row_nw(const View &v, uint32_t pi, uint32_t km, uint32_t r0, uint32_t nc)
    {
        uint32_t nb[NW], hs[NW], cur[NW], old[NW];
        bool ok[NW];
#pragma unroll
        for (uint32_t r = 0; r < NW; ++r) {
            const uint32_t j = lane + 32 * (r0 + r);
            nb[r] = j < v.deg ? adj()[pi * v.deg_pad + j] : ANN_INVALID_ID;
            ok[r] = nb[r] != ANN_INVALID_ID && ((km >> (r0 + r)) & 1u);
        }
#pragma unroll
        for (uint32_t r = 0; r < NW; ++r) {
            if (ok[r]) {
                hs[r] = hash_home(nb[r]);
                cur[r] = nb[r] + 1;
                old[r] = atomicCAS(vt + hs[r], 0u, cur[r]);
            }
        }
#pragma unroll
        for (uint32_t r = 0; r < NW; ++r) {
            const bool isnew = ok[r] && hash_finish(hs[r], cur[r], old[r]);
            const uint32_t m = __ballot_sync(0xffffffffu, isnew);
            if (isnew) ci()[nc + __popc(m & lanemask_lt())] = nb[r];
            nc += __popc(m);
        }
        return nc;
    }

    __device__ uint32_t collect_row(const View &v, uint32_t pi, uint32_t km, uint32_t nc)
    {
        if (gbm) {
            #pragma unroll 1
            for (uint32_t r = 0; r * 32 < v.deg; ++r) {
                const uint32_t j = lane + 32 * r;
                const uint32_t nb = j < v.deg ? adj()[pi * v.deg_pad + j] : ANN_INVALID_ID;
                nc = collect(nb != ANN_INVALID_ID && ((km >> r) & 1u), nb, nc);
            }
            return nc;
        }
        if (v.deg <= 32) return collect_row_nw<1>(v, pi, km, 0, nc);
        #pragma unroll 1
        for (uint32_t r0 = 0; r0 * 32 < v.deg; r0 += 2) nc = collect_row_nw<2>(v, pi, km, r0, nc);
        return nc;
    }

    // Collect a lane's id into the candidate list if it is new to the
    // visited set; returns the warp's new count.
    __device__ __forceinline__ uint32_t collect(bool valid, uint32_t v, uint32_t nc)
    {
        const bool isnew = valid && hash_insert(v);
        const uint32_t m = __ballot_sync(0xffffffffu, isnew);
        if (isnew) ci()[nc + __popc(m & lanemask_lt())] = v;
        return nc + __popc(m);
    }

    // ------------------------------------------------------------- seeding
    // Seeds (Step 2): given nodes (ids, the learned entry's ghost nodes;
    // invalid or out-of-range ids skipped) or, with ids NULL, m random nodes
    // deduplicated without redraw: node j is splitmix64(key ^ (qid << 32) ^ j)
    // mod n, key = splitmix64(seed ^ tag). Seeds [j0, j0 + chunk) that are
    // new to the visited set become the candidates; returns their count.
    __device__ uint32_t collect_seeds(const View &v, const uint32_t *ids, uint64_t key, uint32_t j0, uint32_t chunk)
    {
        uint32_t nc = 0;
        #pragma unroll 1
        for (uint32_t b = 0; b < chunk; b += 32) {
            const uint32_t j = j0 + b + lane;
            uint32_t id = kEmpty;
            if (b + lane < chunk)
                id = ids ? __ldcg(ids + j) : (uint32_t)(splitmix64(key ^ (qid << 32) ^ (uint64_t)j) % v.n);
            nc = collect(id < v.n, id, nc);
        }
        return nc;
    }

    // ---------------------------------------------------------- iterations
    // Parents: the first `W` eligible queue entries in queue order.
    __device__ uint32_t select_parents(uint32_t W, bool cool)
    {
        uint32_t np = 0;
        const uint8_t *s8 = bs();
        #pragma unroll 1
        for (uint32_t b = 0; b < cnt && np < W; b += 32) {
            const uint32_t i = b + lane;
            bool e = false;
            if (i < cnt) {
                const uint32_t s = s8[i];
                e = s == kUnexpanded || (cool && s == kPartial);
            }
            uint32_t m = __ballot_sync(0xffffffffu, e);
            while (m && np < W) {
                const uint32_t bit = __ffs(m) - 1;
                m &= m - 1;
                if (lane == 0) par()[np] = b + bit;
                ++np;
            }
        }
        __syncwarp();
        return np;
    }

    __device__ bool any_partial()
    {
        bool p = false;
        #pragma unroll 1
        for (uint32_t i = lane; i < cnt; i += 32) p |= bs()[i] == kPartial;
        return __any_sync(0xffffffffu, p);
    }

    // DGS keep-mask of parent pi (bit r of the result: slot lane + 32 r is
    // kept). Score = matching sign bits; keep the top n_keep by (score desc,
    // slot asc): find the threshold score t by a radix select with ballots
    // (most significant bit first), keep scores above t and the first ties
    // at t. With min_match > 0, keep instead every neighbour scoring at
    // least min_match. NW = number of 32-slot words the degree spans (1, 2
    // or 4), so no ballot is spent on slots past the degree.
    template <uint32_t NW>
    __device__ uint32_t dgs_keep_nw(const View &v, uint32_t pi, uint32_t n_keep, uint32_t min_match, float ps)
    {
        const uint32_t w = a.w, deg = v.deg;
        const uint8_t *pr = prow() + pi * a.prow_bytes;
        // mismatching sign bits per slot, 4 words of the query's sign bits
        // relative to the parent ([q > x_parent], one ballot per 32
        // dimensions) at a time. Words past w have no dimension (their bits
        // are 0) and count nothing; the loads stay in the row (clamped), so
        // a chunk has no branch and its loads issue together.
        int diff[NW];
        bool live[NW];
        const uint32_t *db[NW];
#pragma unroll
        for (uint32_t r = 0; r < NW; ++r) {
            const uint32_t j = min(lane + 32 * r, deg - 1);
            live[r] = lane + 32 * r < deg && adj()[pi * v.deg_pad + j] != ANN_INVALID_ID;
            db[r] = dirs() + (pi * v.deg_pad + j) * w;
            diff[r] = 0;
        }
        for (uint32_t t0 = 0; t0 < w; t0 += 4) {
            uint32_t qw[4];
#pragma unroll
            for (uint32_t x = 0; x < 4; ++x) {
                const uint32_t i = 32 * (t0 + x) + lane;
                const uint32_t ic = min(i, a.d - 1);
                qw[x] = __ballot_sync(0xffffffffu, i < a.d && q()[ic] > stored_elem<ST>(pr, ic, ps));
            }
#pragma unroll
            for (uint32_t r = 0; r < NW; ++r)
#pragma unroll
                for (uint32_t x = 0; x < 4; ++x) {
                    const uint32_t dw = db[r][min(t0 + x, w - 1)];
                    diff[r] += t0 + x < w ? __popc(qw[x] ^ dw) : 0;
                }
        }
        // u = score + 2: 0 past the degree (never kept), 1 for an empty
        // slot, 2 + matching bits for a neighbour
        uint32_t u[NW];
#pragma unroll
        for (uint32_t r = 0; r < NW; ++r) {
            const uint32_t j = lane + 32 * r;
            u[r] = j >= deg ? 0u : (live[r] ? a.d + 2 - (uint32_t)diff[r] : 1u);
        }
        if (min_match > 0) {
            uint32_t keep = 0;
#pragma unroll
            for (uint32_t r = 0; r < NW; ++r)
                if (u[r] >= min_match + 2) keep |= 1u << r;
            return keep;
        }
        // radix select of the n_keep-th largest u: t collects its bits from
        // the top; `need` counts how many of the values equal to t's bits so
        // far are still to be kept. At the end every u > t is kept and
        // `need` of the ties at t.
        uint32_t t = 0, need = n_keep;
        for (int bit = 31 - __clz(a.d + 2); bit >= 0; --bit) {
            const uint32_t hi = (t >> bit) | 1u;
            uint32_t c = 0;
#pragma unroll
            for (uint32_t r = 0; r < NW; ++r) c += __popc(__ballot_sync(0xffffffffu, (u[r] >> bit) == hi));
            if (c >= need) t |= 1u << bit;
            else need -= c;
        }
        uint32_t keep = 0, ties_before = 0;
#pragma unroll
        for (uint32_t r = 0; r < NW; ++r) {
            const uint32_t tm = __ballot_sync(0xffffffffu, u[r] == t);
            const bool tie_kept = u[r] == t && ties_before + __popc(tm & lanemask_lt()) < need;
            if (u[r] > t || tie_kept) keep |= 1u << r;
            ties_before += __popc(tm);
        }
        return keep;
    }

    __device__ uint32_t dgs_keep(const View &v, uint32_t pi, uint32_t n_keep, uint32_t min_match, float ps)
    {
        if (v.deg <= 32) return dgs_keep_nw<1>(v, pi, n_keep, min_match, ps);
        if (v.deg <= 64) return dgs_keep_nw<2>(v, pi, n_keep, min_match, ps);
        return dgs_keep_nw<kMaxDegWords>(v, pi, n_keep, min_match, ps);
    }

    // Step 2 (m seeds, in chunks of the candidate capacity), then Steps 3-4
    // repeated with DGS and its cool-down (Section 3.3.2). Seed chunks and
    // parent expansions share one loop body, so the distance and merge code
    // exists once in the kernel (the kernel is bound by instruction fetch).
    template <int RST>
    // The judge of a ghost stage from given seeds (run() sets it in judge(),
    // else zero): at iteration T, a queue holding no node nearer than
    // judge()[0] (FP32 bits) goes on to judge()[1] iterations in all. Kept in
    // shared memory so the loop carries no extra registers.
    __device__ bool iterate(const View &v, const uint32_t *seed_ids, uint32_t m, uint64_t seed_key, uint32_t lcap,
                            uint32_t W, uint32_t T, uint32_t n_keep, uint32_t min_match, uint32_t it_cool,
                            uint32_t reexpand,
                            uint32_t &c_iters, uint32_t &c_parents, uint32_t &c_dgs, uint32_t &c_rows)
    {
        const uint32_t deg = v.deg;
        const bool dgs_on = v.dir != nullptr && (min_match > 0 || n_keep < deg);
        const uint32_t w = a.w;
        bool cool = false;
        uint32_t j0 = 0, it = 0;
        for (;;) {
            uint32_t nc = 0;
            if (j0 < m) {
                const uint32_t chunk = min(a.cap_cand, m - j0);
                hash_make_room(chunk);
                nc = collect_seeds(v, seed_ids, seed_key, j0, chunk);
                j0 += chunk;
                mark(PH_VISIT);
            } else {
                if (it == T) {
                    const uint32_t t_ext = judge()[1];
                    if (t_ext <= T || cnt == 0 || !(bd()[0] > __uint_as_float(judge()[0]))) break;
                    T = t_ext;   // judged too far: the rest of the ghost iterations
                }
                if (dgs_on && it >= it_cool) cool = true;
                uint32_t np = select_parents(W, cool);
                if (np == 0 && dgs_on && reexpand && !cool && any_partial()) {
                    cool = true;
                    np = select_parents(W, cool);
                }
                if (np == 0) break;
                ++it;
                ++c_iters;
                const bool dgs_now = dgs_on && !cool;
                // mark the parents; fetch adjacency (and, under DGS, direction
                // and vector) rows in one bulk-copy round
                const uint32_t adj_bytes = v.deg_pad * 4;
                const uint32_t dir_bytes = v.deg_pad * w * 4;
                uint32_t pid = 0;
                if (lane < np) {
                    const uint32_t b = par()[lane];
                    pid = bi()[b];
                    bs()[b] = (dgs_now && reexpand) ? kPartial : kExpanded;
                }
                if (lane == 0) {
                    fence_proxy_async();
                    mbar_arrive_expect_tx(bar(), np * (adj_bytes + (dgs_now ? dir_bytes + v.row_bytes : 0)));
                }
                __syncwarp();
                if (lane < np) {
                    bulk_g2s(adj() + lane * v.deg_pad, v.graph + (uint64_t)pid * v.deg_pad, adj_bytes, bar());
                    if (dgs_now) {
                        bulk_g2s(dirs() + lane * v.deg_pad * w, v.dir + (uint64_t)pid * v.deg_pad * w, dir_bytes,
                                 bar());
                        bulk_g2s(prow() + lane * a.prow_bytes, v.codes + (uint64_t)pid * v.row_bytes, v.row_bytes,
                                 bar());
                        // the parent's scale replaces its queue slot in
                        // par() (read by DGS after the wait)
                        if (RST != ANN_F32) par()[lane] = __float_as_uint(__ldg(v.scales + pid));
                    }
                }
                if (!wait_copies()) return false;
                mark(PH_SELECT);
                c_parents += np;
                if (dgs_now) c_dgs += np;
                hash_make_room(np * deg);
                for (uint32_t pi = 0; pi < np; ++pi) {
                    uint32_t km = 0xffffffffu;
                    if (dgs_now) {
                        km = dgs_keep(v, pi, n_keep, min_match,
                                      RST != ANN_F32 ? __uint_as_float(par()[pi]) : 1.0f);
                        mark(PH_DGS);
                    }
                    nc = collect_row(v, pi, km, nc);
                    mark(PH_VISIT);
                }
            }
            __syncwarp();
            hash_count += nc;
            if (!evaluate<RST>(v.codes, v.scales, v.row_bytes, ci(), nc, cd(), a.stage_rows, a.stage_stride))
                return false;
            c_rows += nc;
            merge(nc, lcap);
            mark(PH_MERGE);
        }
        return true;
    }

    // ------------------------------------------------------------- a query
    // One query: qg its vector, given its ghost seeds (or NULL), oid/odist
    // its k outputs, stats_out its counters (or NULL); qidx indexes the RNG
    // stream (qid = qp.qid_base + qidx).
    __device__ void run(const QParams &qp, uint64_t qidx, const float *qg, const uint32_t *given_row, uint32_t *oid,
                        float *odist, ann_query_stats *stats_out)
    {
        qid = qp.qid_base + qidx;
        st = ann_query_stats{};
        cnt = 0;
        if (PROF) {
            pt = clock64();
            pstage = ghost_entry(qp.entry) ? PS_GHOST : PS_BASE;
        }
        const uint32_t dpad = (a.d + 31) & ~31u;
        // read through L2 only: a serving ring rewrites query slots between
        // uses, and L1 is not kept coherent with those copies
        #pragma unroll 1
        for (uint32_t i = lane; i < dpad; i += 32) q()[i] = i < a.d ? __ldcg(qg + i) : 0.0f;
        __syncwarp();
        const bool ghost = ghost_entry(qp.entry);
        gbm = ghost && a.gbm_words > 0;
        hash_clear();
        const uint32_t *given = nullptr;
        if (given_entry(qp.entry) && given_row && given_row[0] != ANN_INVALID_ID)
            given = given_row;   // else: fall back to random (ghost) seeds
        // stage 0: the ghost stage (Section 3.2.2) on the ghost graph; stage
        // 1: the search on the base graph. One loop body serves both.
        bool ok = true;
        for (uint32_t stage = ghost ? 0u : 1u; stage < 2 && ok; ++stage) {
            const View v = stage ? a.base : a.ghost;
            const uint32_t lcap = stage ? qp.L : qp.Lg;
            uint32_t rows = 0, iters = 0, parents = 0, dgs_parents = 0;
            if (PROF && stage == 1 && ghost) {
                mark(PH_OTHER);   // the rest of the ghost stage
                pstage = PS_BASE;
            }
            if (stage == 1 && ghost) {
                // transition: the top g ghost results become the base queue;
                // ghost ids are ascending, so the (dist, id) order carries over
                const uint32_t g = min(min(qp.g, cnt), qp.L);
                #pragma unroll 1
                for (uint32_t i = lane; i < g; i += 32) {
                    bi()[i] = __ldg(a.ghost_ids + bi()[i]);
                    bs()[i] = kUnexpanded;
                }
                __syncwarp();
                cnt = g;
                gbm = false;   // the base stage's visited set is the global table
                hash_clear();
                #pragma unroll 1
                for (uint32_t i = lane; i < cnt; i += 32) hash_insert(bi()[i]);
                __syncwarp();
                hash_count = cnt;
                mark(PH_VISIT);
            }
            const bool seeded = !(stage == 1 && ghost);
            // a ghost stage from given seeds may be judged: one whose best
            // node is farther than the judge distance after Tg_given
            // iterations goes on to Tg (the ghost stage has no DGS, so its
            // cool-down start carries that total)
            const bool judged = stage == 0 && given && qp.judge > 0.0f && qp.Tg > qp.Tg_given;
            if (lane == 0) {
                judge()[0] = judged ? __float_as_uint(qp.judge) : 0u;
                judge()[1] = judged ? qp.Tg : 0u;
            }
            __syncwarp();
            ok = iterate<ST>(v, given, seeded ? (given ? qp.n_given : (stage ? qp.m : v.deg)) : 0,
                             splitmix64(qp.seed ^ (stage ? 0 : kGhostTag)), lcap, stage ? qp.W : qp.Wg,
                             stage ? qp.T : (given ? qp.Tg_given : qp.Tg), stage ? qp.n_keep : v.deg,
                             stage ? qp.min_match : 0,
                             stage ? qp.it_cool : 0, stage ? qp.reexpand : 0, iters, parents, dgs_parents, rows);
            // given seeds start the first stage only: the ghost stage (learned
            // entry) or, without one, the base stage (an extended path's start)
            given = nullptr;
            if (stage) {
                st.iters = iters;
                st.parents = parents;
                st.dgs_parents = dgs_parents;
                st.vec_rows = rows;
            } else {
                st.ghost_iters = iters;
                st.ghost_parents = parents;
                st.ghost_vec_rows = rows;
            }
        }
        if (PROF) {
            mark(PH_OTHER);
            pstage = PS_FINISH;
        }
        if (ok && qp.rerank) {
            // FP32 distances of the whole queue on the originals, then the top k
            // (a launch planned without rerank has no rerank rounds: such a
            // query fails instead of looping)
            ok = a.rr_rows > 0 && evaluate<ANN_F32>(a.x32, nullptr, a.row32_bytes, bi(), cnt, bd(), a.rr_rows,
                                                    a.rr_stride);
            st.rerank_rows += cnt;
            if (ok) {
                #pragma unroll 1
                for (uint32_t e = lane; e < cnt; e += 32) {
                    const float kd = bd()[e];
                    const uint32_t kid = bi()[e];
                    uint32_t r = 0;
                    #pragma unroll 1
                    for (uint32_t e2 = 0; e2 < cnt; ++e2) r += key_less(bd()[e2], bi()[e2], kd, kid);
                    if (r < qp.k) {
                        oid[r] = kid;
                        odist[r] = kd;
                    }
                }
                #pragma unroll 1
                for (uint32_t j = cnt + lane; j < qp.k; j += 32) {
                    oid[j] = ANN_INVALID_ID;
                    odist[j] = INFINITY;
                }
            }
        } else if (ok) {
            #pragma unroll 1
            for (uint32_t j = lane; j < qp.k; j += 32) {
                oid[j] = j < cnt ? bi()[j] : ANN_INVALID_ID;
                odist[j] = j < cnt ? bd()[j] : INFINITY;
            }
        }
        if (!ok) {
            #pragma unroll 1
            for (uint32_t j = lane; j < qp.k; j += 32) {
                oid[j] = ANN_INVALID_ID;
                odist[j] = INFINITY;
            }
            st.status = 1;
        }
        if (stats_out && lane == 0) *stats_out = st;
        __syncwarp();
        mark(PH_OTHER);
    }
};

template <int ST, bool PROF = false, int LPR = 2>
__global__ void __launch_bounds__(128, kSearchBlocksPerSm) search_kernel(const Args a)
{
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSearch<ST, PROF, LPR> ws(a, smem + (size_t)warp * a.lay.total, a.slot_base + blockIdx.x * (blockDim.x >> 5) + warp);
    if (lane == 0) mbar_init(ws.bar(), 1);
    fence_mbar_init();
    __syncwarp();
    while (true) {
        uint32_t qi = 0;
        if (lane == 0) qi = atomicAdd(a.counter, 1u);
        qi = __shfl_sync(0xffffffffu, qi, 0);
        if (qi >= a.nq) break;
        const QParams &qp = a.qp;
        ws.run(qp, qi, a.queries + (uint64_t)qi * a.d,
               (given_entry(qp.entry) && a.given) ? a.given + (uint64_t)qi * qp.n_given : nullptr,
               a.out_ids + (uint64_t)qi * qp.k, a.out_dists + (uint64_t)qi * qp.k, a.stats ? a.stats + qi : nullptr);
        if (ws.failed) break;
    }
}

// Continuous batching: warps of every running serve kernel pop queries, in
// arrival order, from one device ring that the host appends to while they
// run (head/tail are monotonic query counters; slot = counter mod capacity).
// A warp serves at most `per_warp` queries and then leaves, so a launch's
// capacity is blocks x warps x per_warp and SMs free up for other kernels.
// The request's parameters are copied into the warp's shared memory; the
// warp that finishes a request's last query raises its completion flag in
// host-mapped memory after a system-scope fence.
template <int ST, int LPR = 2>
__global__ void __launch_bounds__(128, kSearchBlocksPerSm) serve_kernel(const Args a, const ServeRing r)
{
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *base = smem + (size_t)warp * a.lay.total;
    WarpSearch<ST, false, LPR> ws(a, base, a.slot_base + blockIdx.x * (blockDim.x >> 5) + warp);
    QParams *qp = reinterpret_cast<QParams *>(base + a.lay.qp);
    if (lane == 0) mbar_init(ws.bar(), 1);
    fence_mbar_init();
    __syncwarp();
    for (uint32_t served = 0; served < r.per_warp; ++served) {
        unsigned long long h = 0;
        uint32_t got = 0;
        if (lane == 0) {
            for (uint32_t attempt = 0; attempt < (1u << 20); ++attempt) {  // lock-free: a failed CAS means another warp won
                h = *reinterpret_cast<volatile unsigned long long *>(r.head);
                const unsigned long long t = *reinterpret_cast<volatile const unsigned long long *>(r.tail);
                if (h >= t) break;
                if (atomicCAS(r.head, h, h + 1) == h) { got = 1; break; }
            }
        }
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) break;
        h = __shfl_sync(0xffffffffu, h, 0);
        const uint32_t slot = (uint32_t)(h % r.cap);
        ServeReq *rq = r.reqs + __ldcg(r.slot_req + slot);
        if (lane < sizeof(QParams) / 4)
            reinterpret_cast<uint32_t *>(qp)[lane] = reinterpret_cast<const volatile uint32_t *>(&rq->qp)[lane];
        __syncwarp();
        const uint32_t j = (slot + r.cap - *reinterpret_cast<volatile uint32_t *>(&rq->slot0)) % r.cap;
        const uint32_t *seeds = (qp->entry == ANN_ENTRY_GIVEN_GHOST && r.seeds) ? r.seeds + (size_t)slot * r.P : nullptr;
        ws.run(*qp, j, r.queries + (size_t)slot * a.d, seeds, r.ids + (size_t)slot * r.kmax,
               r.dists + (size_t)slot * r.kmax, nullptr);
        if (ws.failed) break;
        __threadfence();
        __syncwarp();
        if (lane == 0) {
            const uint32_t done = atomicAdd(&rq->done, 1u) + 1;
            if (done == *reinterpret_cast<volatile uint32_t *>(&rq->nq)) {
                __threadfence_system();
                r.flags[rq->flag] = 1u;
            }
        }
        __syncwarp();
    }
}

uint32_t align16(uint32_t x) { return (x + 15) & ~15u; }

Layout make_layout(uint32_t d, uint32_t w, uint32_t cap_buf, uint32_t cap_cand, uint32_t W, uint32_t W_max,
                   uint32_t adj_words, uint32_t dir_words, uint32_t prow_bytes, uint32_t stage_rows,
                   uint32_t stage_stride, uint32_t rr_stride, uint32_t gbm_words, bool serve)
{
    Layout L{};
    uint32_t o = 0;
    auto take = [&](uint32_t bytes) {
        const uint32_t at = o;
        o = align16(o + bytes);
        return at;
    };
    L.q = take(((d + 31) & ~31u) * 4);
    L.bd = take(cap_buf * 4);
    L.bi = take(cap_buf * 4);
    L.bs = take(cap_buf);
    L.cd = take(std::max(cap_cand, cap_buf) * 4);
    L.ci = take(cap_cand * 4);
    L.cs = take(cap_cand * 4);
    L.adj = take(adj_words * 4);
    // the base stage's direction and parent rows share their space with the
    // ghost stage's visited bitmap (the two stages never overlap)
    const uint32_t dir_part = align16(dir_words * 4) + align16(dir_words ? W * prow_bytes : 0);
    L.dir = take(std::max(dir_part, gbm_words * 4));
    L.prow = L.dir + align16(dir_words * 4);
    L.par = take(W_max * 4);   // parents of an iteration of either stage
    // the staged rows (at least one of the rerank's FP32 rows); the merge
    // keeps its candidates' insertion points here
    L.stage = take(std::max(std::max(stage_rows * stage_stride, rr_stride), cap_cand * 4));
    L.bar = take(16);
    L.qp = take(serve ? 96 : 0);
    L.total = align16(o);
    return L;
}

template <int ST, bool PROF, int LPR>
cudaError_t launch_lpr(const Args &a, int warps, int blocks, size_t smem, cudaStream_t st)
{
    cudaError_t e =
        cudaFuncSetAttribute(search_kernel<ST, PROF, LPR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    search_kernel<ST, PROF, LPR><<<blocks, warps * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int ST, bool PROF = false>
cudaError_t launch(const Args &a, int warps, int blocks, size_t smem, cudaStream_t st)
{
    return a.lpr == 4 ? launch_lpr<ST, PROF, 4>(a, warps, blocks, smem, st)
                      : launch_lpr<ST, PROF, 2>(a, warps, blocks, smem, st);
}

template <int ST, int LPR>
int blocks_per_sm_lpr(int warps, size_t smem)
{
    int nb = 0;
    cudaFuncSetAttribute(search_kernel<ST, false, LPR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, search_kernel<ST, false, LPR>, warps * 32, smem);
    return nb;
}

template <int ST>
int blocks_per_sm(int warps, size_t smem, uint32_t lpr)
{
    return lpr == 4 ? blocks_per_sm_lpr<ST, 4>(warps, smem) : blocks_per_sm_lpr<ST, 2>(warps, smem);
}

int env_int(const char *name, int dflt)
{
    const char *s = getenv(name);
    return s ? atoi(s) : dflt;
}

}  // namespace

namespace ann {

ann_status derive_qparams(const ann_index *ix, const ann_search_params *p, uint32_t n_given, QParams *out)
{
    if (!ix || !p) { set_error("ann_search: NULL index or params"); return ANN_EINVAL; }
    const uint32_t L = p->itopk, W = p->search_width, deg = ix->degree;
    if (p->k == 0 || p->k > L || L == 0 || L > ANN_MAX_ITOPK || W == 0 || W > ANN_MAX_WIDTH) {
        set_error("ann_search: need 1 <= k <= itopk <= %u and 1 <= search_width <= %u", ANN_MAX_ITOPK,
                  ANN_MAX_WIDTH);
        return ANN_EINVAL;
    }
    if (!(p->dgs_discard >= 0.0f && p->dgs_discard < 1.0f) || !(p->dgs_cooldown >= 0.0f && p->dgs_cooldown <= 1.0f)) {
        set_error("ann_search: dgs_discard must be in [0,1) and dgs_cooldown in [0,1]");
        return ANN_EINVAL;
    }
    if (!(p->dgs_min_match >= 0.0f && p->dgs_min_match <= 1.0f) ||
        (p->dgs_min_match > 0.0f && p->dgs_discard > 0.0f)) {
        set_error("ann_search: dgs_min_match must be in [0,1], and not set together with dgs_discard");
        return ANN_EINVAL;
    }
    if ((p->dgs_discard > 0.0f || p->dgs_min_match > 0.0f) && !ix->dir) {
        set_error("ann_search: DGS needs an index built with the direction table");
        return ANN_EINVAL;
    }
    if (p->entry > ANN_ENTRY_GIVEN_BASE || (ghost_entry(p->entry) && ix->n_ghost == 0)) {
        set_error("ann_search: entry %u is unknown or needs a ghost set", p->entry);
        return ANN_EINVAL;
    }
    if (given_entry(p->entry) && n_given == 0) {
        set_error("ann_search: given seeds missing");
        return ANN_EINVAL;
    }
    if (p->rerank && !ix->x32) {
        set_error("ann_search: rerank needs the FP32 originals (keep_fp32)");
        return ANN_EINVAL;
    }
    const uint32_t Lg = p->ghost_itopk ? p->ghost_itopk : std::min(L, 64u);
    if (Lg > ANN_MAX_ITOPK) {
        set_error("ann_search: ghost_itopk > %u", ANN_MAX_ITOPK);
        return ANN_EINVAL;
    }
    if (!(p->ghost_judge >= 0.0f && p->ghost_judge <= 3.402823466e38f)) {
        set_error("ann_search: ghost_judge must be finite and >= 0");
        return ANN_EINVAL;
    }
    const uint32_t Wg = p->ghost_search_width ? p->ghost_search_width : 1;
    if (Wg > ANN_MAX_WIDTH) {
        set_error("ann_search: ghost_search_width must be <= %u", ANN_MAX_WIDTH);
        return ANN_EINVAL;
    }
    QParams q{};
    q.n_given = n_given;
    q.k = p->k;
    q.L = L;
    q.W = W;
    q.T = p->max_iters;
    q.m = p->num_seeds ? p->num_seeds : W * deg;
    // Section 3.3.2 readings: keep n = deg - round(rho * deg) (at least 1);
    // the cool-down is the last round(c * T) iterations (half-up, in double).
    uint32_t n_keep = deg;
    if (p->dgs_discard > 0.0f) {
        const int64_t drop = (int64_t)std::floor((double)p->dgs_discard * deg + 0.5);
        n_keep = (uint32_t)std::max<int64_t>(1, std::min<int64_t>(deg, (int64_t)deg - drop));
    }
    q.n_keep = n_keep;
    // the similarity threshold: ceil(f * d) agreeing dimensions, in double
    q.min_match = p->dgs_min_match > 0.0f ? (uint32_t)std::ceil((double)p->dgs_min_match * ix->dim) : 0;
    const int64_t n_cool = (int64_t)std::floor((double)p->dgs_cooldown * p->max_iters + 0.5);
    q.it_cool = (uint32_t)std::max<int64_t>(0, (int64_t)p->max_iters - n_cool);
    q.reexpand = p->dgs_reexpand ? 1 : 0;
    q.entry = p->entry;
    q.Lg = Lg;
    q.Tg = p->ghost_max_iters;
    q.Tg_given = p->ghost_max_iters_given;
    q.Wg = Wg;
    q.g = p->ghost_seeds_out ? p->ghost_seeds_out : Lg;
    q.judge = p->ghost_judge;
    q.rerank = p->rerank ? 1 : 0;
    q.seed = p->seed;
    q.qid_base = p->qid_base;
    *out = q;
    return ANN_OK;
}

namespace planning {

// Kernel arguments and launch shape for parameters q (the largest a launch
// must serve): shared-memory layout per warp, warps per block, blocks per SM.
ann_status plan_args(ann_index *ix, const QParams &q, Args &a, int &warps, size_t &smem, int &nb, bool serve)
{
    const uint32_t deg = ix->degree;
    a.base = View{(const uint8_t *)ix->codes, ix->scales, ix->row_bytes, ix->graph, deg, ix->deg_pad,
                  ix->dir, (uint32_t)ix->n};
    a.ghost = View{(const uint8_t *)ix->ghost_codes, ix->ghost_scales, ix->row_bytes, ix->ghost_graph,
                   ix->ghost_degree, ix->gdeg_pad, nullptr, ix->n_ghost};
    a.ghost_ids = ix->ghost_ids;
    a.x32 = (const uint8_t *)ix->x32;
    a.row32_bytes = ix->storage == ANN_F32 ? ix->row_bytes : ix->row32_bytes;
    a.d = ix->dim;
    a.w = ix->words;
    a.qp = q;
    const uint32_t cap_buf = std::max(q.L, ghost_entry(q.entry) ? q.Lg : 1u);
    uint32_t cap_cand = std::max(q.W * deg, 32u);
    if (ghost_entry(q.entry)) cap_cand = std::max(cap_cand, q.Wg * ix->ghost_degree);
    cap_cand = round_up(cap_cand, 32);
    a.cap_cand = cap_cand;
    const uint32_t adj_words = std::max(q.W * ix->deg_pad, q.Wg * ix->gdeg_pad);
    const bool dgs = q.n_keep < deg || q.min_match > 0;
    const uint32_t dir_words = dgs ? q.W * ix->deg_pad * ix->words : 0;
    a.prow_bytes = ix->row_bytes;
    // the search stages stored rows; the rerank stages FP32 rows in the same
    // area, fewer per round (it reads itopk rows per query, the search
    // thousands), so the area is sized by the stored rows
    const uint32_t stage_bytes = std::max(ix->row_bytes, q.rerank ? a.row32_bytes : 0u);
    a.stage_stride = smem_row_stride(ix->row_bytes);
    a.rr_stride = q.rerank ? smem_row_stride(a.row32_bytes) : 0u;
    // rows of more than 1 KB (wide FP32 vectors, 512 and up to ANN_MAX_DIM
    // dimensions) are computed by four lanes each, at most 8 per round;
    // narrower ones by lane pairs, 16 per round
    a.lpr = stage_bytes > 1024 ? 4 : 2;
    // visited tables: the queue plus one iteration's candidates must fit in
    // half a table (the reset threshold)
    if (cap_buf + cap_cand > (1u << (kVisitedBits - 1))) {
        set_error("ann_search: queue (%u) + candidates (%u) exceed the visited table", cap_buf, cap_cand);
        return ANN_EINVAL;
    }
    a.vtab = ix->visited.tab;
    a.vstride_bits = ix->visited.bits;
    a.vbits = ix->visited.bits;   // 4,096 entries: measured faster than 2,048 or 1,024 (L2-resident either way)
    a.slot_base = 0;
    a.gbm_words = (ghost_entry(q.entry) && ix->n_ghost <= kGhostBitmapMax) ? (ix->n_ghost + 31) / 32 : 0;
    // Shape for `rows` staged rows per gather round: the per-warp layout,
    // warps per block (wide rows: fewer staged rows before fewer warps) and
    // resident blocks per SM. False if no shape fits.
    struct Shape {
        Layout lay;
        uint32_t rows;
        int warps, nb;
        size_t smem;
    };
    auto fit = [&](uint32_t rows, Shape &sh) -> bool {
        sh.rows = rows;
        sh.warps = 4;
        for (;;) {
            sh.lay = make_layout(ix->dim, ix->words, cap_buf, cap_cand, q.W,
                                 std::max(q.W, ghost_entry(q.entry) ? q.Wg : 1u), adj_words, dir_words,
                                 a.prow_bytes, sh.rows, a.stage_stride, a.rr_stride, a.gbm_words, serve);
            if ((size_t)sh.lay.total * sh.warps <= ix->smem_optin) break;
            if (sh.rows > 4) { sh.rows /= 2; continue; }
            if (sh.warps > 1) { sh.warps /= 2; continue; }
            set_error("ann_search: per-query state (%u bytes) exceeds shared memory", sh.lay.total);
            return false;
        }
        sh.smem = (size_t)sh.lay.total * sh.warps;
        switch (ix->storage) {
        case ANN_F32: sh.nb = blocks_per_sm<ANN_F32>(sh.warps, sh.smem, a.lpr); break;
        case ANN_F16: sh.nb = blocks_per_sm<ANN_F16>(sh.warps, sh.smem, a.lpr); break;
        default: sh.nb = blocks_per_sm<ANN_E4M3>(sh.warps, sh.smem, a.lpr); break;
        }
        if (sh.nb <= 0) {
            set_error("ann_search: kernel does not fit on an SM (%zu bytes shared)", sh.smem);
            return false;
        }
        return true;
    };
    // The staged rows take most of a warp's shared memory. With the full
    // round (16 rows, 8 wide ones) shared memory can hold fewer warps than
    // the registers allow (large queues, 1 KB rows); half a round then
    // doubles the gather rounds but admits more resident warps, and the
    // latency those warps hide is worth more (measured: +19% to +43% where
    // the warps per SM rose, -18% where they did not). So half a round is
    // taken only when it admits more warps per SM. ANN_STAGE_ROWS fixes the
    // count instead (experiments).
    const int env_rows = env_int("ANN_STAGE_ROWS", 0);
    const uint32_t full = 32 / a.lpr;
    Shape best;
    if (!fit(env_rows > 0 ? (uint32_t)std::min<int>((int)full, env_rows) : full, best)) return ANN_EINVAL;
    if (env_rows <= 0 && best.rows == full) {
        Shape half;
        if (fit(full / 2, half) && half.nb * half.warps > best.nb * best.warps) best = half;
    }
    a.stage_rows = best.rows;
    a.rr_rows = a.rr_stride ? std::min(full, std::max(1u, best.rows * a.stage_stride / a.rr_stride)) : 0u;
    a.lay = best.lay;
    warps = best.warps;
    smem = best.smem;
    nb = best.nb;
    return ANN_OK;
}

struct ServePlanImpl {
    Args a;
    int warps, nb, num_sms, storage;
    size_t smem;
    ann_visited_pool visited;     // the plan's own tables: n_streams launches at once
    uint32_t slots_per_launch;
};

template <int ST, int LPR>
cudaError_t launch_serve_lpr(const ServePlanImpl &pl, const ServeRing &r, int blocks, cudaStream_t st)
{
    cudaError_t e =
        cudaFuncSetAttribute(serve_kernel<ST, LPR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
    if (e != cudaSuccess) return e;
    serve_kernel<ST, LPR><<<blocks, pl.warps * 32, pl.smem, st>>>(pl.a, r);
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_serve(const ServePlanImpl &pl, const ServeRing &r, int blocks, cudaStream_t st)
{
    return pl.a.lpr == 4 ? launch_serve_lpr<ST, 4>(pl, r, blocks, st) : launch_serve_lpr<ST, 2>(pl, r, blocks, st);
}

}  // namespace planning

using namespace planning;

ann_status search_launch_ex(ann_index *ix, const float *queries, uint32_t nq, const ann_search_params *p,
                            const uint32_t *given, uint32_t n_given, uint32_t *ids, float *dists,
                            ann_query_stats *stats, cudaStream_t stream, uint32_t *counter, int *err,
                            unsigned long long *prof)
{
    QParams q;
    ann_status s = derive_qparams(ix, p, given ? n_given : 0, &q);
    if (s != ANN_OK) return s;
    if (nq && (!queries || !ids || !dists)) {
        set_error("ann_search: NULL queries or outputs");
        return ANN_EINVAL;
    }
    if (nq == 0) return ANN_OK;
    Args a{};
    int warps = 0, nb = 0;
    size_t smem = 0;
    s = plan_args(ix, q, a, warps, smem, nb, false);
    if (s != ANN_OK) return s;
    a.queries = queries;
    a.nq = nq;
    a.given = given;
    a.out_ids = ids;
    a.out_dists = dists;
    a.stats = stats;
    a.counter = counter;
    a.err = err;
    a.prof = prof;
    const uint64_t want = ((uint64_t)nq + warps - 1) / warps;
    // every resident warp needs its own visited table
    const uint64_t cap = std::min<uint64_t>((uint64_t)nb * ix->num_sms, ix->visited.slots / (uint32_t)warps);
    const int blocks = (int)std::min<uint64_t>(want, cap);
    // one search of this index at a time: its visited tables (and work
    // counter) are shared, so a launch on another stream waits for the last
    if (ix->busy_set && ix->busy_stream != stream) ANN_CUDA(cudaStreamWaitEvent(stream, ix->busy, 0));
    ANN_CUDA(cudaMemsetAsync(counter, 0, sizeof(uint32_t), stream));
    cudaError_t e;
    if (prof) {
        switch (ix->storage) {
        case ANN_F32: e = launch<ANN_F32, true>(a, warps, blocks, smem, stream); break;
        case ANN_F16: e = launch<ANN_F16, true>(a, warps, blocks, smem, stream); break;
        default: e = launch<ANN_E4M3, true>(a, warps, blocks, smem, stream); break;
        }
    } else {
        switch (ix->storage) {
        case ANN_F32: e = launch<ANN_F32>(a, warps, blocks, smem, stream); break;
        case ANN_F16: e = launch<ANN_F16>(a, warps, blocks, smem, stream); break;
        default: e = launch<ANN_E4M3>(a, warps, blocks, smem, stream); break;
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "search_kernel launch");
    ANN_CUDA(cudaEventRecord(ix->busy, stream));
    ix->busy_stream = stream;
    ix->busy_set = true;
    return ANN_OK;
}

ann_status serve_plan(ann_index *ix, const ann_search_params *maxp, uint32_t n_given_max, uint32_t n_streams,
                      void **plan)
{
    QParams q;
    ann_status s = derive_qparams(ix, maxp, n_given_max, &q);
    if (s != ANN_OK) return s;
    ServePlanImpl *pl = new ServePlanImpl();
    s = plan_args(ix, q, pl->a, pl->warps, pl->smem, pl->nb, true);
    if (s == ANN_OK) {
        pl->slots_per_launch = (uint32_t)(pl->nb * ix->num_sms * pl->warps);
        s = visited_pool_alloc(pl->visited, pl->slots_per_launch * std::max(1u, n_streams), kVisitedBits);
    }
    if (s != ANN_OK) { delete pl; return s; }
    pl->a.vtab = pl->visited.tab;
    pl->a.counter = ix->d_counter;
    pl->a.err = ix->d_error;
    pl->num_sms = ix->num_sms;
    pl->storage = ix->storage;
    *plan = pl;
    return ANN_OK;
}

void serve_plan_free(void *plan)
{
    ServePlanImpl *pl = static_cast<ServePlanImpl *>(plan);
    if (!pl) return;
    visited_pool_free(pl->visited);
    delete pl;
}

ann_status serve_launch(void *plan, const ServeRing &ring, uint32_t queries, cudaStream_t stream,
                        uint32_t stream_index)
{
    ServePlanImpl &pl = *static_cast<ServePlanImpl *>(plan);
    pl.a.slot_base = stream_index * pl.slots_per_launch;
    const uint64_t per_block = (uint64_t)pl.warps * ring.per_warp;
    const uint64_t want = ((uint64_t)queries + per_block - 1) / per_block;
    const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)pl.nb * pl.num_sms));
    cudaError_t e;
    switch (pl.storage) {
    case ANN_F32: e = launch_serve<ANN_F32>(pl, ring, blocks, stream); break;
    case ANN_F16: e = launch_serve<ANN_F16>(pl, ring, blocks, stream); break;
    default: e = launch_serve<ANN_E4M3>(pl, ring, blocks, stream); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "serve_kernel launch");
    return ANN_OK;
}

// The search with the index's own work counter and error word.
ann_status search_launch(ann_index *ix, const float *queries, uint32_t nq, const ann_search_params *p,
                         const uint32_t *given, uint32_t n_given, uint32_t *ids, float *dists,
                         ann_query_stats *stats, cudaStream_t stream)
{
    if (!ix) { set_error("ann_search: NULL index or params"); return ANN_EINVAL; }
    return search_launch_ex(ix, queries, nq, p, given, n_given, ids, dists, stats, stream, ix->d_counter,
                            ix->d_error, nullptr);
}

}  // namespace ann

extern "C" {

ann_status ann_search(ann_index *ix, const float *queries, uint32_t nq, const ann_search_params *p,
                      const uint32_t *given, uint32_t n_given, uint32_t *ids, float *dists, ann_query_stats *stats,
                      void *stream)
{
    if (!ix) { set_error("ann_search: NULL index"); return ANN_EINVAL; }
    int prev = -1;
    ann_status s = enter_device(ix->device, &prev, "ann_search");
    if (s != ANN_OK) return s;
    s = search_launch(ix, queries, nq, p, given, n_given, ids, dists, stats, (cudaStream_t)stream);
    leave_device(ix->device, prev);
    return s;
}

ann_status ann_search_host(ann_index *ix, const float *queries, uint32_t nq, const ann_search_params *p,
                           const uint32_t *given, uint32_t n_given, uint32_t *ids, float *dists, void *stream)
{
    if (!ix || !p) { set_error("ann_search_host: NULL index or params"); return ANN_EINVAL; }
    if (nq == 0) return ANN_OK;
    if (!queries || !ids || !dists) { set_error("ann_search_host: NULL buffers"); return ANN_EINVAL; }
    int prev = -1;
    ann_status s = enter_device(ix->device, &prev, "ann_search_host");
    if (s != ANN_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t qb = (size_t)nq * ix->dim * 4;
    const size_t gb = (given_entry(p->entry) && given) ? (size_t)nq * n_given * 4 : 0;
    const size_t ob = (size_t)nq * p->k * 4;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t need = up(qb) + up(gb) + 2 * up(ob);
    if (need > ix->ws_bytes) {
        if (ix->ws) cudaFree(ix->ws);
        ix->ws = nullptr;
        ix->ws_bytes = 0;
        cudaError_t e = cudaMalloc(&ix->ws, need);
        if (e != cudaSuccess) s = cuda_fail(e, "ann_search_host workspace");
        else ix->ws_bytes = need;
    }
    if (s == ANN_OK) {
        uint8_t *w = (uint8_t *)ix->ws;
        float *dq = (float *)w;
        uint32_t *dg = gb ? (uint32_t *)(w + up(qb)) : nullptr;
        uint32_t *di = (uint32_t *)(w + up(qb) + up(gb));
        float *dd = (float *)(w + up(qb) + up(gb) + up(ob));
        cudaError_t e = cudaMemcpyAsync(dq, queries, qb, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && gb) e = cudaMemcpyAsync(dg, given, gb, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) s = cuda_fail(e, "ann_search_host upload");
        if (s == ANN_OK) s = search_launch(ix, dq, nq, p, dg, n_given, di, dd, nullptr, st);
        if (s == ANN_OK) {
            e = cudaMemcpyAsync(ids, di, ob, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dists, dd, ob, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) s = cuda_fail(e, "ann_search_host download");
        }
    }
    leave_device(ix->device, prev);
    return s;
}

// The search with the per-phase clock profile: the same results as
// ann_search, from a build of the kernel that reads the SM clock at every
// phase boundary and charges each warp's elapsed cycles to (stage, phase).
ann_status ann_search_profile(ann_index *ix, const float *queries, uint32_t nq, const ann_search_params *p,
                              const uint32_t *given, uint32_t n_given, uint32_t *ids, float *dists,
                              uint64_t *cycles, void *stream)
{
    if (!ix || !cycles) { set_error("ann_search_profile: NULL index or cycles"); return ANN_EINVAL; }
    constexpr uint32_t kCells = ANN_PROFILE_STAGES * ANN_PROFILE_PHASES;
    for (uint32_t i = 0; i < kCells; ++i) cycles[i] = 0;
    int prev = -1;
    ann_status s = enter_device(ix->device, &prev, "ann_search_profile");
    if (s != ANN_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cells = (size_t)ix->visited.slots * kCells;
    unsigned long long *acc = nullptr;
    cudaError_t e = cudaMalloc(&acc, cells * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, cells * sizeof(unsigned long long), st);
    if (e != cudaSuccess) s = cuda_fail(e, "ann_search_profile counters");
    if (s == ANN_OK)
        s = search_launch_ex(ix, queries, nq, p, given, n_given, ids, dists, nullptr, st, ix->d_counter,
                             ix->d_error, acc);
    if (s == ANN_OK) {
        std::vector<unsigned long long> h(cells);
        e = cudaMemcpyAsync(h.data(), acc, cells * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(e, "ann_search_profile");
        else
            for (size_t i = 0; i < cells; ++i) cycles[i % kCells] += h[i];
    }
    if (acc) cudaFree(acc);
    leave_device(ix->device, prev);
    return s;
}

}  // extern "C"
