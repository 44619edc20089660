/*
 * CPU oracle for batched graph beam search with ghost staging and
 * direction-guided selection (PathWeaver, arXiv 2507.17094).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library. The CUDA library never
 * links, includes or calls it, and it includes nothing of the CUDA library.
 *
 * Everything here is written to be read against the paper, not to be fast:
 * plain loops, qsort for every sort, a bitmap for the visited set, FP32
 * distances with one fused multiply-add per element into four interleaved
 * partial sums (dist_f32), and FP64 for the exact ground truth.
 *
 * Parts and the passages they follow:
 *   - exact kNN ground truth ............ Section 2.1, Eq. 1 (squared L2)
 *   - beam search ....................... Section 2.2, Steps 1-4, Eq. 2
 *   - ghost staging ..................... Section 3.2.2
 *   - direction table + DGS + cool-down . Section 3.3.2 (a)-(c), Section 4
 *   - FP16 / FP8-E4M3 storage, rerank ... not in the paper (IEEE 754 binary16,
 *                                          OCP 8-bit floating point E4M3)
 * Readings where the paper is silent are stated beside the code.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_INVALID 0xFFFFFFFFu
#define OR_GHOST_TAG 0x67686F7374ull /* "ghost": separates the ghost-seed stream */

enum { OR_F32 = 0, OR_F16 = 1, OR_E4M3 = 2 };
enum { OR_UNEXPANDED = 0, OR_PARTIAL = 1, OR_EXPANDED = 2 };
enum { OR_ENTRY_RANDOM = 0, OR_ENTRY_GHOST = 1, OR_ENTRY_GIVEN_GHOST = 2, OR_ENTRY_GIVEN_BASE = 3 };

/* ------------------------------------------------------------------------ */
/* Number formats: round-to-nearest-even into a binary format with p       */
/* explicit mantissa bits and minimum normal exponent emin, computed in    */
/* double where every step below is exact.                                 */
/* ------------------------------------------------------------------------ */

/* Round |a| (finite, >= 0) to the format's grid; returns the rounded value. */
static double round_to_format(double a, int p, int emin)
{
    if (a == 0.0) return 0.0;
    int e2;
    (void)frexp(a, &e2);           /* a = f * 2^e2, f in [0.5, 1) */
    int E = e2 - 1;                /* floor(log2 a) */
    int qexp = (E < emin ? emin : E) - p;  /* grid spacing 2^qexp */
    double r = ldexp(a, -qexp);    /* exact: scaling by a power of two */
    double fl = floor(r);
    double frac = r - fl;          /* exact */
    double rounded;
    if (frac > 0.5) rounded = fl + 1.0;
    else if (frac < 0.5) rounded = fl;
    else rounded = (fmod(fl, 2.0) == 0.0) ? fl : fl + 1.0;  /* tie: even */
    return ldexp(rounded, qexp);
}

/* Encode an already-rounded magnitude v into (exponent field, mantissa). */
static uint32_t pack_format(double v, int p, int emin, int bias)
{
    if (v == 0.0) return 0;
    int e2;
    (void)frexp(v, &e2);
    int E = e2 - 1;
    if (E < emin) {                                   /* subnormal */
        return (uint32_t)ldexp(v, -(emin - p));
    }
    uint32_t mant = (uint32_t)(ldexp(v, p - E) - ldexp(1.0, p));
    return ((uint32_t)(E + bias) << p) | mant;
}

/* IEEE 754 binary16: p = 10, emin = -14, bias 15, max finite 65504. */
uint16_t oracle_f32_to_f16(float x)
{
    uint16_t sign = signbit(x) ? 0x8000u : 0;
    if (isnan(x)) return 0x7E00u;
    double a = fabs((double)x);
    if (isinf(x)) return sign | 0x7C00u;
    double v = round_to_format(a, 10, -14);
    if (v > 65504.0) return sign | 0x7C00u;           /* overflow -> inf */
    return sign | (uint16_t)pack_format(v, 10, -14, 15);
}

float oracle_f16_to_f32(uint16_t h)
{
    int s = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
    double v;
    if (e == 0) v = ldexp((double)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexp((double)(1024 + m), e - 25);
    return (float)(s ? -v : v);
}

/* OCP FP8 E4M3: p = 3, emin = -6, bias 7, no infinities, S.1111.111 = NaN,
 * max finite 448. Round to nearest even, then saturate to +-448. */
uint8_t oracle_f32_to_e4m3(float x)
{
    uint8_t sign = signbit(x) ? 0x80u : 0;
    if (isnan(x)) return 0x7Fu;
    double a = fabs((double)x);
    if (isinf(x) || a > 448.0) return sign | 0x7Eu;
    double v = round_to_format(a, 3, -6);
    if (v > 448.0) return sign | 0x7Eu;
    return sign | (uint8_t)pack_format(v, 3, -6, 7);
}

float oracle_e4m3_to_f32(uint8_t c)
{
    int s = (c >> 7) & 1, e = (c >> 3) & 15, m = c & 7;
    double v;
    if (e == 0) v = ldexp((double)m, -9);
    else if (e == 15 && m == 7) v = NAN;
    else v = ldexp((double)(8 + m), e - 10);
    return (float)(s ? -v : v);
}

/* Per-vector scale and codes.
 * FP16: scale 2^(floor(log2 max|x|) - 14) (clamped to a normal float), so the
 *   largest element lands in [2^14, 2^15) and integers up to 2^11 * scale
 *   stay exact; code = f16(x * 2^-e).
 * E4M3: scale = max|x| / 448 (FP32 division); code = e4m3_sat(x / scale).
 * An all-zero vector gets scale 1. */
void oracle_encode(const float *X, uint64_t n, uint32_t d, int storage, void *codes, float *scales)
{
    for (uint64_t r = 0; r < n; ++r) {
        const float *x = X + r * d;
        float mx = 0.0f;
        for (uint32_t i = 0; i < d; ++i) { float a = fabsf(x[i]); if (a > mx) mx = a; }
        if (storage == OR_F16) {
            int e = 0;
            if (mx > 0.0f) { int e2; (void)frexpf(mx, &e2); e = (e2 - 1) - 14; }
            if (e < -126) e = -126;
            float s = ldexpf(1.0f, e), inv = ldexpf(1.0f, -e);
            scales[r] = (mx > 0.0f) ? s : 1.0f;
            if (mx == 0.0f) inv = 1.0f;
            uint16_t *c = (uint16_t *)codes + r * d;
            for (uint32_t i = 0; i < d; ++i) c[i] = oracle_f32_to_f16(x[i] * inv);
        } else if (storage == OR_E4M3) {
            float s = (mx > 0.0f) ? mx / 448.0f : 1.0f;
            scales[r] = s;
            uint8_t *c = (uint8_t *)codes + r * d;
            for (uint32_t i = 0; i < d; ++i) c[i] = oracle_f32_to_e4m3(x[i] / s);
        }
    }
}

/* Stored value of element i = scale * decode(code), one FP32 multiply. */
void oracle_decode(const void *codes, const float *scales, uint64_t n, uint32_t d, int storage, float *out)
{
    for (uint64_t r = 0; r < n; ++r)
        for (uint32_t i = 0; i < d; ++i) {
            float v;
            if (storage == OR_F16) v = oracle_f16_to_f32(((const uint16_t *)codes)[r * d + i]);
            else if (storage == OR_E4M3) v = oracle_e4m3_to_f32(((const uint8_t *)codes)[r * d + i]);
            else v = ((const float *)codes)[r * d + i];
            out[r * d + i] = (storage == OR_F32) ? v : scales[r] * v;
        }
}

/* ------------------------------------------------------------------------ */
/* Direction table (Section 3.3.2 (a), Section 4): for edge u->v, bit b of */
/* word w is 1 iff x_v[32w+b] > x_u[32w+b]; pad bits past d are 0; a       */
/* missing neighbour (INVALID) has all words 0.                            */
/* ------------------------------------------------------------------------ */
void oracle_dir_table(const float *Xs, uint64_t n, uint32_t d, const uint32_t *G, uint32_t deg, uint32_t *dir)
{
    uint32_t w = (d + 31) / 32;
    for (uint64_t u = 0; u < n; ++u)
        for (uint32_t j = 0; j < deg; ++j) {
            uint32_t *out = dir + (u * deg + j) * w;
            for (uint32_t k = 0; k < w; ++k) out[k] = 0;
            uint32_t v = G[u * deg + j];
            if (v == OR_INVALID) continue;
            for (uint32_t i = 0; i < d; ++i)
                if (Xs[(uint64_t)v * d + i] > Xs[u * d + i]) out[i / 32] |= 1u << (i % 32);
        }
}

/* ------------------------------------------------------------------------ */
/* splitmix64 output function (Steele, Lea, Flood 2014; constants as        */
/* published by Vigna), used as a counter-based generator.                  */
/* ------------------------------------------------------------------------ */
uint64_t oracle_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* ------------------------------------------------------------------------ */
/* Parallel-for over queries (threads only split the query range).          */
/* ------------------------------------------------------------------------ */
typedef void (*or_task_fn)(void *ctx, uint32_t q, void *scratch);
typedef struct { or_task_fn fn; void *ctx; uint32_t nq; int tid, nthreads; size_t scratch_bytes; } or_job;

static void *or_worker(void *arg)
{
    or_job *j = (or_job *)arg;
    void *scratch = j->scratch_bytes ? malloc(j->scratch_bytes) : NULL;
    for (uint32_t q = (uint32_t)j->tid; q < j->nq; q += (uint32_t)j->nthreads) j->fn(j->ctx, q, scratch);
    free(scratch);
    return NULL;
}

static void or_parallel(or_task_fn fn, void *ctx, uint32_t nq, int threads, size_t scratch_bytes)
{
    if (threads < 1) threads = 1;
    if ((uint32_t)threads > nq) threads = nq ? (int)nq : 1;
    pthread_t *th = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    or_job *jobs = (or_job *)calloc((size_t)threads, sizeof(or_job));
    for (int t = 0; t < threads; ++t) {
        jobs[t] = (or_job){fn, ctx, nq, t, threads, scratch_bytes};
        if (t > 0) pthread_create(&th[t], NULL, or_worker, &jobs[t]);
    }
    or_worker(&jobs[0]);
    for (int t = 1; t < threads; ++t) pthread_join(th[t], NULL);
    free(th);
    free(jobs);
}

/* ------------------------------------------------------------------------ */
/* Exact kNN ground truth in FP64 (Eq. 1 with squared L2): ties by id.      */
/* ------------------------------------------------------------------------ */
typedef struct { const float *X; uint64_t n; uint32_t d; const float *Q; uint32_t k; uint32_t *ids; double *dists; } knn_ctx;

static void knn_one(void *vctx, uint32_t q, void *scratch)
{
    (void)scratch;
    knn_ctx *c = (knn_ctx *)vctx;
    uint32_t k = c->k, cnt = 0;
    uint32_t *ids = c->ids + (uint64_t)q * k;
    double *ds = c->dists + (uint64_t)q * k;
    const float *qv = c->Q + (uint64_t)q * c->d;
    for (uint64_t i = 0; i < c->n; ++i) {
        const float *x = c->X + i * c->d;
        double s = 0.0;
        for (uint32_t t = 0; t < c->d; ++t) { double df = (double)qv[t] - (double)x[t]; s += df * df; }
        if (cnt == k && !(s < ds[k - 1])) continue;  /* later ids lose ties */
        uint32_t pos = (cnt < k) ? cnt++ : k - 1;
        while (pos > 0 && ds[pos - 1] > s) { ds[pos] = ds[pos - 1]; ids[pos] = ids[pos - 1]; --pos; }
        ds[pos] = s;
        ids[pos] = (uint32_t)i;
    }
    for (uint32_t t = cnt; t < k; ++t) { ids[t] = OR_INVALID; ds[t] = INFINITY; }
}

void oracle_knn_f64(const float *X, uint64_t n, uint32_t d, const float *Q, uint32_t nq, uint32_t k,
                    uint32_t *ids, double *dists, int threads)
{
    knn_ctx c = {X, n, d, Q, k, ids, dists};
    or_parallel(knn_one, &c, nq, threads, 0);
}

/* FP64 squared distance of given (query, id) pairs; INVALID ids give +inf. */
void oracle_pair_dist_f64(const float *X, uint32_t d, const float *Q, uint32_t nq, uint32_t k,
                          const uint32_t *ids, double *out)
{
    for (uint32_t q = 0; q < nq; ++q)
        for (uint32_t j = 0; j < k; ++j) {
            uint32_t id = ids[(uint64_t)q * k + j];
            if (id == OR_INVALID) { out[(uint64_t)q * k + j] = INFINITY; continue; }
            double s = 0.0;
            for (uint32_t t = 0; t < d; ++t) {
                double df = (double)Q[(uint64_t)q * d + t] - (double)X[(uint64_t)id * d + t];
                s += df * df;
            }
            out[(uint64_t)q * k + j] = s;
        }
}

/* ------------------------------------------------------------------------ */
/* The search (Section 2.2 Steps 1-4 with Section 3.2.2 and 3.3.2).         */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t k;             /* results returned */
    uint32_t L;             /* itopk: priority-queue size l */
    uint32_t W;             /* search_width: parents r per iteration */
    uint32_t T;             /* max_iters */
    uint32_t m;             /* random seeds (entry 0); 0 = W * degree */
    uint32_t n_keep;        /* DGS keeps the top n_keep neighbours; >= degree disables DGS */
    uint32_t it_cool;       /* first cool-down iteration (no selection from here on) */
    uint32_t reexpand;      /* 1: DGS parents are PARTIAL and expand fully in cool-down */
    uint32_t entry;         /* 0 random, 1 ghost staging, 2 ghost staging from given seeds,
                               3 given base nodes as the Step-2 seeds */
    uint32_t Lg;            /* ghost queue size */
    uint32_t Tg;            /* ghost iterations, random ghost seeds */
    uint32_t Tg_given;      /* ghost iterations, given ghost seeds */
    uint32_t g;             /* ghost results that seed the base queue */
    uint32_t rerank;        /* 1: rescore the final queue against the FP32 originals */
    uint64_t seed;
    uint64_t qid_base;      /* global index of query 0 of this call */
    uint32_t Wg;            /* parents per ghost iteration */
    uint32_t min_match;     /* > 0: DGS keeps the neighbours scoring >= min_match instead of the top n_keep */
    float judge;            /* > 0: given ghost seeds whose ghost result is farther continue to Tg */
} oracle_params;

typedef struct {
    uint64_t n; uint32_t d, deg;
    const float *Xs;          /* stored (decoded) vectors, n x d */
    const float *X32;         /* FP32 originals for rerank (may be NULL) */
    const uint32_t *G;        /* n x deg */
    const uint32_t *dir;      /* n x deg x ceil(d/32) (may be NULL without DGS) */
    uint32_t nS, deg_g;
    const uint32_t *S;        /* ghost ids, ascending */
    const uint32_t *Gg;       /* nS x deg_g, over ghost indices */
} oracle_index;

typedef struct {
    uint64_t iters, parents, dgs_parents, vec_rows;
    uint64_t ghost_iters, ghost_parents, ghost_vec_rows, rerank_rows;
} oracle_counters;

typedef struct { float dist; uint32_t id; uint32_t state; } or_entry;

static int entry_cmp(const void *a, const void *b)
{
    const or_entry *x = (const or_entry *)a, *y = (const or_entry *)b;
    if (x->dist < y->dist) return -1;
    if (x->dist > y->dist) return 1;
    return (x->id < y->id) ? -1 : (x->id > y->id);
}

/* Eq. 2, squared, in FP32. The paper fixes no summation order; this one
 * keeps four partial sums, element i going to sum i mod 4 (one fma each, in
 * index order), and returns (s0 + s1) + (s2 + s3). */
static float dist_f32(const float *q, const float *x, uint32_t d)
{
    float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (uint32_t i = 0; i < d; ++i) { float df = q[i] - x[i]; s[i & 3] = fmaf(df, df, s[i & 3]); }
    return (s[0] + s[1]) + (s[2] + s[3]);
}

static int bit_get(const uint8_t *bm, uint64_t i) { return (bm[i >> 3] >> (i & 7)) & 1; }
static void bit_set(uint8_t *bm, uint64_t i) { bm[i >> 3] |= (uint8_t)(1u << (i & 7)); }

/* One graph (base or ghost) as the search sees it. */
typedef struct {
    uint64_t n; uint32_t d, deg;
    const float *Xs;            /* rows by local index */
    const uint32_t *S;          /* local -> stored-row map (ghost) or NULL (base) */
    const uint32_t *G;
    const uint32_t *dir;        /* NULL: no DGS on this graph */
} or_graph;

static const float *row_of(const or_graph *g, uint64_t v)
{
    uint64_t r = g->S ? g->S[v] : v;
    return g->Xs + r * g->d;
}

typedef struct {
    or_entry *buf; uint32_t cnt;      /* priority queue p, sorted by (dist, id) */
    or_entry *tmp;                    /* queue + candidates before truncation */
    uint8_t *visited;
} or_state;

/* Steps 3-4 repeated (Section 2.2) with DGS (Section 3.3.2 (b)-(c)).
 * Readings:
 *  - parents: the first W entries in queue order that are eligible;
 *    UNEXPANDED is always eligible, PARTIAL only in cool-down;
 *  - DGS scores a parent's neighbours by matching sign bits against the
 *    query's sign bits relative to the parent and keeps the top n_keep
 *    (ties by adjacency position); dropped neighbours are not marked visited;
 *  - with min_match > 0, DGS instead keeps every neighbour whose score is at
 *    least min_match (the similarity-criterion pruning the paper names as an
 *    alternative to a fixed top n in its comparison with static pruning,
 *    Section 6.3);
 *  - the cool-down starts at it_cool, or earlier once only PARTIAL entries
 *    are left, and then stays on;
 *  - stop when no eligible parent is left or after T iterations. */
static void or_iterate(const or_graph *g, const float *q, or_state *st, uint32_t L, uint32_t W, uint32_t T,
                       uint32_t n_keep, uint32_t min_match, uint32_t it_cool, uint32_t reexpand,
                       uint64_t *c_iters, uint64_t *c_parents, uint64_t *c_dgs, uint64_t *c_rows)
{
    uint32_t deg = g->deg, d = g->d, w = (d + 31) / 32;
    int dgs_on = g->dir != NULL && (min_match > 0 || n_keep < deg);
    int cool = 0;
    uint32_t par[64];
    int score[1024];
    uint8_t keep[1024];
    uint32_t qbits[64];
    for (uint32_t it = 0; it < T; ++it) {
        if (dgs_on && it >= it_cool) cool = 1;
        uint32_t np = 0;
        for (int pass = 0; pass < 2 && np == 0; ++pass) {
            for (uint32_t i = 0; i < st->cnt && np < W; ++i) {
                uint32_t s = st->buf[i].state;
                if (s == OR_UNEXPANDED || (cool && s == OR_PARTIAL)) par[np++] = i;
            }
            if (np == 0 && dgs_on && reexpand && !cool) {
                int any_partial = 0;
                for (uint32_t i = 0; i < st->cnt; ++i) any_partial |= st->buf[i].state == OR_PARTIAL;
                if (any_partial) cool = 1; else break;
            }
        }
        if (np == 0) break;
        ++*c_iters;
        int dgs_now = dgs_on && !cool;
        uint32_t nc = st->cnt;
        memcpy(st->tmp, st->buf, sizeof(or_entry) * st->cnt);
        for (uint32_t pi = 0; pi < np; ++pi) {
            or_entry *pe = &st->buf[par[pi]];
            pe->state = (dgs_now && reexpand) ? OR_PARTIAL : OR_EXPANDED;
            st->tmp[par[pi]].state = pe->state;
            uint32_t u = pe->id;
            ++*c_parents;
            for (uint32_t j = 0; j < deg; ++j) keep[j] = 1;
            if (dgs_now) {
                ++*c_dgs;
                const float *xu = row_of(g, u);
                for (uint32_t t = 0; t < w; ++t) qbits[t] = 0;
                for (uint32_t i = 0; i < d; ++i) if (q[i] > xu[i]) qbits[i / 32] |= 1u << (i % 32);
                for (uint32_t j = 0; j < deg; ++j) {
                    uint32_t v = g->G[(uint64_t)u * deg + j];
                    if (v == OR_INVALID) { score[j] = -1; continue; }
                    const uint32_t *dr = g->dir + ((uint64_t)u * deg + j) * w;
                    int diff = 0;
                    for (uint32_t t = 0; t < w; ++t) diff += __builtin_popcount(qbits[t] ^ dr[t]);
                    score[j] = (int)d - diff;
                }
                if (min_match > 0) {
                    for (uint32_t j = 0; j < deg; ++j) keep[j] = score[j] >= (int)min_match;
                } else {
                    /* rank j = #neighbours ahead of it (higher score, or equal and earlier) */
                    for (uint32_t j = 0; j < deg; ++j) {
                        uint32_t rank = 0;
                        for (uint32_t i = 0; i < deg; ++i)
                            if (score[i] > score[j] || (score[i] == score[j] && i < j)) ++rank;
                        keep[j] = rank < n_keep;
                    }
                }
            }
            for (uint32_t j = 0; j < deg; ++j) {
                uint32_t v = g->G[(uint64_t)u * deg + j];
                if (!keep[j] || v == OR_INVALID || bit_get(st->visited, v)) continue;
                bit_set(st->visited, v);
                st->tmp[nc].dist = dist_f32(q, row_of(g, v), d);
                st->tmp[nc].id = v;
                st->tmp[nc].state = OR_UNEXPANDED;
                ++nc;
                ++*c_rows;
            }
        }
        qsort(st->tmp, nc, sizeof(or_entry), entry_cmp);
        st->cnt = nc < L ? nc : L;
        memcpy(st->buf, st->tmp, sizeof(or_entry) * st->cnt);
    }
}

typedef struct {
    const oracle_index *ix; const float *Q; const oracle_params *p;
    const uint32_t *given; uint32_t P;
    uint32_t *ids; float *dists; oracle_counters *cnt;
} search_ctx;

static void search_one(void *vctx, uint32_t qi, void *scratch)
{
    (void)scratch;
    search_ctx *c = (search_ctx *)vctx;
    const oracle_index *ix = c->ix;
    const oracle_params *p = c->p;
    const float *q = c->Q + (uint64_t)qi * ix->d;
    uint64_t qid = p->qid_base + qi;
    oracle_counters cn = {0};
    uint32_t m = p->m ? p->m : p->W * ix->deg;
    uint64_t cap = (uint64_t)p->L + (uint64_t)p->W * ix->deg + m + p->Lg + (uint64_t)p->Wg * ix->deg_g + c->P + 16;
    or_state st;
    st.buf = (or_entry *)malloc(sizeof(or_entry) * cap);
    st.tmp = (or_entry *)malloc(sizeof(or_entry) * cap);
    st.visited = (uint8_t *)calloc((size_t)(ix->n / 8 + 1), 1);
    st.cnt = 0;

    or_graph base = {ix->n, ix->d, ix->deg, ix->Xs, NULL, ix->G, ix->dir};
    int use_ghost = (p->entry == OR_ENTRY_GHOST || p->entry == OR_ENTRY_GIVEN_GHOST) && ix->nS > 0;
    const uint32_t *given_base = (p->entry == OR_ENTRY_GIVEN_BASE && c->given) ? c->given + (uint64_t)qi * c->P : NULL;
    if (given_base && given_base[0] == OR_INVALID) given_base = NULL;   /* fall back to random seeds */
    if (!use_ghost) {
        /* Steps 1-3: m random nodes, deduplicated by the visited set without
         * redraw, sorted into the queue. Node j of query qid is
         * splitmix64(key ^ (qid << 32) ^ j) mod n with key = splitmix64(seed):
         * mixing the seed first keeps seeds that differ in low bits from
         * drawing permutations of one seed set. With given base nodes (the
         * first node of an extended path, Section 3.1.2), those nodes are the
         * seeds instead: invalid or out-of-range ones are skipped. */
        const uint64_t key = oracle_splitmix64(p->seed);
        uint32_t nc = 0;
        const uint32_t ms = given_base ? c->P : m;
        for (uint32_t j = 0; j < ms; ++j) {
            uint64_t v;
            if (given_base) {
                if (given_base[j] == OR_INVALID || given_base[j] >= ix->n) continue;
                v = given_base[j];
            } else {
                v = oracle_splitmix64(key ^ (qid << 32) ^ (uint64_t)j) % ix->n;
            }
            if (bit_get(st.visited, v)) continue;
            bit_set(st.visited, v);
            st.tmp[nc].dist = dist_f32(q, ix->Xs + v * ix->d, ix->d);
            st.tmp[nc].id = (uint32_t)v;
            st.tmp[nc].state = OR_UNEXPANDED;
            ++nc;
            ++cn.vec_rows;
        }
        qsort(st.tmp, nc, sizeof(or_entry), entry_cmp);
        st.cnt = nc < p->L ? nc : p->L;
        memcpy(st.buf, st.tmp, sizeof(or_entry) * st.cnt);
    } else {
        /* Ghost staging (Section 3.2.2): search the ghost graph first, from
         * random ghost nodes or from given ones, with width Wg and no DGS. */
        or_graph gg = {ix->nS, ix->d, ix->deg_g, ix->Xs, ix->S, ix->Gg, NULL};
        uint8_t *gvis = (uint8_t *)calloc(ix->nS / 8 + 1, 1);
        or_state gs = {st.buf, 0, st.tmp, gvis};
        uint32_t nc = 0, Tg = p->Tg;
        int judged = 0;
        const uint32_t *given = (p->entry == OR_ENTRY_GIVEN_GHOST && c->given) ? c->given + (uint64_t)qi * c->P : NULL;
        if (given && given[0] != OR_INVALID) {
            Tg = p->Tg_given;
            judged = p->judge > 0.0f && p->Tg > p->Tg_given;
            for (uint32_t j = 0; j < c->P; ++j) {
                uint32_t v = given[j];
                if (v == OR_INVALID || v >= ix->nS || bit_get(gvis, v)) continue;
                bit_set(gvis, v);
                st.tmp[nc] = (or_entry){dist_f32(q, row_of(&gg, v), ix->d), v, OR_UNEXPANDED};
                ++nc; ++cn.ghost_vec_rows;
            }
        } else {
            const uint64_t gkey = oracle_splitmix64(p->seed ^ OR_GHOST_TAG);
            for (uint32_t j = 0; j < ix->deg_g; ++j) {
                uint64_t v = oracle_splitmix64(gkey ^ (qid << 32) ^ (uint64_t)j) % ix->nS;
                if (bit_get(gvis, v)) continue;
                bit_set(gvis, v);
                st.tmp[nc] = (or_entry){dist_f32(q, row_of(&gg, v), ix->d), (uint32_t)v, OR_UNEXPANDED};
                ++nc; ++cn.ghost_vec_rows;
            }
        }
        qsort(st.tmp, nc, sizeof(or_entry), entry_cmp);
        gs.cnt = nc < p->Lg ? nc : p->Lg;
        memcpy(gs.buf, st.tmp, sizeof(or_entry) * gs.cnt);
        uint64_t no_dgs = 0;
        or_iterate(&gg, q, &gs, p->Lg, p->Wg ? p->Wg : 1, Tg, ix->deg_g, 0, 0, 0,
                   &cn.ghost_iters, &cn.ghost_parents, &no_dgs, &cn.ghost_vec_rows);
        /* The judge of given seeds: if the ghost queue's best node is farther
         * than the judge distance, the ghost stage goes on from where it is,
         * up to Tg iterations in all, as plain ghost staging would. */
        if (judged && gs.cnt > 0 && gs.buf[0].dist > p->judge)
            or_iterate(&gg, q, &gs, p->Lg, p->Wg ? p->Wg : 1, p->Tg - p->Tg_given, ix->deg_g, 0, 0, 0,
                       &cn.ghost_iters, &cn.ghost_parents, &no_dgs, &cn.ghost_vec_rows);
        /* Transition: the top g ghost results, as base ids with their
         * distances, become the base queue; only they are marked visited. */
        uint32_t g = p->g < gs.cnt ? p->g : gs.cnt;
        for (uint32_t i = 0; i < g; ++i) {
            st.tmp[i].dist = gs.buf[i].dist;
            st.tmp[i].id = ix->S[gs.buf[i].id];
            st.tmp[i].state = OR_UNEXPANDED;
        }
        qsort(st.tmp, g, sizeof(or_entry), entry_cmp);
        st.cnt = g < p->L ? g : p->L;
        memcpy(st.buf, st.tmp, sizeof(or_entry) * st.cnt);
        for (uint32_t i = 0; i < st.cnt; ++i) bit_set(st.visited, st.buf[i].id);
        free(gvis);
    }

    or_iterate(&base, q, &st, p->L, p->W, p->T, p->n_keep, p->min_match, p->it_cool, p->reexpand,
               &cn.iters, &cn.parents, &cn.dgs_parents, &cn.vec_rows);

    /* Output (Step 4's end): the top k; with rerank, the whole queue is
     * rescored against the FP32 originals and re-sorted first. */
    if (p->rerank && ix->X32) {
        for (uint32_t i = 0; i < st.cnt; ++i)
            st.buf[i].dist = dist_f32(q, ix->X32 + (uint64_t)st.buf[i].id * ix->d, ix->d);
        cn.rerank_rows += st.cnt;
        qsort(st.buf, st.cnt, sizeof(or_entry), entry_cmp);
    }
    for (uint32_t j = 0; j < p->k; ++j) {
        c->ids[(uint64_t)qi * p->k + j] = j < st.cnt ? st.buf[j].id : OR_INVALID;
        c->dists[(uint64_t)qi * p->k + j] = j < st.cnt ? st.buf[j].dist : INFINITY;
    }
    if (c->cnt) c->cnt[qi] = cn;
    free(st.buf);
    free(st.tmp);
    free(st.visited);
}

/* Returns 0 on success, -1 on arguments the search cannot run with. */
int oracle_search(const oracle_index *ix, const float *Q, uint32_t nq, const oracle_params *p,
                  const uint32_t *given_ghost_seeds, uint32_t P, uint32_t *ids, float *dists,
                  oracle_counters *counters, int threads)
{
    if (!ix || !p || p->k == 0 || p->L == 0 || p->k > p->L || p->W == 0 || p->W > 64 || ix->deg > 1024 ||
        ix->d == 0 || ix->n == 0 || (ix->d + 31) / 32 > 64 || p->min_match > ix->d)
        return -1;
    search_ctx c = {ix, Q, p, given_ghost_seeds, P, ids, dists, counters};
    or_parallel(search_one, &c, nq, threads, 0);
    return 0;
}
