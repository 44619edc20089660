/*
 * ann.h — C ABI of the GB300 graph-search library (libann.so).
 *
 * Batched best-first (beam) search over a fixed-degree proximity graph, with
 * ghost staging and direction-guided selection, after PathWeaver
 * (arXiv 2507.17094). All search work runs in the library's own CUDA kernels
 * for sm_103a; there is no CPU fallback.
 *
 * Conventions for every call:
 *   - Ids are uint32; ANN_INVALID_ID marks "no result". Distances are SQUARED
 *     L2 (Eq. 2 without the root; the ranking is the same).
 *   - Results are ordered by (distance, id) ascending.
 *   - "device" pointers are CUDA device memory of the index's device; "host"
 *     pointers are ordinary (preferably pinned) host memory. The caller owns
 *     every buffer it passes; the library owns the index and its scratch.
 *   - Calls return ann_status. Argument errors are found on the host before
 *     any launch and return ANN_EINVAL with nothing launched; the message is
 *     in ann_last_error() (thread-local). Work on a stream is asynchronous;
 *     device-side failures (a bounded wait that ran out) are recorded in the
 *     index's device error word and reported by ann_sync().
 *   - An index is not thread-safe: one host thread drives it at a time.
 */
#ifndef ANN_H
#define ANN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ANN_INVALID_ID 0xFFFFFFFFu
#define ANN_MAX_ITOPK 512u
#define ANN_MAX_DIM 1024u
#define ANN_MAX_DEGREE 128u
#define ANN_MAX_WIDTH 8u
#define ANN_MAX_SHARDS 16u      /* shards in one path-extension ring */
#define ANN_MAX_FORWARD 8u      /* nodes forwarded per query between shards */

typedef enum {
    ANN_OK = 0,
    ANN_EINVAL = 1,    /* bad argument; nothing was launched */
    ANN_ENOMEM = 2,    /* device or host allocation failed */
    ANN_ECUDA = 3,     /* a CUDA runtime call failed */
    ANN_EIO = 4,       /* index file unreadable or malformed */
    ANN_ETIMEOUT = 5,  /* a bounded device wait ran out (reported by ann_sync) */
    ANN_EBUSY = 6,     /* serving: not admissible right now */
    ANN_EDEVICE = 7    /* no usable CUDA device */
} ann_status;

typedef enum { ANN_F32 = 0, ANN_F16 = 1, ANN_E4M3 = 2 } ann_storage;

typedef enum {
    ANN_ENTRY_RANDOM = 0,      /* Section 2.2 Step 2: m random nodes */
    ANN_ENTRY_GHOST = 1,       /* Section 3.2.2: ghost staging from random ghost nodes */
    ANN_ENTRY_GIVEN_GHOST = 2, /* ghost staging from caller-given ghost nodes (learned entry);
                                  a query whose first given id is ANN_INVALID_ID falls back to 1 */
    ANN_ENTRY_GIVEN_BASE = 3   /* Step 2 from caller-given base nodes instead of random ones (the
                                  start of an extended path, Section 3.1.2: the node I(z) of this
                                  shard linked to the previous shard's result z); invalid or
                                  out-of-range ids are skipped, and a query whose first given id is
                                  ANN_INVALID_ID falls back to 0 */
} ann_entry;

/* Search parameters. Paper notation: itopk = l (queue size), search_width =
 * r (parents per iteration), max_iters = the iteration cap (Section 2.2). */
typedef struct {
    uint32_t k;                 /* results per query, 1 <= k <= itopk */
    uint32_t itopk;             /* queue size l, 1..ANN_MAX_ITOPK */
    uint32_t search_width;      /* parents per iteration r, 1..ANN_MAX_WIDTH */
    uint32_t max_iters;         /* iteration cap T (0 = seeds only) */
    uint32_t num_seeds;         /* random seeds m (entry 0); 0 = search_width * degree */
    float dgs_discard;          /* DGS discard ratio rho in [0,1); 0 disables DGS (Section 3.3.2) */
    float dgs_cooldown;         /* cool-down fraction c of max_iters without selection (default 0.3) */
    uint32_t dgs_reexpand;      /* 1: parents expanded under DGS expand fully again in cool-down */
    uint32_t entry;             /* ann_entry */
    uint32_t ghost_itopk;       /* ghost queue size; 0 = min(itopk, 64) */
    uint32_t ghost_max_iters;   /* ghost iterations from random ghost seeds (default 16) */
    uint32_t ghost_max_iters_given; /* ghost iterations from given ghost seeds (default 4) */
    uint32_t ghost_seeds_out;   /* ghost results that seed the base queue; 0 = ghost_itopk */
    uint32_t rerank;            /* 1: rescore the final queue on the FP32 originals (low precision) */
    uint64_t seed;              /* search RNG seed (splitmix64 counter stream) */
    uint64_t qid_base;          /* global index of query 0 of this call (RNG stream per query) */
    uint32_t ghost_search_width; /* parents per ghost iteration, 1..ANN_MAX_WIDTH (0 or default: 1) */
    float dgs_min_match;        /* DGS by similarity (the paper's alternative to a fixed top n, in its
                                   comparison with static pruning, Section 6.3): f in (0,1] keeps the
                                   neighbours whose direction agrees with the query's in at least
                                   ceil(f * dim) dimensions; 0 = the top-n rule of dgs_discard.
                                   Setting both is ANN_EINVAL. */
    float ghost_judge;          /* ghost staging as the judge of given ghost seeds (entry 2; no
                                   counterpart in the paper): when > 0, a query whose ghost queue,
                                   after the ghost_max_iters_given iterations from its given seeds,
                                   holds no node nearer than this squared distance continues the
                                   ghost stage up to ghost_max_iters iterations in all (as plain
                                   ghost staging, from the state reached). 0 = off; finite, >= 0. */
} ann_search_params;

/* Per-query event counters (exact counts of the work done). */
typedef struct {
    uint32_t iters, parents, dgs_parents, vec_rows;
    uint32_t ghost_iters, ghost_parents, ghost_vec_rows, rerank_rows;
    uint32_t hash_resets, status;
} ann_query_stats;

typedef struct ann_index ann_index;

/* Fill *p with the defaults above (k 10, itopk 64, width 1, 64 iterations,
 * DGS off, cool-down 0.3, random entry, ghost 16/4 iterations). */
void ann_default_params(ann_search_params *p);

/* Build an index on `device` from host arrays (Section 2.1 takes the graph as
 * given; Section 3.2.2 the ghost sample and its graph; Section 3.3.2 (a) the
 * direction table, which is built here on the GPU).
 *   vectors      host, n x dim FP32, row-major (the source values)
 *   graph        host, n x degree uint32 (ANN_INVALID_ID = missing edge)
 *   ghost_ids    host, n_ghost distinct node ids in ascending order (may be NULL if n_ghost = 0)
 *   ghost_graph  host, n_ghost x ghost_degree uint32 over ghost indices 0..n_ghost-1
 *   storage      ANN_F32 / ANN_F16 / ANN_E4M3 (codes with a per-vector FP32 scale)
 *   keep_fp32    1: also keep the FP32 originals on the device for rerank
 *   build_dir    1: build the direction table (needed for DGS)
 * Errors: ANN_EINVAL (sizes, ids out of range), ANN_ENOMEM, ANN_ECUDA, ANN_EDEVICE. */
ann_status ann_index_create(int device, ann_storage storage, uint64_t n, uint32_t dim, uint32_t degree,
                            const float *vectors, const uint32_t *graph, uint32_t n_ghost,
                            const uint32_t *ghost_ids, uint32_t ghost_degree, const uint32_t *ghost_graph,
                            uint32_t keep_fp32, uint32_t build_dir, ann_index **out);

/* Load an index file (magic "ANNIDX01", then u64 n, u32 dim, degree, n_ghost,
 * ghost_degree, then the arrays of ann_index_create in that order, all
 * little-endian) and build it as ann_index_create does. Errors: ANN_EIO plus
 * those of ann_index_create. */
ann_status ann_index_load(const char *path, int device, ann_storage storage, uint32_t keep_fp32,
                          uint32_t build_dir, ann_index **out);

/* Release the index and all of its device memory; waits first for the last
 * search launched on it. NULL is accepted (ANN_OK). The caller must not use
 * the handle afterwards. */
ann_status ann_index_free(ann_index *index);

/* Shape of the index; any output pointer may be NULL. ANN_EINVAL for a NULL
 * index. storage receives the ann_storage value. */
ann_status ann_index_info(const ann_index *index, uint64_t *n, uint32_t *dim, uint32_t *degree,
                          uint32_t *storage, uint32_t *n_ghost, uint32_t *ghost_degree);

/* Copy one of the index's device arrays to host memory (for inspection):
 *   0 codes (n x dim, element type of the storage, row stride padded away)
 *   1 scales (n floats; FP16/E4M3 only)
 *   2 direction table (n x degree x ceil(dim/32) uint32)
 *   3 ghost codes (n_ghost x dim)   4 ghost scales (n_ghost floats)
 * `bytes` must equal the array's size. */
ann_status ann_index_export(const ann_index *index, int which, void *host_dst, uint64_t bytes);

/* Batched search (Section 2.2 Steps 1-4, Section 3.2.2, Section 3.3.2).
 *   queries      device, nq x dim FP32 row-major
 *   given_seeds  device, nq x n_given ghost indices (entry ANN_ENTRY_GIVEN_GHOST) or base
 *                node ids (entry ANN_ENTRY_GIVEN_BASE), else NULL
 *   ids, dists   device, nq x k (caller-owned)
 *   stats        device, nq ann_query_stats, or NULL
 *   stream       cudaStream_t (NULL = legacy default stream)
 * Asynchronous on `stream`; returns after the launch. The launch shape is
 * chosen per call from the parameters (rows gathered per round: 16, or 8 of
 * rows over 1 KB, halved when that admits more resident warps per SM); the
 * environment variable ANN_STAGE_ROWS fixes the rows per round instead (for
 * experiments). Results do not depend on the shape. */
ann_status ann_search(ann_index *index, const float *queries, uint32_t nq, const ann_search_params *params,
                      const uint32_t *given_seeds, uint32_t n_given, uint32_t *ids, float *dists,
                      ann_query_stats *stats, void *stream);

/* The same search with HOST buffers: copies the queries in, searches, copies
 * the results out, and synchronises `stream` before returning. Uses a device
 * workspace owned by the index (grown on demand). */
ann_status ann_search_host(ann_index *index, const float *queries, uint32_t nq,
                           const ann_search_params *params, const uint32_t *given_seeds, uint32_t n_given,
                           uint32_t *ids, float *dists, void *stream);

/* The paper has no counterpart to this call. ann_search_host without any
 * device allocation, for callers that must not allocate device memory on
 * their request path (a server that reserves all device memory at start-up,
 * code under an external memory budget, a host thread with a deadline that
 * cannot afford the device synchronisation cudaMalloc/cudaFree may cause).
 * Queries, results, the kernel's work counter and its error word live in one
 * fixed device array of ANN_NOALLOC_SCRATCH_BYTES per GPU, held until the
 * process exits. A call needing more staging than that (256 + nq*dim*4 +
 * 2*nq*k*4 bytes, parts rounded up to 256) returns ANN_EINVAL: split the
 * batch. All calls on a device share the array, so calls that overlap on the
 * GPU (other streams or host threads) race; each call clears what it relies
 * on. The first call on a device looks up the array's address there; make it
 * before any stream capture. Given ghost seeds are not supported here.
 * Synchronous: returns after the results are in the host buffers. */
#define ANN_NOALLOC_SCRATCH_BYTES (8u << 20)
ann_status ann_search_host_noalloc(ann_index *index, const float *queries, uint32_t nq,
                                   const ann_search_params *params, uint32_t *ids, float *dists, void *stream);

/* Per-phase time of the search (the measurement of Section 5.5, Fig. 11:
 * SM clock readings around the parts of the kernel). The same search and
 * results as ann_search (ids, dists device nq x k; no stats), run by a build
 * of the kernel that reads the clock at every phase boundary and adds each
 * warp's elapsed cycles to cycles[stage * ANN_PROFILE_PHASES + phase] (host,
 * ANN_PROFILE_STAGES x ANN_PROFILE_PHASES uint64, summed over all warps;
 * zeroed first). Stages: 0 ghost stage, 1 base graph, 2 rerank and output.
 * Phases: 0 parent selection and the adjacency / direction / parent-row
 * fetch, 1 DGS selection, 2 visited-set test-and-insert (and seeding),
 * 3 waiting for gathered rows, 4 distances, 5 merge, 6 the rest (query load,
 * set clears, stage switch, output). Cycles are per-warp wall time, so they
 * include time a warp waits while others issue. Allocates a temporary of
 * 192 bytes per warp slot; synchronous on `stream`. */
#define ANN_PROFILE_STAGES 3u
#define ANN_PROFILE_PHASES 8u
ann_status ann_search_profile(ann_index *index, const float *queries, uint32_t nq, const ann_search_params *params,
                              const uint32_t *given_seeds, uint32_t n_given, uint32_t *ids, float *dists,
                              uint64_t *cycles, void *stream);

/* ------------------------------------------------------------------------
 * Pipelining-based path extension (Section 3.1.2, Eq. 3, Section 4) with
 * the shards as separate indexes on one GPU. The dataset is partitioned into
 * N shards (each an ann_index over its own points, local ids 0..n_i-1, with
 * its own graph and, optionally, ghost set); shard i links every node u to
 * I(u), its nearest node in shard (i + 1) mod N (Eq. 3). A search splits the
 * queries into N chunks (chunk c = rows [c nq / N, (c + 1) nq / N)); chunk c
 * starts on shard c with the entry of `params` (random or ghost staging) and
 * continues on shards c + 1, ... from I(z) for the best n_forward nodes z of
 * its previous local result (the paper forwards one), until it has searched
 * every shard; the N local top-k lists are reduced to the top k by
 * (distance, dataset id). With n_forward = 0 every shard starts from the
 * entry of `params`: the paper's baseline sharding. The RNG stream of query
 * row r is qid_base + r on every shard.
 * ------------------------------------------------------------------------ */
typedef struct ann_shards ann_shards;
/* A ring over n_shards (1..ANN_MAX_SHARDS) indexes on one device with equal
 * dimension and storage; global_ids[i] (host, n_i uint32) maps shard i's
 * local ids to dataset ids (copied). The ring does not own the indexes:
 * free it before them. Searches of the ring use the indexes' own visited
 * tables, so do not search a shard's index on its own while a ring search
 * of it runs. */
ann_status ann_shards_create(ann_index *const *shards, uint32_t n_shards, const uint32_t *const *global_ids,
                             ann_shards **out);
ann_status ann_shards_free(ann_shards *shards);
/* Build every shard's links as Section 4 does: node u of shard i (its FP32
 * vector; the index must keep FP32 originals unless its storage is FP32) is
 * the query of a search of shard i + 1 with `params` (k is taken as 1; entry
 * random or ghost staging; node u's RNG stream is qid_base + u), and I(u) is
 * the top-1 result. Synchronous on `stream`. */
ann_status ann_shards_link(ann_shards *shards, const ann_search_params *params, void *stream);
/* Set shard `shard`'s links from host memory (n_shard local ids of the next
 * shard, e.g. the exact Eq. 3 links); ANN_EINVAL for an id out of range. */
ann_status ann_shards_set_links(ann_shards *shards, uint32_t shard, const uint32_t *links);
/* Host copy of shard `shard`'s links (n_shard uint32). */
ann_status ann_shards_get_links(const ann_shards *shards, uint32_t shard, uint32_t *links);
/* The sharded search. queries device nq x dim; ids (dataset ids) and dists
 * device nq x k; stats device N x nq ann_query_stats (row t: every query's
 * stage-t search) or NULL. n_forward <= min(k, ANN_MAX_FORWARD); with
 * n_forward > 0 every shard must be linked. Asynchronous on `stream` (the
 * chunks run on the ring's own streams, joined back to `stream`). */
ann_status ann_shards_search(ann_shards *shards, const float *queries, uint32_t nq, const ann_search_params *params,
                             uint32_t n_forward, uint32_t *ids, float *dists, ann_query_stats *stats, void *stream);

/* ------------------------------------------------------------------------
 * Graph construction (the paper takes the proximity graph as given, Section
 * 2.1, and times its build beside the method's preprocessing, Section 5.7).
 * ------------------------------------------------------------------------ */
/* Exact kNN lists: ids (device, n x K) gets, for every node u of X (device,
 * n x dim FP32 row-major), the K other nodes nearest to u by squared L2 in
 * FP32 (one fused multiply-add per element, index order), ordered by
 * (distance, id). Brute force: O(n^2 dim) work, for building graphs of up to
 * a few million nodes. 2 <= n < 2^32 - 1, 1 <= K < n, K <= 2 ANN_MAX_DEGREE,
 * and (96 rows x (dim + 1) + 32 K x 2) x 4 bytes of shared memory must fit a
 * block (ANN_EINVAL otherwise). Asynchronous on `stream`. */
ann_status ann_knn_exact(const float *X, uint64_t n, uint32_t dim, uint32_t K, uint32_t *ids, void *stream);
/* Prune kNN lists (device, n x K; each row distinct ids, ANN_INVALID_ID
 * allowed) to a fixed-degree graph (device, n x degree): edge u -> v at rank
 * r is detoured via the node at rank a < r of u's list when v sits in that
 * node's list at a rank c < r; u's list is ordered by (number of detours,
 * rank) and its first degree / 2 entries are kept; every kept edge w -> v,
 * at position p of w's kept part, offers w to v, and v takes its offers in
 * (p, w) order, at most degree - degree / 2; v's row is its kept part, then
 * those reverse edges, then the rest of its ordered list, with repeats and v
 * itself dropped, cut to `degree` and padded with ANN_INVALID_ID. degree <=
 * min(K, ANN_MAX_DEGREE), K <= 2 ANN_MAX_DEGREE. Allocates temporaries of
 * about n (K + 4 degree) x 4 bytes; synchronous on `stream`. */
ann_status ann_graph_prune(const uint32_t *knn, uint64_t n, uint32_t K, uint32_t degree, uint32_t *graph,
                           void *stream);

/* Ghost index of each node id (device ids, n) by binary search over the
 * ascending ghost ids, into out (device, n); ANN_INVALID_ID where an id is
 * not a ghost node. Turns ghost-staging results into training labels. */
ann_status ann_ghost_index_of(const ann_index *index, const uint32_t *ids, uint32_t n, uint32_t *out, void *stream);

/* Synchronise `stream` and report (then clear) the index's device error
 * word: ANN_OK, or ANN_ETIMEOUT if a bounded device wait ran out. */
ann_status ann_sync(ann_index *index, void *stream);

/* Check the device-failure path (not in the paper): one warp waits about
 * 1 ms on a barrier that nothing completes, the bounded wait runs out and
 * records a timeout in the index's device error word, and ann_sync reports
 * it (then clears it). Returns ANN_OK when all of that happened, ANN_EDEVICE
 * if the timeout was not reported, or the CUDA error. Synchronises the
 * device; the index stays usable. */
ann_status ann_selftest_timeout(ann_index *index);

/* Preprocessing primitives on caller-owned device memory (Section 3.3.2 (a)
 * and the low-precision codec), used by ann_index_create.
 * ann_encode: x (n x dim FP32) -> codes (n x dim FP16 or E4M3, dense rows) +
 *   scales (n floats). FP16 scale 2^(floor(log2 max|x|) - 14); E4M3 scale
 *   max|x| / 448 with round-to-nearest-even saturating codes.
 * ann_dir_table: stored vectors (codes + scales, or FP32 when storage is
 *   ANN_F32 and scales NULL), graph (n x degree) -> dir (n x degree x
 *   ceil(dim/32) uint32); bit b of word w is 1 iff x_v[32w+b] > x_u[32w+b]. */
ann_status ann_encode(const float *x, uint64_t n, uint32_t dim, ann_storage storage, void *codes,
                      float *scales, void *stream);
ann_status ann_dir_table(const void *vectors, const float *scales, ann_storage storage, uint64_t n,
                         uint32_t dim, const uint32_t *graph, uint32_t degree, uint32_t *dir, void *stream);

/* ------------------------------------------------------------------------
 * Learned entry (not in the paper; builds on the ghost set of Section
 * 3.2.2): an MLP in_dim -> hidden1 -> hidden2 -> out_dim (ReLU, one logit
 * per ghost node), BF16 tensor-core GEMMs with FP32 accumulation, FP32
 * master weights trained with AdamW on softmax cross-entropy. Its top-P
 * ghost nodes become `given_seeds` of ann_search (ANN_ENTRY_GIVEN_GHOST).
 * All sizes must be positive multiples of 8. Weights are row-major
 * (W1: hidden1 x in_dim, W2: hidden2 x hidden1, W3: out_dim x hidden2).
 * ------------------------------------------------------------------------ */
typedef struct ann_mlp ann_mlp;

ann_status ann_mlp_create(int device, uint32_t in_dim, uint32_t hidden1, uint32_t hidden2, uint32_t out_dim,
                          uint32_t max_batch, ann_mlp **out);
ann_status ann_mlp_free(ann_mlp *mlp);
/* Host FP32 parameters in; resets the optimizer state and the step count. */
ann_status ann_mlp_set_params(ann_mlp *mlp, const float *W1, const float *b1, const float *W2, const float *b2,
                              const float *W3, const float *b3);
/* Host copies of the parameters (which = 0) or of the last training step's
 * gradients (which = 1); a NULL pointer skips that array. Synchronises. */
ann_status ann_mlp_get(const ann_mlp *mlp, int which, float *W1, float *b1, float *W2, float *b2, float *W3,
                       float *b3);
/* logits (device, n x out_dim FP32) of queries x (device, n x in_dim FP32); n <= max_batch. */
ann_status ann_mlp_forward(ann_mlp *mlp, const float *x, uint32_t n, float *logits, void *stream);
/* One AdamW step on a minibatch: x (device, n x in_dim), labels (device, n
 * indices < out_dim), n a multiple of 8 <= max_batch; the batch's mean
 * cross-entropy goes to *loss (device float, may be NULL). */
ann_status ann_mlp_train_step(ann_mlp *mlp, const float *x, const uint32_t *labels, uint32_t n, float lr,
                              float beta1, float beta2, float eps, float weight_decay, float *loss, void *stream);
/* Fused prediction: seeds (device, n x P) = the P highest-logit ghost indices
 * (ties: smaller index), pmax (device, n, may be NULL) = the largest softmax
 * probability; a query with pmax < tau gets ANN_INVALID_ID as its first seed
 * (ann_search then falls back to random ghost seeds). 1 <= P <= 8. The
 * (n x out_dim) logits are never written to memory. */
ann_status ann_mlp_predict(ann_mlp *mlp, const float *x, uint32_t n, uint32_t P, float tau, uint32_t *seeds,
                           float *pmax, void *stream);
/* Epochs of minibatch AdamW over (x, labels) (device, n rows, n >= 8): each
 * epoch visits the rows in a fresh seeded order, in batches of `batch` (a
 * multiple of 8 <= max_batch); epoch_loss (host, `epochs` floats, may be
 * NULL) receives each epoch's mean batch loss. Synchronous. */
ann_status ann_mlp_train_epochs(ann_mlp *mlp, const float *x, const uint32_t *labels, uint32_t n, uint32_t batch,
                                uint32_t epochs, float lr, float beta1, float beta2, float eps, float weight_decay,
                                uint64_t seed, float *epoch_loss, void *stream);
/* Synchronise `stream` and report (then clear) the MLP's device error word. */
ann_status ann_mlp_sync(ann_mlp *mlp, void *stream);
/* Per-dimension input standardisation, applied on the device to every query
 * (forward, training, prediction) before its BF16 rounding:
 * x' = (x - mean) * inv_std, each operation rounded in FP32. mean and inv_std
 * are host arrays of in_dim finite floats; both NULL restores the identity
 * (mean 0, inv_std 1, the state after ann_mlp_create). */
ann_status ann_mlp_set_input_norm(ann_mlp *mlp, const float *mean, const float *inv_std);
/* Host copies of the standardisation (in_dim floats each). */
ann_status ann_mlp_get_input_norm(const ann_mlp *mlp, float *mean, float *inv_std);
/* Standardisation statistics computed on the device (no counterpart in the
 * paper): x holds n training queries (device, n x in_dim FP32, n >= 1). Per
 * dimension j, mean_j = (1/n) sum_i x_ij and std_j = sqrt((1/n) sum_i
 * (x_ij - mean_j)^2), accumulated in FP64 in a fixed order (deterministic);
 * inv_std_j = 1 / max(std_j, 1e-6 * max(max_j std_j, 1e-30)); both rounded
 * once to FP32 and installed as by ann_mlp_set_input_norm. The call
 * allocates a temporary of about (n/512 + 2) x in_dim doubles and is
 * synchronous on `stream`. ANN_EINVAL for NULL x or n = 0. */
ann_status ann_mlp_fit_input_norm(ann_mlp *mlp, const float *x, uint32_t n, void *stream);
/* The fallback threshold tau of the learned entry (no counterpart in the
 * paper), computed on the device: with q = min(fallback, 1), the value of
 * 0-based rank floor(q * (n - 1)) (q and the product in double) among the n
 * values pmax (device FP32, e.g. ann_mlp_predict's largest softmax
 * probabilities of validation queries) in ascending order, i.e. numpy's
 * quantile with method "lower". *tau (host) receives it; 0 when n = 0 or
 * fallback <= 0 (no query falls back). Values are ordered as FP32 numbers
 * (-0 before +0; NaN, which pmax never holds, after +inf). Synchronous on
 * `stream`. ANN_EINVAL for NULL tau, NULL pmax with n > 0, or a NaN fallback. */
ann_status ann_mlp_confidence_threshold(ann_mlp *mlp, const float *pmax, uint32_t n, double fallback, float *tau,
                                        void *stream);
/* Save the network and its training state to a file: the 8 bytes "ANNMLP02",
 * the four sizes (in_dim, hidden1, hidden2, out_dim) as little-endian uint32,
 * then W1, b1, W2, b2, W3, b3, mean, inv_std as little-endian FP32 in the
 * row-major layout above, then the AdamW step count (uint32) and, per layer
 * 1..3, the first and second moments of W and then of b (FP32, same layouts),
 * so that training resumes where it stopped. ANN_EIO if the file cannot be
 * written. */
ann_status ann_mlp_save(const ann_mlp *mlp, const char *path);
/* Create an MLP on `device` with room for max_batch rows from a file written
 * by ann_mlp_save: version "ANNMLP02" restores the optimizer state too;
 * version "ANNMLP01" (parameters and standardisation only) starts with a
 * fresh one. ANN_EIO if the file cannot be read or is short, ANN_EINVAL if
 * its magic or sizes are not valid. */
ann_status ann_mlp_load(const char *path, int device, uint32_t max_batch, ann_mlp **out);

/* ------------------------------------------------------------------------
 * Continuous-batching server (not in the paper). Requests (batches of any
 * size, each with its own ann_search_params up to the server's max_params)
 * are admitted while others run and share the GPU query by query: one device
 * ring of query slots, a FIFO that the warps of every running search kernel
 * take queries from, per-warp queue and visited state resident in shared
 * memory while a query runs. Admission is by buffer memory: submit returns
 * ANN_EBUSY when the ring or the request records are full (poll, then retry).
 * Results are deterministic per request (the RNG stream is qid_base + the
 * query's index within its request), so a request's answer is the same alone
 * or in any mix. One host thread drives a server.
 * ------------------------------------------------------------------------ */
typedef struct ann_server ann_server;

typedef struct {
    uint32_t capacity;            /* query slots resident on the device */
    uint32_t max_requests;        /* requests in flight */
    ann_search_params max_params; /* largest k, itopk, search_width, ghost_itopk of any request, and the
                                     features allowed (DGS if dgs_discard > 0, rerank, entry != random) */
    uint32_t seeds_per_query;     /* learned entry (max_params.entry == ANN_ENTRY_GIVEN_GHOST): P, 1..8 */
    float tau;                    /* learned entry: fallback threshold on the top softmax probability */
    uint32_t queries_per_warp;    /* queries a warp serves before its kernel may end; 0 = 4 */
    uint32_t streams;             /* compute streams; 0 = 4 */
} ann_server_config;

typedef struct {
    uint64_t req_id;
    uint32_t status;      /* ANN_OK */
    uint32_t nq;
    double latency_s;     /* submit -> completion observed by ann_server_poll */
} ann_completion;

/* mlp: the learned entry (required when max_params.entry is ANN_ENTRY_GIVEN_GHOST, else NULL);
 * requests with entry ANN_ENTRY_GIVEN_GHOST get their ghost seeds from it. */
ann_status ann_server_create(ann_index *index, const ann_server_config *config, ann_mlp *mlp, ann_server **out);
/* Admit one request: queries (host, nq x dim FP32) are copied in before the
 * call returns; ids / dists (host, nq x k) are filled by ann_server_poll when
 * the request completes and must stay valid until then. */
ann_status ann_server_submit(ann_server *server, uint64_t req_id, const float *queries, uint32_t nq,
                             const ann_search_params *params, uint32_t *ids, float *dists);
/* Collect up to `max` completed requests (their results are in place). */
ann_status ann_server_poll(ann_server *server, ann_completion *out, uint32_t max, uint32_t *n_out);
/* Requests submitted and not yet collected by ann_server_poll's bookkeeping. */
uint32_t ann_server_in_flight(const ann_server *server);
ann_status ann_server_destroy(ann_server *server);

/* Thread-local message for the last failing call on this thread. */
const char *ann_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ANN_H */
