// Continuous-batching server (not in the paper): requests of any size, each
// with its own k / itopk / entry, are admitted while others run and share the
// GPU query by query.
//
// Device state: a ring of `capacity` query slots (query vector, learned-entry
// seeds, kmax results), a ring of request records, and two monotonic query
// counters, head (taken) and tail (published). Host state: the requests in
// flight, in slot order.
//
// submit(): admission checks ring space and request records (ANN_EBUSY when
// either is short: admission by buffer memory). On one high-priority ingest
// stream, in order: the request record, the query vectors, the slot->request
// map, the learned-entry seeds (if any), then the new tail. The serve kernel
// launch for the request waits on an event after the tail update and runs on
// one of several compute streams, so kernels of successive requests overlap
// and every running kernel takes queries from the same FIFO: a request that
// arrives while others are on the GPU is picked up as soon as a warp frees.
// Each launch has capacity (blocks x warps x queries per warp) for every
// query in flight, its own request's included (so a burst of small requests
// fills the GPU instead of one block per request), and a kernel only leaves
// early when the ring is empty, so every published query is served.
//
// poll(): a request is done when its host-mapped flag is set (by the warp
// that finished its last query, after a system-scope fence); its results are
// copied out and its ring space is reclaimed in slot order. Latency is
// submit -> poll-observed completion on the host's steady clock.
#include <chrono>
#include <deque>
#include <vector>

#include "ann_internal.cuh"

using namespace ann;

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

__global__ void fill_slot_req_kernel(uint32_t *slot_req, uint64_t slot0, uint32_t n, uint32_t cap, uint32_t r)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        slot_req[(slot0 + i) % cap] = r;
}

struct Pending {
    uint64_t req_id;
    uint32_t ri;
    uint64_t start;    // first query counter
    uint32_t nq, k;
    uint32_t *ids_out;
    float *dists_out;
    double t_submit;
    bool done;
};

}  // namespace

struct ann_server {
    ann_index *ix = nullptr;
    ann_mlp *mlp = nullptr;
    uint32_t P = 0;
    float tau = 0.0f;
    uint32_t cap = 0, nreq = 0, kmax = 0, per_warp = 4;
    ann_search_params maxp{};
    void *plan = nullptr;
    float *d_queries = nullptr;
    uint32_t *d_seeds = nullptr, *d_ids = nullptr, *d_slot_req = nullptr;
    float *d_dists = nullptr;
    ServeReq *d_reqs = nullptr;
    unsigned long long *d_ctr = nullptr;       // [0] head, [1] tail
    uint32_t *h_flags = nullptr, *d_flags = nullptr;
    ServeReq *h_reqs = nullptr;
    unsigned long long *h_tails = nullptr;
    cudaStream_t ingest = nullptr;
    std::vector<cudaStream_t> compute;
    std::vector<cudaEvent_t> ev;
    uint32_t next_stream = 0;
    uint64_t tail = 0, seq = 0;
    std::deque<Pending> inflight;
    std::deque<ann_completion> ready;
};

namespace {

void server_release(ann_server *s)
{
    if (s->ingest) cudaStreamSynchronize(s->ingest);
    for (cudaStream_t c : s->compute) cudaStreamSynchronize(c);
    void *dev[] = {s->d_queries, s->d_seeds, s->d_ids, s->d_slot_req, s->d_dists, s->d_reqs, s->d_ctr};
    for (void *p : dev) if (p) cudaFree(p);
    if (s->h_flags) cudaFreeHost(s->h_flags);
    if (s->h_reqs) cudaFreeHost(s->h_reqs);
    if (s->h_tails) cudaFreeHost(s->h_tails);
    for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
    for (cudaStream_t c : s->compute) cudaStreamDestroy(c);
    if (s->ingest) cudaStreamDestroy(s->ingest);
    if (s->plan) serve_plan_free(s->plan);
}

// Copy `n` consecutive ring rows starting at counter `start` (wrapping) of
// width `w` elements (pitch kmax) into dst rows of width w.
template <typename T>
cudaError_t copy_out(T *dst, const T *ring, uint64_t start, uint32_t n, uint32_t w, uint32_t pitch, uint32_t cap)
{
    const uint32_t s0 = (uint32_t)(start % cap);
    const uint32_t first = std::min<uint32_t>(n, cap - s0);
    cudaError_t e = cudaMemcpy2D(dst, w * sizeof(T), ring + (size_t)s0 * pitch, pitch * sizeof(T), w * sizeof(T), first,
                                 cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && first < n)
        e = cudaMemcpy2D(dst + (size_t)first * w, w * sizeof(T), ring, pitch * sizeof(T), w * sizeof(T), n - first,
                         cudaMemcpyDeviceToHost);
    return e;
}

}  // namespace

extern "C" {

ann_status ann_server_create(ann_index *ix, const ann_server_config *cfg, ann_mlp *mlp, ann_server **out)
{
    if (!ix || !cfg || !out) { set_error("ann_server_create: NULL argument"); return ANN_EINVAL; }
    *out = nullptr;
    if (cfg->capacity == 0 || cfg->max_requests == 0) {
        set_error("ann_server_create: capacity and max_requests must be positive");
        return ANN_EINVAL;
    }
    const ann_search_params &mp = cfg->max_params;
    if (mp.entry > ANN_ENTRY_GIVEN_GHOST) {
        set_error("ann_server_create: entry %u is not served (given base seeds need ann_search)", mp.entry);
        return ANN_EINVAL;
    }
    if (mp.entry == ANN_ENTRY_GIVEN_GHOST && (!mlp || cfg->seeds_per_query == 0 || cfg->seeds_per_query > 8)) {
        set_error("ann_server_create: the learned entry needs an MLP and 1..8 seeds per query");
        return ANN_EINVAL;
    }
    int prev = -1;
    {
        const ann_status ds = enter_device(ix->device, &prev, "ann_server_create");
        if (ds != ANN_OK) return ds;
    }
    ann_server *s = new ann_server();
    s->ix = ix;
    s->mlp = mlp;
    s->P = mp.entry == ANN_ENTRY_GIVEN_GHOST ? cfg->seeds_per_query : 0;
    s->tau = cfg->tau;
    s->cap = cfg->capacity;
    s->nreq = cfg->max_requests;
    s->kmax = mp.k;
    s->per_warp = cfg->queries_per_warp ? cfg->queries_per_warp : 4;
    s->maxp = mp;
    const uint32_t ns = cfg->streams ? cfg->streams : 4;
    ann_status st = serve_plan(ix, &mp, s->P ? s->P : 1, ns, &s->plan);
    cudaError_t e = cudaSuccess;
    auto al = [&](void **p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
    if (st == ANN_OK) {
        al((void **)&s->d_queries, (size_t)s->cap * ix->dim * 4);
        if (s->P) al((void **)&s->d_seeds, (size_t)s->cap * s->P * 4);
        al((void **)&s->d_ids, (size_t)s->cap * s->kmax * 4);
        al((void **)&s->d_dists, (size_t)s->cap * s->kmax * 4);
        al((void **)&s->d_slot_req, (size_t)s->cap * 4);
        al((void **)&s->d_reqs, (size_t)s->nreq * sizeof(ServeReq));
        al((void **)&s->d_ctr, 64);
        if (e == cudaSuccess) e = cudaMemset(s->d_ctr, 0, 64);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->h_flags, (size_t)s->nreq * 4, cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&s->d_flags, s->h_flags, 0);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->h_reqs, (size_t)s->nreq * sizeof(ServeReq), 0);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->h_tails, (size_t)s->nreq * 8, 0);
        int lo = 0, hi = 0;
        if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->ingest, cudaStreamNonBlocking, hi);
        for (uint32_t i = 0; i < ns && e == cudaSuccess; ++i) {
            cudaStream_t c;
            e = cudaStreamCreateWithPriority(&c, cudaStreamNonBlocking, lo);
            if (e == cudaSuccess) s->compute.push_back(c);
        }
        for (uint32_t i = 0; i < s->nreq && e == cudaSuccess; ++i) {
            cudaEvent_t ev;
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) s->ev.push_back(ev);
        }
        if (e != cudaSuccess) st = cuda_fail(e, "ann_server_create");
        else memset(s->h_flags, 0, (size_t)s->nreq * 4);
    }
    leave_device(ix->device, prev);
    if (st != ANN_OK) {
        server_release(s);
        delete s;
        return st;
    }
    *out = s;
    return ANN_OK;
}

ann_status ann_server_submit(ann_server *s, uint64_t req_id, const float *queries, uint32_t nq,
                             const ann_search_params *p, uint32_t *ids, float *dists)
{
    if (!s || !p || (nq && (!queries || !ids || !dists))) { set_error("ann_server_submit: NULL argument"); return ANN_EINVAL; }
    if (nq == 0) { set_error("ann_server_submit: empty request"); return ANN_EINVAL; }
    const ann_search_params &mp = s->maxp;
    if (p->k > mp.k || p->itopk > mp.itopk || p->search_width > mp.search_width ||
        (p->ghost_search_width ? p->ghost_search_width : 1) > (mp.ghost_search_width ? mp.ghost_search_width : 1) ||
        ((p->dgs_discard > 0.0f || p->dgs_min_match > 0.0f) &&
         !(mp.dgs_discard > 0.0f || mp.dgs_min_match > 0.0f)) ||
        (p->rerank && !mp.rerank) || p->entry > ANN_ENTRY_GIVEN_GHOST ||
        (p->entry != ANN_ENTRY_RANDOM && mp.entry == ANN_ENTRY_RANDOM) ||
        (p->entry == ANN_ENTRY_GIVEN_GHOST && !s->P) ||
        (p->entry != ANN_ENTRY_RANDOM && (p->ghost_itopk ? p->ghost_itopk : std::min(p->itopk, 64u)) >
                                             (mp.ghost_itopk ? mp.ghost_itopk : std::min(mp.itopk, 64u)))) {
        set_error("ann_server_submit: parameters exceed the server's max_params");
        return ANN_EINVAL;
    }
    if (nq > s->cap) { set_error("ann_server_submit: %u queries exceed the ring capacity %u", nq, s->cap); return ANN_EINVAL; }
    QParams q;
    ann_status st = derive_qparams(s->ix, p, p->entry == ANN_ENTRY_GIVEN_GHOST ? s->P : 0, &q);
    if (st != ANN_OK) return st;
    const uint64_t oldest = s->inflight.empty() ? s->tail : s->inflight.front().start;
    if (s->inflight.size() >= s->nreq || s->tail + nq - oldest > s->cap) {
        set_error("ann_server_submit: no room (ring or request records full)");
        return ANN_EBUSY;
    }
    int prev = -1;
    {
        const ann_status ds = enter_device(s->ix->device, &prev, "ann_server_submit");
        if (ds != ANN_OK) return ds;
    }
    const uint32_t ri = (uint32_t)(s->seq % s->nreq);
    const uint32_t dim = s->ix->dim;
    const uint32_t slot0 = (uint32_t)(s->tail % s->cap);
    const uint32_t first = std::min<uint32_t>(nq, s->cap - slot0);
    reinterpret_cast<volatile uint32_t *>(s->h_flags)[ri] = 0;
    ServeReq &hr = s->h_reqs[ri];
    hr.qp = q;
    hr.nq = nq;
    hr.slot0 = slot0;
    hr.done = 0;
    hr.flag = ri;
    cudaStream_t in = s->ingest;
    cudaError_t e = cudaMemcpyAsync(s->d_reqs + ri, &hr, sizeof(ServeReq), cudaMemcpyHostToDevice, in);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_queries + (size_t)slot0 * dim, queries, (size_t)first * dim * 4, cudaMemcpyHostToDevice, in);
    if (e == cudaSuccess && first < nq)
        e = cudaMemcpyAsync(s->d_queries, queries + (size_t)first * dim, (size_t)(nq - first) * dim * 4,
                            cudaMemcpyHostToDevice, in);
    if (e == cudaSuccess) {
        fill_slot_req_kernel<<<(nq + 255) / 256, 256, 0, in>>>(s->d_slot_req, s->tail, nq, s->cap, ri);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && p->entry == ANN_ENTRY_GIVEN_GHOST) {
        st = ann_mlp_predict(s->mlp, s->d_queries + (size_t)slot0 * dim, first, s->P, s->tau,
                             s->d_seeds + (size_t)slot0 * s->P, nullptr, in);
        if (st == ANN_OK && first < nq)
            st = ann_mlp_predict(s->mlp, s->d_queries, nq - first, s->P, s->tau, s->d_seeds, nullptr, in);
    }
    if (st == ANN_OK && e == cudaSuccess) {
        s->h_tails[ri] = s->tail + nq;
        e = cudaMemcpyAsync(s->d_ctr + 1, &s->h_tails[ri], 8, cudaMemcpyHostToDevice, in);
        if (e == cudaSuccess) e = cudaEventRecord(s->ev[ri], in);
    }
    if (st == ANN_OK && e == cudaSuccess) {
        const uint32_t si = (uint32_t)(s->next_stream++ % s->compute.size());
        cudaStream_t c = s->compute[si];
        e = cudaStreamWaitEvent(c, s->ev[ri], 0);
        if (e == cudaSuccess) {
            ServeRing r{};
            r.queries = s->d_queries;
            r.seeds = s->d_seeds;
            r.P = s->P;
            r.ids = s->d_ids;
            r.dists = s->d_dists;
            r.slot_req = s->d_slot_req;
            r.reqs = s->d_reqs;
            r.head = s->d_ctr;
            r.tail = s->d_ctr + 1;
            r.flags = s->d_flags;
            r.cap = s->cap;
            r.kmax = s->kmax;
            r.per_warp = s->per_warp;
            // sized for every query not yet known complete (this request and
            // the ones before it), not just this request's: the kernel's
            // warps pop any query from the ring, and warps that find it empty
            // leave at once, so a burst of small requests still fills the GPU
            const uint64_t pending = s->tail + nq - oldest;
            st = serve_launch(s->plan, r, (uint32_t)std::min<uint64_t>(pending, s->cap), c, si);
        }
    }
    if (st == ANN_OK && e != cudaSuccess) st = cuda_fail(e, "ann_server_submit");
    if (st == ANN_OK) {
        s->inflight.push_back(Pending{req_id, ri, s->tail, nq, p->k, ids, dists, now_s(), false});
        s->tail += nq;
        s->seq++;
    }
    leave_device(s->ix->device, prev);
    return st;
}

ann_status ann_server_poll(ann_server *s, ann_completion *out, uint32_t max, uint32_t *n_out)
{
    if (!s || (max && !out) || !n_out) { set_error("ann_server_poll: NULL argument"); return ANN_EINVAL; }
    int prev = -1;
    {
        const ann_status ds = enter_device(s->ix->device, &prev, "ann_server_poll");
        if (ds != ANN_OK) return ds;
    }
    ann_status st = ANN_OK;
    for (Pending &pd : s->inflight) {
        if (pd.done || !reinterpret_cast<volatile uint32_t *>(s->h_flags)[pd.ri]) continue;
        cudaError_t e = copy_out(pd.ids_out, s->d_ids, pd.start, pd.nq, pd.k, s->kmax, s->cap);
        if (e == cudaSuccess) e = copy_out(pd.dists_out, s->d_dists, pd.start, pd.nq, pd.k, s->kmax, s->cap);
        if (e != cudaSuccess) { st = cuda_fail(e, "ann_server_poll"); break; }
        pd.done = true;
        s->ready.push_back(ann_completion{pd.req_id, 0, pd.nq, now_s() - pd.t_submit});
    }
    while (!s->inflight.empty() && s->inflight.front().done) s->inflight.pop_front();
    uint32_t n = 0;
    while (n < max && !s->ready.empty()) {
        out[n++] = s->ready.front();
        s->ready.pop_front();
    }
    *n_out = n;
    leave_device(s->ix->device, prev);
    return st;
}

uint32_t ann_server_in_flight(const ann_server *s) { return s ? (uint32_t)s->inflight.size() : 0; }

ann_status ann_server_destroy(ann_server *s)
{
    if (!s) return ANN_OK;
    int prev = -1;
    const bool switched = enter_device(s->ix->device, &prev, "ann_server_destroy") == ANN_OK;   // frees best-effort
    server_release(s);
    if (switched) leave_device(s->ix->device, prev);
    delete s;
    return ANN_OK;
}

}  // extern "C"
