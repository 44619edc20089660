// ann_search_host_noalloc: the host-buffer search without any device
// allocation. (No counterpart in the paper.)
//
// ann_search_host stages queries and results in a device workspace that the
// index grows with cudaMalloc on first use. Some callers cannot allow that:
// a serving process that reserves all device memory up front and must not
// allocate (or synchronise the device, as cudaMalloc/cudaFree may) on its
// request path, code running under an external memory budget, or a host
// thread with a latency deadline. This entry point instead uses one
// file-scope device array of fixed size for the query copy, the result
// copies, the kernel's work counter and its error word.
//
// Limits and sharing:
//   - the array holds ANN_NOALLOC_SCRATCH_BYTES; a call whose staging needs
//     more (256 + nq * dim * 4 + 2 * nq * k * 4 bytes, each part rounded up
//     to 256) is rejected with ANN_EINVAL before anything runs;
//   - every GPU that loads the library holds one such array until the
//     process exits; all calls on a device share it and it keeps the last
//     call's contents, so each call zeroes the work counter and error word it
//     relies on, and calls that overlap on the GPU (other streams, other host
//     threads) race on it;
//   - the call is synchronous: it returns once the results are in the
//     caller's host buffers;
//   - the first call on a device looks up that device's address of the array
//     (cudaGetSymbolAddress, with that device current) and caches it; that
//     lookup is a set-up step, so make the first call on each device before
//     any stream capture starts there.
#include <mutex>

#include "ann_internal.cuh"

using namespace ann;

namespace {

static __device__ __align__(256) uint8_t g_noalloc_scratch[ANN_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint8_t *g_addr[kMaxDevices] = {};

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of this device's copy of the array (host code may not use
// the array's name as an address).
ann_status scratch_for(int device, uint8_t **out)
{
    if (device < 0 || device >= kMaxDevices) {
        set_error("ann_search_host_noalloc: device %d out of range", device);
        return ANN_EDEVICE;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_addr[device] = static_cast<uint8_t *>(p);
    }
    *out = g_addr[device];
    return ANN_OK;
}

}  // namespace

extern "C" ann_status ann_search_host_noalloc(ann_index *ix, const float *queries, uint32_t nq,
                                              const ann_search_params *p, uint32_t *ids, float *dists,
                                              void *stream)
{
    if (!ix || !p) { set_error("ann_search_host_noalloc: NULL index or params"); return ANN_EINVAL; }
    if (p->entry == ANN_ENTRY_GIVEN_GHOST) {
        set_error("ann_search_host_noalloc: given ghost seeds are not supported; use ann_search");
        return ANN_EINVAL;
    }
    if (nq == 0) return ANN_OK;
    if (!queries || !ids || !dists) { set_error("ann_search_host_noalloc: NULL buffers"); return ANN_EINVAL; }
    const size_t qb = (size_t)nq * ix->dim * 4, ob = (size_t)nq * p->k * 4;
    const size_t need = 256 + up256(qb) + 2 * up256(ob);
    if (need > ANN_NOALLOC_SCRATCH_BYTES) {
        set_error("ann_search_host_noalloc: %u queries of dim %u with k %u need %zu bytes of staging; the fixed "
                  "scratch holds %u (split the batch)", nq, ix->dim, p->k, need, (unsigned)ANN_NOALLOC_SCRATCH_BYTES);
        return ANN_EINVAL;
    }
    // the array's address is looked up (and cached) only with the index's
    // device current: return before that if the switch fails
    int prev = -1;
    ann_status s = enter_device(ix->device, &prev, "ann_search_host_noalloc");
    if (s != ANN_OK) return s;
    uint8_t *base = nullptr;
    s = scratch_for(ix->device, &base);
    if (s == ANN_OK) {
        cudaStream_t st = (cudaStream_t)stream;
        uint32_t *counter = reinterpret_cast<uint32_t *>(base);
        int *err = reinterpret_cast<int *>(base + 64);
        float *dq = reinterpret_cast<float *>(base + 256);
        uint32_t *di = reinterpret_cast<uint32_t *>(base + 256 + up256(qb));
        float *dd = reinterpret_cast<float *>(base + 256 + up256(qb) + up256(ob));
        cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dq, queries, qb, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) s = cuda_fail(e, "ann_search_host_noalloc upload");
        if (s == ANN_OK) s = search_launch_ex(ix, dq, nq, p, nullptr, 0, di, dd, nullptr, st, counter, err);
        int herr = 0;
        if (s == ANN_OK) {
            e = cudaMemcpyAsync(ids, di, ob, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dists, dd, ob, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) s = cuda_fail(e, "ann_search_host_noalloc download");
        }
        if (s == ANN_OK && herr) {
            set_error("ann_search_host_noalloc: a bounded device wait ran out (code %d)", herr);
            s = ANN_ETIMEOUT;
        }
    }
    leave_device(ix->device, prev);
    return s;
}
