// noalloc.cu -- the dimension-1 filtration (edges inside a threshold, sorted in
// coboundary order) for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another runtime's
// device memory pool, where every allocation has to go through that owner, and
// latency-critical loops, where cudaMalloc and cudaFree would implicitly
// synchronise the device. This entry point takes the caller's input and output
// buffers and keeps its scratch (counters, binomial table, the radix sort's
// control block, look-back entries and ping-pong buffers) in one static device
// array of fixed size, declared below. Every GPU that loads the library holds
// that array until the process exits.
#include <cmath>
#include <string>

#include "../../include/rpp.h"
#include "internal.h"

namespace rpp {

namespace {

constexpr int64_t NA_MAX_EDGES = 1 << 18;  // largest output the scratch can sort
constexpr int64_t NA_MAX_N = 724;          // C(724, 2) = 261,726 <= NA_MAX_EDGES
constexpr size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t OFF_STATE = 0;
constexpr size_t OFF_BINOM = up256(sizeof(DevState));
constexpr size_t OFF_SORT = up256(OFF_BINOM + 3 * (NA_MAX_N + 1) * sizeof(uint64_t));
constexpr size_t OFF_TMP_HI = up256(OFF_SORT + radix_scratch_bound(NA_MAX_EDGES));
constexpr size_t OFF_TMP_LO = up256(OFF_TMP_HI + NA_MAX_EDGES * sizeof(uint32_t));
constexpr size_t SCRATCH_BYTES = up256(OFF_TMP_LO + NA_MAX_EDGES * sizeof(uint64_t));

// The scratch of rpp_filtration_edges_noalloc (about 3.8 MB per GPU). In host
// code this name is only a stand-in: its device address comes from
// cudaGetSymbolAddress, looked up on every call with the caller's device
// current (a cached address would go stale if the device were reset and the
// module placed elsewhere).
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

// Zero the counters, set the threshold, and write C(v, k) for k = 0, 1, 2.
__global__ void k_noalloc_init(DevState *st, float t, uint64_t *binom, int64_t n) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        DevState z = {};
        z.t = t;
        *st = z;
    }
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n;
         v += (int64_t)gridDim.x * blockDim.x) {
        binom[v] = 1;
        binom[(n + 1) + v] = (uint64_t)v;
        binom[2 * (n + 1) + v] = (uint64_t)v * (uint64_t)(v > 0 ? v - 1 : 0) / 2;
    }
}

// Sort keys held ~bits(diameter); turn them back into diameters.
__global__ void k_noalloc_finish(uint32_t *key_hi, uint64_t cap, const unsigned long long *count) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cap && i < *count) key_hi[i] = ~key_hi[i];
}

int bits_for(uint64_t x) {
    int b = 0;
    while (b < 64 && (x >> b)) ++b;
    return b;
}

}  // namespace

}  // namespace rpp

using namespace rpp;

extern "C" rpp_status rpp_filtration_edges_noalloc(const float *D, int64_t n, float threshold,
                                                   float *diam_out, uint64_t *cidx_out,
                                                   int64_t capacity, int64_t *count_out,
                                                   void *stream) {
    if (!D || !diam_out || !cidx_out || !count_out || n < 1 || std::isnan(threshold) ||
        threshold < 0.0f) {
        set_last_error("rpp_filtration_edges_noalloc: invalid arguments");
        return RPP_E_INVALID;
    }
    if (n > NA_MAX_N) {
        set_last_error("rpp_filtration_edges_noalloc: n exceeds the static scratch bound of 724 "
                       "points (262,144 edges)");
        return RPP_E_INVALID;
    }
    const uint64_t m = (uint64_t)n * (uint64_t)(n - 1) / 2;
    if (capacity < (int64_t)m) {
        set_last_error("rpp_filtration_edges_noalloc: output capacity below C(n, 2)");
        return RPP_E_INVALID;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        set_last_error("rpp_filtration_edges_noalloc: no current CUDA device");
        return RPP_E_CUDA;
    }
    // D and both outputs must be memory of the current device (the scratch
    // address below is the current device's), and so must the stream
    const void *bufs[3] = {D, diam_out, cidx_out};
    const char *names[3] = {"D", "diam_out", "cidx_out"};
    for (int i = 0; i < 3; ++i) {
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, bufs[i]) != cudaSuccess ||
            (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) ||
            (attr.type == cudaMemoryTypeDevice && attr.device != dev)) {
            cudaGetLastError();
            set_last_error(std::string("rpp_filtration_edges_noalloc: ") + names[i] +
                           " must be device memory of the current device");
            return RPP_E_INVALID;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (s) {
        int sdev = -1;
        if (cudaStreamGetDevice(s, &sdev) != cudaSuccess || sdev != dev) {
            cudaGetLastError();
            set_last_error("rpp_filtration_edges_noalloc: the stream belongs to another device");
            return RPP_E_INVALID;
        }
    }
    unsigned char *base = nullptr;
    {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            set_last_error(std::string("rpp_filtration_edges_noalloc: cudaGetSymbolAddress: ") +
                           cudaGetErrorString(e));
            return RPP_E_CUDA;
        }
        base = (unsigned char *)p;
    }
    DevState *st = (DevState *)(base + OFF_STATE);
    uint64_t *binom = (uint64_t *)(base + OFF_BINOM);
    void *sort_scratch = base + OFF_SORT;
    uint32_t *tmp_hi = (uint32_t *)(base + OFF_TMP_HI);
    uint64_t *tmp_lo = (uint64_t *)(base + OFF_TMP_LO);
    uint32_t *key_hi = (uint32_t *)diam_out;  // sorted as ~bits(diameter), then converted

    // build, sort and conversion are queued with the edge count left on the
    // device; one wait at the end reads the count and the sort's wait flag
    ++g_launches;
    k_noalloc_init<<<4, 256, 0, s>>>(st, threshold, binom, n);
    launch_build_columns(D, n, n, 1, binom, m, nullptr, st, key_hi, cidx_out, s);
    radix_sort(key_hi, cidx_out, nullptr, tmp_hi, tmp_lo, nullptr, sort_scratch, m, &st->ncols,
               bits_for(m > 0 ? m - 1 : 0), &st->err, s);
    if (m > 0) {
        ++g_launches;
        k_noalloc_finish<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(key_hi, m, &st->ncols);
    }
    DevState hs;
    cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string("rpp_filtration_edges_noalloc: ") + cudaGetErrorString(e));
        return RPP_E_CUDA;
    }
    if (hs.err & ERR_INTERNAL) {
        set_last_error("rpp_filtration_edges_noalloc: a bounded device wait ran out (sort)");
        return RPP_E_CUDA;
    }
    const unsigned long long count = hs.ncols;
    *count_out = (int64_t)count;
    return RPP_OK;
}
