// l2_probe.cu -- a read-bandwidth probe of the L2 cache.
//
// The apparent-pair pass (Alg. 3) reads distance rows that stay in L2 at the
// sizes it serves (a 2000-point matrix is 16 MB against the GB300's 129 MB
// L2), so its DRAM traffic is a small part of what it loads and its HBM
// roofline fraction is low by construction. The ceiling that bounds those
// loads is the L2's read bandwidth to the SMs, which this kernel measures on
// the running GPU: the grid reads a caller's buffer `reps` times with loads
// that are cached in L2 only (ld.global.cg, so L1 cannot serve a repeat), and
// the caller times the launch. With a buffer that fits in L2 and one launch
// beforehand to bring it there, bytes * reps / time is the L2 read bandwidth.
//
// Every word read is summed (mod 2^32) into one counter, so a test can check
// that every load was made, reps times over the whole buffer.
#include <string>

#include "../../include/rpp.h"
#include "internal.h"

namespace rpp {

namespace {

constexpr int PROBE_THREADS = 512;
constexpr int32_t PROBE_MAX_REPS = 1 << 20;
constexpr int32_t PROBE_MAX_BLOCKS = 65535;

// One 16-byte load cached in L2 only. Written as volatile PTX so the compiler
// keeps every load of every repetition (identical loads of a pure intrinsic
// could be merged across the repetition loop).
__device__ __forceinline__ uint4 load_l2_only(const uint4 *p) {
    uint4 v;
    asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ unsigned int word_sum(uint4 v) { return (v.x + v.y) + (v.z + v.w); }

// Thread t of T reads the 16-byte elements t, t + T, t + 2T, ... of the
// buffer, four independent loads in flight per step, in every repetition.
__global__ void __launch_bounds__(PROBE_THREADS)
k_l2_read(const uint4 *__restrict__ buf, uint64_t n16, int32_t reps, unsigned int *sink) {
    const uint64_t T = (uint64_t)gridDim.x * PROBE_THREADS;
    const uint64_t t0 = (uint64_t)blockIdx.x * PROBE_THREADS + threadIdx.x;
    unsigned int acc = 0;
    for (int32_t r = 0; r < reps; ++r) {
        uint64_t i = t0;
        for (; i + 3 * T < n16; i += 4 * T) {
            const uint4 a = load_l2_only(buf + i);
            const uint4 b = load_l2_only(buf + i + T);
            const uint4 c = load_l2_only(buf + i + 2 * T);
            const uint4 d = load_l2_only(buf + i + 3 * T);
            acc += (word_sum(a) + word_sum(b)) + (word_sum(c) + word_sum(d));
        }
        for (; i < n16; i += T) acc += word_sum(load_l2_only(buf + i));
    }
    // one atomic per block: warp sums, then the first warp sums the warps
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ unsigned int part[PROBE_THREADS / 32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned int v = threadIdx.x < PROBE_THREADS / 32 ? part[threadIdx.x] : 0u;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) atomicAdd(sink, v);
    }
}

rpp_status probe_fail(rpp_status st, const std::string &why) {
    set_last_error("rpp_l2_read_probe: " + why);
    return st;
}

}  // namespace

}  // namespace rpp

using namespace rpp;

extern "C" rpp_status rpp_l2_read_probe(const void *buf, size_t bytes, int32_t reps,
                                        int32_t blocks, uint32_t *sink, void *stream) {
    if (!buf || !sink) return probe_fail(RPP_E_INVALID, "buf and sink must not be NULL");
    if (((uintptr_t)buf & 15) != 0 || bytes == 0 || (bytes & 15) != 0)
        return probe_fail(RPP_E_INVALID,
                          "buf must be 16-byte aligned and bytes a positive multiple of 16");
    if (((uintptr_t)sink & 3) != 0) return probe_fail(RPP_E_INVALID, "sink must be 4-byte aligned");
    if (reps < 1 || reps > PROBE_MAX_REPS)
        return probe_fail(RPP_E_INVALID, "reps must be in [1, 2^20]");
    if (blocks < 1 || blocks > PROBE_MAX_BLOCKS)
        return probe_fail(RPP_E_INVALID, "blocks must be in [1, 65535]");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return probe_fail(RPP_E_CUDA, "no current CUDA device");
    }
    const void *ptrs[2] = {buf, sink};
    const char *names[2] = {"buf", "sink"};
    for (int i = 0; i < 2; ++i) {
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, ptrs[i]) != cudaSuccess ||
            attr.type != cudaMemoryTypeDevice || attr.device != dev) {
            cudaGetLastError();
            return probe_fail(RPP_E_INVALID,
                              std::string(names[i]) + " must be device memory of the current device");
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (s) {
        int sdev = -1;
        if (cudaStreamGetDevice(s, &sdev) != cudaSuccess || sdev != dev) {
            cudaGetLastError();
            return probe_fail(RPP_E_INVALID, "the stream belongs to another device");
        }
    }
    ++g_launches;
    k_l2_read<<<(unsigned)blocks, PROBE_THREADS, 0, s>>>((const uint4 *)buf, (uint64_t)(bytes / 16),
                                                        reps, (unsigned int *)sink);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return probe_fail(RPP_E_CUDA, cudaGetErrorString(e));
    return RPP_OK;
}
