// radix_sort.cu -- least-significant-digit radix sort of (hi, lo) keys with an
// optional 64-bit payload (the "GPU-sort" of Alg. 7, whose implementation the
// paper leaves open).
//
// Keys are 96-bit: a 64-bit low word (the combinatorial index) and a 32-bit
// high word (the inverted diameter bits). 8-bit digits are processed from the
// least significant upwards, so each pass must be stable. One histogram kernel
// first counts every digit position at once; passes whose digit is the same
// for every key are skipped. Each remaining pass is reduce-then-scan:
//   count   : per 2048-key tile, a 256-bin histogram of the pass's digit,
//             stored digit-major (all tiles of digit 0, then digit 1, ...);
//   scan    : one block per digit: the digit's start among all keys (from the
//             up-front histogram) plus an exclusive scan over the tiles;
//   scatter : each tile ranks its keys stably (warp match + per-warp counts in
//             tile order) and writes them to their final positions.
#include <cuda_runtime.h>

#include <vector>

#include "device_common.cuh"
#include "internal.h"

namespace rpp {

namespace {

constexpr int RADIX = 256;
constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 8;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;
constexpr int MAX_DIGITS = 12;  // 8 low-word digits + 4 high-word digits

__device__ __forceinline__ unsigned digit_of(const uint32_t *hi, const uint64_t *lo, uint64_t i,
                                             int sel) {
    if (sel < 8) return (unsigned)((lo[i] >> (8 * sel)) & 0xffu);
    return (hi[i] >> (8 * (sel - 8))) & 0xffu;
}

__global__ void __launch_bounds__(SORT_THREADS) k_hist_all(const uint32_t *__restrict__ hi,
                                                           const uint64_t *__restrict__ lo,
                                                           uint64_t n, int nlo, int nhi,
                                                           uint32_t *__restrict__ hist) {
    __shared__ uint32_t sh[MAX_DIGITS * RADIX];
    for (int i = threadIdx.x; i < MAX_DIGITS * RADIX; i += SORT_THREADS) sh[i] = 0;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * SORT_THREADS;
    for (uint64_t i = (uint64_t)blockIdx.x * SORT_THREADS + threadIdx.x; i < n; i += stride) {
        const uint64_t l = lo[i];
        for (int d = 0; d < nlo; ++d) atomicAdd(&sh[d * RADIX + ((l >> (8 * d)) & 0xff)], 1u);
        if (nhi) {
            const uint32_t h = hi[i];
            for (int d = 0; d < nhi; ++d)
                atomicAdd(&sh[(8 + d) * RADIX + ((h >> (8 * d)) & 0xff)], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < MAX_DIGITS * RADIX; i += SORT_THREADS)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

__global__ void __launch_bounds__(SORT_THREADS) k_count(const uint32_t *__restrict__ hi,
                                                        const uint64_t *__restrict__ lo, uint64_t n,
                                                        int sel, uint32_t *__restrict__ counts) {
    __shared__ uint32_t sh[RADIX];
    sh[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * SORT_TILE;
#pragma unroll
    for (int j = 0; j < SORT_ITEMS; ++j) {
        const uint64_t i = base + (uint64_t)j * SORT_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&sh[digit_of(hi, lo, i, sel)], 1u);
    }
    __syncthreads();
    counts[(uint64_t)threadIdx.x * gridDim.x + blockIdx.x] = sh[threadIdx.x];  // digit-major
}

// Block d owns digit d: offsets of (tile, d) = keys with a smaller digit (an
// exclusive scan of the digit totals, redone by every block) + keys with
// digit d in earlier tiles (an exclusive scan over this digit's tile counts).
constexpr int SCAN_THREADS = 256;

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_digit(uint32_t *__restrict__ counts,
                                                             uint64_t ntiles,
                                                             const uint32_t *__restrict__ digit_total) {
    __shared__ uint32_t warp_sums[SCAN_THREADS / 32];
    __shared__ uint32_t carry;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int d = blockIdx.x;
    // 1. start of digit d: sum of the totals of digits below d
    uint32_t x = tid < d ? digit_total[tid] : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL_MASK, x, o);
    if (lane == 0) warp_sums[w] = x;
    __syncthreads();
    if (tid == 0) {
        uint32_t b = 0;
        for (int i = 0; i < SCAN_THREADS / 32; ++i) b += warp_sums[i];
        carry = b;
    }
    __syncthreads();
    // 2. running exclusive scan over the tiles, SCAN_THREADS tiles per round
    uint32_t *row = counts + (uint64_t)d * ntiles;
    for (uint64_t t0 = 0; t0 < ntiles; t0 += SCAN_THREADS) {
        const uint64_t t = t0 + tid;
        const uint32_t c = t < ntiles ? row[t] : 0u;
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += y;
        }
        __syncthreads();  // carry and warp_sums of the previous round are read
        if (lane == 31) warp_sums[w] = incl;
        __syncthreads();
        uint32_t before = carry;
        for (int i = 0; i < w; ++i) before += warp_sums[i];
        if (t < ntiles) row[t] = before + incl - c;
        __syncthreads();
        if (tid == SCAN_THREADS - 1) carry = before + incl;
    }
}

__global__ void __launch_bounds__(SORT_THREADS) k_scatter(
    const uint32_t *__restrict__ hi_in, const uint64_t *__restrict__ lo_in,
    const uint64_t *__restrict__ val_in, uint32_t *__restrict__ hi_out,
    uint64_t *__restrict__ lo_out, uint64_t *__restrict__ val_out, uint64_t n, int sel,
    const uint32_t *__restrict__ offsets) {
    constexpr int WARPS = SORT_THREADS / 32;
    __shared__ uint32_t s_run[RADIX];
    __shared__ uint32_t s_warp[WARPS][RADIX];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    s_run[tid] = offsets[(uint64_t)tid * gridDim.x + blockIdx.x];
    const uint64_t base = (uint64_t)blockIdx.x * SORT_TILE;
    for (int j = 0; j < SORT_ITEMS; ++j) {
        const uint64_t i = base + (uint64_t)j * SORT_THREADS + tid;
        const bool valid = i < n;
        const unsigned d = valid ? digit_of(hi_in, lo_in, i, sel) : RADIX;
#pragma unroll
        for (int k = 0; k < WARPS; ++k) s_warp[k][tid] = 0;
        __syncthreads();
        const unsigned peers = __match_any_sync(FULL_MASK, d);
        const unsigned rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) s_warp[w][d] = __popc(peers);
        __syncthreads();
        {  // thread tid owns digit tid: exclusive scan over the warps of this round
            uint32_t run = s_run[tid];
#pragma unroll
            for (int k = 0; k < WARPS; ++k) {
                uint32_t c = s_warp[k][tid];
                s_warp[k][tid] = run;
                run += c;
            }
            s_run[tid] = run;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = s_warp[w][d] + rank;
            lo_out[pos] = lo_in[i];
            if (hi_in) hi_out[pos] = hi_in[i];
            if (val_in) val_out[pos] = val_in[i];
        }
        __syncthreads();
    }
}

}  // namespace

size_t radix_tile_counts_size(uint64_t n) {
    return (size_t)((n + SORT_TILE - 1) / SORT_TILE) * RADIX;
}

void radix_sort(uint32_t *hi, uint64_t *lo, uint64_t *val, uint32_t *tmp_hi, uint64_t *tmp_lo,
                uint64_t *tmp_val, uint32_t *tile_counts, uint32_t *digit_hist, uint64_t n,
                int lo_bits, int hi_bits, cudaStream_t s) {
    if (n <= 1) return;
    // absent key halves or payloads have no scratch either, so the buffer
    // swaps below never pair a null array with a live one
    if (!hi) tmp_hi = nullptr;
    if (!val) tmp_val = nullptr;
    const int nlo = (lo_bits + 7) / 8, nhi = hi ? (hi_bits + 7) / 8 : 0;
    cudaMemsetAsync(digit_hist, 0, MAX_DIGITS * RADIX * sizeof(uint32_t), s);
    uint64_t hb = (n + SORT_THREADS - 1) / SORT_THREADS;
    if (hb > 152 * 4) hb = 152 * 4;
    ++g_launches;
    k_hist_all<<<(unsigned)hb, SORT_THREADS, 0, s>>>(hi, lo, n, nlo, nhi, digit_hist);
    std::vector<uint32_t> h(MAX_DIGITS * RADIX);
    cudaMemcpyAsync(h.data(), digit_hist, h.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    std::vector<int> passes;
    for (int d = 0; d < MAX_DIGITS; ++d) {
        if (d < 8 && d >= nlo) continue;
        if (d >= 8 && d - 8 >= nhi) continue;
        bool constant = false;
        for (int b = 0; b < RADIX; ++b)
            if (h[d * RADIX + b] == n) constant = true;
        if (!constant) passes.push_back(d);
    }
    const uint64_t ntiles = (n + SORT_TILE - 1) / SORT_TILE;
    uint32_t *hi_a = hi, *hi_b = tmp_hi;
    uint64_t *lo_a = lo, *lo_b = tmp_lo, *val_a = val, *val_b = tmp_val;
    for (int sel : passes) {
        ++g_launches;
        k_count<<<(unsigned)ntiles, SORT_THREADS, 0, s>>>(hi_a, lo_a, n, sel, tile_counts);
        ++g_launches;
        k_scan_digit<<<RADIX, SCAN_THREADS, 0, s>>>(tile_counts, ntiles, digit_hist + sel * RADIX);
        ++g_launches;
        k_scatter<<<(unsigned)ntiles, SORT_THREADS, 0, s>>>(
            hi_a, lo_a, val_a, hi_a ? hi_b : nullptr, lo_b, val_a ? val_b : nullptr, n, sel,
            tile_counts);
        std::swap(hi_a, hi_b);
        std::swap(lo_a, lo_b);
        std::swap(val_a, val_b);
    }
    if (passes.size() & 1) {  // result sits in the scratch buffers: copy it back
        cudaMemcpyAsync(lo, lo_a, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
        if (hi) cudaMemcpyAsync(hi, hi_a, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        if (val) cudaMemcpyAsync(val, val_a, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
    }
}

// The same sort driven without any allocation: the histogram comes back into
// the caller's host buffer host_hist (12 * 256 entries), and no payload.
void radix_sort_noalloc(uint32_t *hi, uint64_t *lo, uint32_t *tmp_hi, uint64_t *tmp_lo,
                        uint32_t *tile_counts, uint32_t *digit_hist, uint32_t *host_hist,
                        uint64_t n, int lo_bits, int hi_bits, cudaStream_t s) {
    if (n <= 1) return;
    const int nlo = (lo_bits + 7) / 8, nhi = (hi_bits + 7) / 8;
    cudaMemsetAsync(digit_hist, 0, MAX_DIGITS * RADIX * sizeof(uint32_t), s);
    uint64_t hb = (n + SORT_THREADS - 1) / SORT_THREADS;
    if (hb > 152 * 4) hb = 152 * 4;
    ++g_launches;
    k_hist_all<<<(unsigned)hb, SORT_THREADS, 0, s>>>(hi, lo, n, nlo, nhi, digit_hist);
    cudaMemcpyAsync(host_hist, digit_hist, MAX_DIGITS * RADIX * sizeof(uint32_t),
                    cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    int passes[MAX_DIGITS], np = 0;
    for (int d = 0; d < MAX_DIGITS; ++d) {
        if (d < 8 && d >= nlo) continue;
        if (d >= 8 && d - 8 >= nhi) continue;
        bool constant = false;
        for (int b = 0; b < RADIX; ++b)
            if (host_hist[d * RADIX + b] == n) constant = true;
        if (!constant) passes[np++] = d;
    }
    const uint64_t ntiles = (n + SORT_TILE - 1) / SORT_TILE;
    uint32_t *hi_a = hi, *hi_b = tmp_hi;
    uint64_t *lo_a = lo, *lo_b = tmp_lo;
    for (int k = 0; k < np; ++k) {
        const int sel = passes[k];
        ++g_launches;
        k_count<<<(unsigned)ntiles, SORT_THREADS, 0, s>>>(hi_a, lo_a, n, sel, tile_counts);
        ++g_launches;
        k_scan_digit<<<RADIX, SCAN_THREADS, 0, s>>>(tile_counts, ntiles, digit_hist + sel * RADIX);
        ++g_launches;
        k_scatter<<<(unsigned)ntiles, SORT_THREADS, 0, s>>>(hi_a, lo_a, nullptr, hi_b, lo_b,
                                                            nullptr, n, sel, tile_counts);
        std::swap(hi_a, hi_b);
        std::swap(lo_a, lo_b);
    }
    if (np & 1) {
        cudaMemcpyAsync(lo, lo_a, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(hi, hi_a, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    }
}

}  // namespace rpp
