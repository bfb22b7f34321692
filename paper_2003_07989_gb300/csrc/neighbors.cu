// neighbors.cu -- per-vertex neighbour lists sorted by distance, for the host
// reduction's lazy coboundary enumeration.
//
// Row v of the output lists every vertex w (v itself included) in increasing
// (D[v][w], w) order, each as the key (bits(D[v][w]) << 32) | w. One block sorts one row: the keys (distance bits << 32 |
// w) are bitonic-sorted in shared memory (distances are non-negative, so
// their bit patterns order like the values).
#include "internal.h"

namespace rpp {

namespace {

__global__ void __launch_bounds__(512) k_sort_rows(const float *__restrict__ D, int64_t ld,
                                                   int64_t n, int pow2,
                                                   uint64_t *__restrict__ out) {
    extern __shared__ unsigned long long keys[];
    const int64_t row = blockIdx.x;
    for (int i = threadIdx.x; i < pow2; i += blockDim.x)
        keys[i] = i < n ? ((unsigned long long)__float_as_uint(D[row * ld + i]) << 32) | (unsigned)i
                        : ~0ull;
    __syncthreads();
    for (int k = 2; k <= pow2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < pow2; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const unsigned long long a = keys[i], b = keys[l];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) out[row * n + i] = keys[i];
}

}  // namespace

bool launch_sort_rows(const float *D, int64_t ld, int64_t n, uint64_t *out, cudaStream_t s) {
    int pow2 = 1;
    while (pow2 < n) pow2 <<= 1;
    const size_t smem = (size_t)pow2 * 8;
    if (smem > 200 * 1024) return false;
    allow_dynamic_smem((const void *)k_sort_rows, smem);
    ++g_launches;
    k_sort_rows<<<(unsigned)n, 512, smem, s>>>(D, ld, n, pow2, out);
    return true;
}

}  // namespace rpp
