// device_common.cuh -- device helpers for the combinatorial number system.
//
// A p-simplex with vertices v_p > ... > v_0 has index
//   cidx = C(v_p, p+1) + ... + C(v_1, 2) + C(v_0, 1)
// (Sec. "The Combinatorial Number System"). Index order is the lexicographic
// order of the decreasing vertex tuple. The table B holds C(v, k) row-major by
// k: B[k * (n + 1) + v] for k = 0..kmax, v = 0..n.
#pragma once

#include <stdint.h>

namespace rpp {

constexpr unsigned FULL_MASK = 0xffffffffu;

// Largest v in [lo, hi] with Bk[v] <= c (Bk[lo] <= c holds for lo = k - 1).
__device__ __forceinline__ int largest_vertex(const uint64_t *Bk, uint64_t c, int lo, int hi) {
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (Bk[mid] <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Vertices x > y of the edge with index c = C(x, 2) + y: x from the inverse
// of C(x, 2) = x (x - 1) / 2 through a float square root, then exact integer
// corrections until C(x, 2) <= c < C(x + 1, 2).
__device__ __forceinline__ void decode_edge(uint64_t c, int *v) {
    int x = (int)((1.0f + sqrtf(8.0f * (float)c + 1.0f)) * 0.5f);
    if (x < 1) x = 1;
    while ((uint64_t)x * (uint64_t)(x - 1) / 2 > c) --x;
    while ((uint64_t)(x + 1) * (uint64_t)x / 2 <= c) ++x;
    v[0] = x;
    v[1] = (int)(c - (uint64_t)x * (uint64_t)(x - 1) / 2);
}

// Decode a dimension-P index into vertices v[0] > v[1] > ... > v[P].
template <int P>
__device__ __forceinline__ void decode_simplex(uint64_t c, const uint64_t *B, int64_t n, int *v) {
    if constexpr (P == 1) {
        decode_edge(c, v);
        return;
    }
    int hi = (int)n - 1;
#pragma unroll
    for (int i = 0; i <= P; ++i) {
        const int k = P + 1 - i;
        const uint64_t *Bk = B + (int64_t)k * (n + 1);
        int x = largest_vertex(Bk, c, k - 1, hi);
        v[i] = x;
        c -= Bk[x];
        hi = x - 1;
    }
}

// Index of the cofacet sigma + {w} of a dimension-P simplex v[0] > ... > v[P]
// (w not a vertex of sigma).
template <int P>
__device__ __forceinline__ uint64_t cofacet_index(const int *v, int w, const uint64_t *B,
                                                  int64_t n) {
    if constexpr (P == 1) {
        // a triangle {a > b > c}: C(a, 3) + C(b, 2) + c, in exact integer
        // arithmetic (a (a-1) (a-2) < 2^63 for every admissible n)
        uint64_t a = (uint64_t)v[0], b = (uint64_t)v[1], c = (uint64_t)w;
        if (c > a) {
            const uint64_t t = c;
            c = b;
            b = a;
            a = t;
        } else if (c > b) {
            const uint64_t t = c;
            c = b;
            b = t;
        }
        return a * (a - 1) * (a - 2) / 6 + b * (b - 1) / 2 + c;
    }
    uint64_t c = 0;
    int k = P + 2;  // the largest vertex of the cofacet carries C(., P + 2)
    bool placed = false;
#pragma unroll
    for (int i = 0; i <= P; ++i) {
        if (!placed && w > v[i]) {
            c += B[(int64_t)k * (n + 1) + w];
            --k;
            placed = true;
        }
        c += B[(int64_t)k * (n + 1) + v[i]];
        --k;
    }
    if (!placed) c += B[(int64_t)1 * (n + 1) + w];
    return c;
}

// A launch's item count: min(*d_count, cap) when the count lives in device
// memory (launches queued before the host knows it), else cap.
__device__ __forceinline__ uint64_t count_of(const unsigned long long *d_count, uint64_t cap) {
    if (!d_count) return cap;
    const uint64_t c = *d_count;
    return c < cap ? c : cap;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Load rows k = 0..kmax of the binomial table into shared memory when it fits;
// returns the pointer the kernel should use (shared or global).
__device__ __forceinline__ const uint64_t *stage_binomial(const uint64_t *gB, int64_t n, int kmax,
                                                          uint64_t *sB, bool use_smem) {
    if (!use_smem) return gB;
    const int64_t total = (int64_t)(kmax + 1) * (n + 1);
    for (int64_t i = threadIdx.x; i < total; i += blockDim.x) sB[i] = gB[i];
    __syncthreads();
    return sB;
}

}  // namespace rpp
