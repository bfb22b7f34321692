// reduce_small.cu -- the submatrix reduction of dimension 1 (Alg. 1 on the
// leftover columns, Sec. "Core System Optimizations") on the device, for the
// clouds of a fused batch whose columns' walks are short.
//
// One warp takes one cloud and reduces its leftover columns in index order,
// exactly as Alg. 1 does (each column's additions only read columns before
// it). A column is the coboundary of an edge set V (the reduction-matrix
// form): V starts as the column's own edge, and an addition toggles edges in
// V (an apparent owner adds its one edge; an earlier leftover column adds its
// final edge set). V is kept as an adjacency bitset of the cloud in shared
// memory, so a triangle {x, y, w} has nonzero coefficient exactly when an odd
// number of its three edges are set.
//   * The first pivot is the column's unreduced pivot, which the fused pass
//     found (the oldest cofacet inside the threshold).
//   * The owner of a pivot tau: its youngest facet s (longest edge, ties by
//     the smaller index) owns it as an apparent pair when the fused pass
//     recorded tau's extra vertex as s's apparent vertex; otherwise an
//     earlier leftover column whose final pivot is tau; otherwise the pivot
//     is free and the column is paired with it.
//   * After an addition every entry up to and including the old pivot is
//     zero (the owner's column has that pivot and nothing older), so the next
//     pivot is the oldest nonzero triangle younger than it. Each edge of V
//     keeps a lazy cursor: its oldest cofacet inside the threshold that the
//     column has not passed (found by a warp scan of the third vertices). The
//     smallest head is a nonzero entry when an odd number of V's edges hold
//     it (a triangle's edges in V all have it as their head); an even one
//     cancels, and those cursors move on.
// A cloud whose column needs more than RS_BUDGET additions, or whose V grows
// past RS_VMAX edges (the long walks that the host sweeps level by level),
// stops and is handed back whole: status 1, and the host reduces it.
#include "device_common.cuh"
#include "internal.h"

namespace rpp {

namespace {

constexpr int RS_VMAX = 64;     // edges of V per column kept by the device
constexpr int RS_BUDGET = 64;   // additions per column before the cloud goes back

// Age key of a triangle: diameter bits over the complemented index; ascending
// key is the filtration order (older first: smaller diameter, then larger index).
__device__ __forceinline__ uint64_t tri_key(float d, uint32_t idx) {
    return ((uint64_t)__float_as_uint(d) << 32) | (uint64_t)(0xffffffffu - idx);
}

__device__ __forceinline__ uint32_t c3(uint32_t v) {
    return (uint32_t)((uint64_t)v * (v - 1) * (v - 2) / 6);
}
__device__ __forceinline__ uint32_t c2(uint32_t v) { return v * (v - 1) / 2; }

// Index of the triangle with vertices a, b, c (any order).
__device__ __forceinline__ uint32_t tri_index(int a, int b, int c) {
    int v0 = a, v1 = b, v2 = c;
    if (v0 < v1) { const int s = v0; v0 = v1; v1 = s; }
    if (v1 < v2) { const int s = v1; v1 = v2; v2 = s; }
    if (v0 < v1) { const int s = v0; v0 = v1; v1 = s; }
    return c3((uint32_t)v0) + c2((uint32_t)v1) + (uint32_t)v2;
}

// Vertices v0 > v1 > v2 of triangle index t.
__device__ __forceinline__ void tri_vertices(uint32_t t, int *v) {
    int x = (int)cbrtf(6.0f * (float)t) + 1;
    if (x < 2) x = 2;
    while (x > 2 && c3((uint32_t)x) > t) --x;
    while (c3((uint32_t)(x + 1)) <= t) ++x;
    v[0] = x;
    int e[2];
    decode_edge((uint64_t)(t - c3((uint32_t)x)), e);
    v[1] = e[0];
    v[2] = e[1];
}

// The oldest cofacet of edge e = {x > y} inside the threshold with age key
// above `after` (~0 if none): the warp scans the third vertices.
__device__ uint64_t cursor_next(const float *D, int n, float t, uint32_t e, uint64_t after) {
    int xy[2];
    decode_edge((uint64_t)e, xy);
    const int x = xy[0], y = xy[1];
    const float dxy = D[x * n + y];
    const float *rx = D + (int64_t)x * n, *ry = D + (int64_t)y * n;
    uint64_t best = ~0ull;
    for (int w = threadIdx.x & 31; w < n; w += 32) {
        if (w == x || w == y) continue;
        const float d = fmaxf(dxy, fmaxf(rx[w], ry[w]));
        if (!(d <= t)) continue;
        const uint64_t key = tri_key(d, tri_index(x, y, w));
        if (key > after && key < best) best = key;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t v = __shfl_xor_sync(FULL_MASK, best, o);
        best = v < best ? v : best;
    }
    return best;
}

// V as an edge list with one lazy cursor per edge (its next cofacet, by age,
// that the working column has not passed) and an adjacency bitset for
// membership. Lane 0 writes the shared arrays; every lane keeps vcount.
struct VSet {
    uint32_t *bits;
    int w32;
    uint32_t *edge;
    uint64_t *head;
    int vcount;
    __device__ bool in(int a, int b) const { return (bits[a * w32 + (b >> 5)] >> (b & 31)) & 1u; }
    __device__ void flip(int x, int y) {
        bits[x * w32 + (y >> 5)] ^= 1u << (y & 31);
        bits[y * w32 + (x >> 5)] ^= 1u << (x & 31);
    }
    // Toggle e in V; an entering edge's cursor starts past `after`. False when
    // the list would overflow (or, never expected, misses a member).
    __device__ bool toggle(const float *D, int n, float t, uint32_t e, uint64_t after) {
        int xy[2];
        decode_edge((uint64_t)e, xy);
        const int lane = threadIdx.x & 31;
        if (in(xy[0], xy[1])) {  // leaves V: swap-remove
            int pos = -1;
            for (int i = lane; i < vcount; i += 32)
                if (edge[i] == e) pos = i;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pos = max(pos, __shfl_xor_sync(FULL_MASK, pos, o));
            if (pos < 0) return false;
            __syncwarp();
            if (lane == 0) {
                edge[pos] = edge[vcount - 1];
                head[pos] = head[vcount - 1];
                flip(xy[0], xy[1]);
            }
            --vcount;
        } else {
            if (vcount >= RS_VMAX) return false;
            const uint64_t h = cursor_next(D, n, t, e, after);
            if (lane == 0) {
                edge[vcount] = e;
                head[vcount] = h;
                flip(xy[0], xy[1]);
            }
            ++vcount;
        }
        __syncwarp();
        return true;
    }
    // Every cursor at or before k moves past k.
    __device__ void pass(const float *D, int n, float t, uint64_t k) {
        for (int q = 0; q < vcount; ++q) {
            const uint64_t h = head[q];
            if (h <= k) {
                const uint64_t nh = cursor_next(D, n, t, edge[q], k);
                if ((threadIdx.x & 31) == 0) head[q] = nh;
                __syncwarp();
            }
        }
    }
    // The oldest nonzero entry of the working column past the cursors: the
    // smallest head held by an odd number of V's edges (a triangle's edges in
    // V all have it as their head, the cursors being past every older entry);
    // even ones cancel and their cursors move on. ~0 if the column is zero.
    __device__ uint64_t pivot(const float *D, int n, float t) {
        const int lane = threadIdx.x & 31;
        for (;;) {
            uint64_t m = ~0ull;
            for (int q = lane; q < vcount; q += 32) m = head[q] < m ? head[q] : m;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const uint64_t v = __shfl_xor_sync(FULL_MASK, m, o);
                m = v < m ? v : m;
            }
            if (m == ~0ull) return m;
            int c = 0;
            for (int q = lane; q < vcount; q += 32) c += head[q] == m;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL_MASK, c, o);
            if (c & 1) return m;
            pass(D, n, t, m);
        }
    }
};

__global__ void __launch_bounds__(32) k_reduce_small(
    const float *__restrict__ Dall, const uint16_t *__restrict__ awall,
    const ReduceJob *__restrict__ jobs, const Leftover *__restrict__ left,
    uint32_t *__restrict__ vpool, uint8_t *__restrict__ vcnt, uint64_t *__restrict__ death,
    float *__restrict__ ddiam, int32_t *__restrict__ status, int32_t *__restrict__ adds_out) {
    extern __shared__ uint32_t bits[];
    __shared__ uint32_t s_edge[RS_VMAX];
    __shared__ uint64_t s_head[RS_VMAX];
    const ReduceJob J = jobs[blockIdx.x];
    const int n = J.n, w32 = (n + 31) >> 5, lane = threadIdx.x & 31;
    const float *D = Dall + J.d_off;  // row stride n
    const uint16_t *aw = awall + J.aw_off;
    const Leftover *L = left + J.left_off;
    const float t = J.t;
    for (int i = lane; i < n * w32; i += 32) bits[i] = 0;
    __syncwarp();
    VSet V{bits, w32, s_edge, s_head, 0};
    int total_adds = 0;
    bool bail = false;
    for (int64_t j = 0; j < J.nleft && !bail; ++j) {
        V.vcount = 0;
        bool have = L[j].pivot != NO_PIVOT;
        uint64_t k = have ? tri_key(L[j].pdiam, (uint32_t)L[j].pivot) : ~0ull;
        // the column's own edge; its oldest cofacet is the unreduced pivot k
        if (lane == 0) {
            int xy[2];
            decode_edge(L[j].sigma, xy);
            s_edge[0] = (uint32_t)L[j].sigma;
            s_head[0] = k;
            V.flip(xy[0], xy[1]);
        }
        V.vcount = 1;
        __syncwarp();
        int adds = 0;
        while (have) {
            // the owner of pivot k
            const uint32_t tau = 0xffffffffu - (uint32_t)k;
            int v[3];
            tri_vertices(tau, v);
            const float fd[3] = {D[v[1] * n + v[2]], D[v[0] * n + v[2]], D[v[0] * n + v[1]]};
            int r = 0;  // facets in increasing index order: without v0, v1, v2
            for (int i = 1; i < 3; ++i)
                if (fd[i] > fd[r]) r = i;
            const int sa = r == 0 ? v[1] : v[0], sb = r == 2 ? v[1] : v[2];
            const uint32_t s = c2((uint32_t)sa) + (uint32_t)sb;
            int owner = -1;  // 0: apparent; 1: a leftover column
            int64_t oi = -1;
            if (aw[s] == (uint16_t)v[r]) {
                owner = 0;
            } else {
                for (int64_t i = lane; i < j; i += 32)
                    if (death[J.left_off + i] == (uint64_t)tau) oi = i;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const int64_t x = __shfl_xor_sync(FULL_MASK, oi, o);
                    oi = x > oi ? x : oi;
                }
                if (oi >= 0) owner = 1;
            }
            if (owner < 0) break;  // free: the column is paired with k
            if (++adds > RS_BUDGET) {
                bail = true;
                break;
            }
            // the addition (every entry up to k is then zero), cursors past k
            if (owner == 0) {
                if (!V.toggle(D, n, t, s, k)) {
                    bail = true;
                    break;
                }
            } else {
                const uint32_t *Vi = vpool + (J.left_off + oi) * RS_VMAX;
                const int ci = vcnt[J.left_off + oi];
                for (int q = 0; q < ci && !bail; ++q)
                    if (!V.toggle(D, n, t, Vi[q], k)) bail = true;
                if (bail) break;
            }
            V.pass(D, n, t, k);
            k = V.pivot(D, n, t);
            if (k == ~0ull) have = false;  // zero column: an essential class
        }
        total_adds += adds;
        if (!bail) {
            if (lane == 0) {
                death[J.left_off + j] = have ? (uint64_t)(0xffffffffu - (uint32_t)k) : NO_PIVOT;
                ddiam[J.left_off + j] = have ? __uint_as_float((uint32_t)(k >> 32)) : 0.0f;
                vcnt[J.left_off + j] = (uint8_t)V.vcount;
            }
            for (int q = lane; q < V.vcount; q += 32)
                vpool[(J.left_off + j) * RS_VMAX + q] = s_edge[q];
        }
        __syncwarp();
        // clear V's bits for the next column
        for (int q = 0; q < V.vcount; ++q) {
            int xy[2];
            decode_edge((uint64_t)s_edge[q], xy);
            if (lane == 0) {
                bits[xy[0] * w32 + (xy[1] >> 5)] &= ~(1u << (xy[1] & 31));
                bits[xy[1] * w32 + (xy[0] >> 5)] &= ~(1u << (xy[0] & 31));
            }
        }
        __syncwarp();
    }
    if (lane == 0) {
        status[blockIdx.x] = bail ? 1 : 0;
        adds_out[blockIdx.x] = total_adds;
    }
}

}  // namespace

size_t reduce_small_vpool_words(uint64_t nleft) { return (size_t)nleft * RS_VMAX; }

void launch_reduce_small(const float *D, const uint16_t *aw, const ReduceJob *jobs, int njobs,
                         int nmax, const Leftover *left, uint32_t *vpool, uint8_t *vcnt,
                         uint64_t *death, float *ddiam, int32_t *status, int32_t *adds,
                         cudaStream_t s) {
    if (njobs <= 0) return;
    const size_t smem = (size_t)nmax * ((nmax + 31) / 32) * 4;
    allow_dynamic_smem((const void *)k_reduce_small, smem);
    ++g_launches;
    k_reduce_small<<<(unsigned)njobs, 32, smem, s>>>(D, aw, jobs, left, vpool, vcnt, death, ddiam,
                                                    status, adds);
}

}  // namespace rpp
