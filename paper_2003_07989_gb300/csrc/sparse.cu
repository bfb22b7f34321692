// sparse.cu -- the thresholded ("sparse 1-skeleton") form of the filtration
// construction and of the apparent-pair pass for dimensions p >= 2 (Sec.
// "Computation Induced by Sparse 1-Skeletons" and "Enumerating Cofacets of
// Simplices Induced by a Sparse 1-Skeleton in Ripser"; Sec. "Warp-based
// Filtering").
//
// With a threshold t well below the enclosing radius most of the C(n, p+1)
// indices of dimension p name simplices with an edge longer than t. Instead
// of decoding every index, the simplices are enumerated as cliques of the
// threshold graph G_t (an edge wherever D[a][b] <= t):
//   * G_t is kept as neighbour lists in ascending vertex order (CSR), built
//     row by row with warp-ballot compaction;
//   * every p-simplex {v_0 > ... > v_{p-1} > w} is its facet s = {v_0 .. v_{p-1}}
//     (a (p-1)-simplex inside t) plus a vertex w below v_{p-1}; w runs over the
//     neighbours of v_{p-1} below v_{p-1} (a prefix of its list), and the other
//     p - 1 distances D[v_i][w] are read from the dense matrix. Each simplex is
//     found once, from its facet without its lowest vertex. One warp takes one
//     facet; the lanes walk the neighbour prefix and compact the kept
//     simplices with one atomic per warp and step;
//   * clearing tests the index against the previous dimension's deaths, two
//     sorted arrays (apparent taus and the pairs the host found), by binary
//     search instead of a bitmap over C(n, p+1) bits;
//   * the apparent test of a column scans, from the largest vertex down, only
//     the neighbour list of the column's vertex of smallest degree: every
//     cofacet inside t adds a neighbour of each vertex of the column.
// A count pass sizes the outputs before the writing pass.
#include "device_common.cuh"
#include "internal.h"

namespace rpp {

namespace {

// deg[a] = #{ w != a : D[a][w] <= t }, one warp per row.
__global__ void __launch_bounds__(256) k_csr_degree(const float *__restrict__ D, int64_t ld,
                                                    int64_t n, const DevState *st,
                                                    unsigned long long *__restrict__ deg) {
    const float t = st->t;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < n; a += nwarps) {
        const float *row = D + a * ld;
        unsigned long long c = 0;
        for (int64_t w = lane; w < n; w += 32) c += (w != a && row[w] <= t) ? 1 : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL_MASK, c, o);
        if (lane == 0) deg[a] = c;
    }
}

// In place: off[0..n] = exclusive prefix sums of deg[0..n-1] (off = deg + 0,
// with off[n] the total). One block.
__global__ void __launch_bounds__(1024) k_csr_offsets(unsigned long long *__restrict__ off,
                                                      int64_t n) {
    __shared__ unsigned long long s_warp[32];
    __shared__ unsigned long long s_carry;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += 1024) {
        const int64_t i = base + tid;
        const unsigned long long v = i < n ? off[i] : 0ull;
        unsigned long long incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_warp[w] = incl;
        __syncthreads();
        unsigned long long before = s_carry;
        for (int k = 0; k < w; ++k) before += s_warp[k];
        if (i < n) off[i] = before + incl - v;
        __syncthreads();
        if (tid == 1023) s_carry = before + incl;
        __syncthreads();
    }
    if (tid == 0) off[n] = s_carry;
}

// The neighbours of a, ascending: one warp per row, ballot compaction.
__global__ void __launch_bounds__(256) k_csr_fill(const float *__restrict__ D, int64_t ld,
                                                  int64_t n, const DevState *st,
                                                  const unsigned long long *__restrict__ off,
                                                  uint32_t *__restrict__ nbr) {
    const float t = st->t;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < n; a += nwarps) {
        const float *row = D + a * ld;
        unsigned long long at = off[a];
        const unsigned long long end = off[a + 1];
        for (int64_t w0 = 0; w0 < n; w0 += 32) {
            const int64_t w = w0 + lane;
            const bool keep = w < n && w != a && row[w] <= t;
            const unsigned ball = __ballot_sync(FULL_MASK, keep);
            if (keep) {
                const unsigned long long pos = at + __popc(ball & lanemask_lt());
                if (pos < end) nbr[pos] = (uint32_t)w;
            }
            at += __popc(ball);
        }
    }
}

__device__ __forceinline__ bool sorted_contains(const uint64_t *a, uint64_t len, uint64_t key) {
    uint64_t lo = 0, hi = len;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo < len && a[lo] == key;
}

// p-simplices from the (p-1)-simplices `prev` (indices). Counts into
// cnt[0] (all simplices inside t) and cnt[1] (columns: not cleared); when
// `write` is set, appends the columns' keys and, if all_out is given, every
// simplex's index.
template <int P>
__global__ void __launch_bounds__(256) k_sparse_build(
    const float *__restrict__ D, int64_t ld, int64_t n, const uint64_t *__restrict__ B,
    const uint64_t *__restrict__ prev, uint64_t nprev, const unsigned long long *__restrict__ off,
    const uint32_t *__restrict__ nbr, const DevState *st, const uint64_t *__restrict__ dead_a,
    uint64_t ndead_a, const uint64_t *__restrict__ dead_b, uint64_t ndead_b, bool write,
    unsigned long long *cnt, uint32_t *__restrict__ key_hi, uint64_t *__restrict__ key_lo,
    uint64_t col_cap, uint64_t *__restrict__ all_out, uint64_t all_cap) {
    const float t = st->t;
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long n_all = 0, n_col = 0;  // count pass: per-lane tallies
    for (uint64_t f = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; f < nprev;
         f += nwarps) {
        int u[P];  // the facet, u[0] > ... > u[P-1]
        decode_simplex<P - 1>(prev[f], B, n, u);
        float pd = 0.0f;
        uint64_t base = 0;  // index of the facet's vertices in the p-simplex
#pragma unroll
        for (int a = 0; a < P; ++a) {
            base += B[(int64_t)(P + 1 - a) * (n + 1) + u[a]];
#pragma unroll
            for (int b = a + 1; b < P; ++b) pd = fmaxf(pd, D[(int64_t)u[a] * ld + u[b]]);
        }
        const int low = u[P - 1];
        const unsigned long long l0 = off[low], l1 = off[low + 1];
        for (unsigned long long j0 = l0; j0 < l1; j0 += 32) {
            const unsigned long long j = j0 + lane;
            const int w = j < l1 ? (int)nbr[j] : 0x7fffffff;
            // the list ascends: once a lane passes `low`, so do the later ones
            if (__all_sync(FULL_MASK, w >= low)) break;
            bool keep = false, col = false;
            float d = pd;
            uint64_t c = 0;
            if (w < low) {
                d = fmaxf(d, D[(int64_t)low * ld + w]);
#pragma unroll
                for (int a = 0; a < P - 1; ++a) d = fmaxf(d, D[(int64_t)u[a] * ld + w]);
                keep = d <= t;
                if (keep) {
                    c = base + (uint64_t)w;
                    col = !(sorted_contains(dead_a, ndead_a, c) ||
                            sorted_contains(dead_b, ndead_b, c));
                }
            }
            if (!write) {
                n_all += keep;
                n_col += col;
                continue;
            }
            const unsigned bk = __ballot_sync(FULL_MASK, keep);
            if (bk && all_out) {
                unsigned long long at = 0;
                if (lane == 0) at = atomicAdd(&cnt[0], (unsigned long long)__popc(bk));
                at = __shfl_sync(FULL_MASK, at, 0);
                if (keep) {
                    const uint64_t pos = at + __popc(bk & lanemask_lt());
                    if (pos < all_cap) all_out[pos] = c;
                }
            }
            const unsigned bc = __ballot_sync(FULL_MASK, col);
            if (bc) {
                unsigned long long at = 0;
                if (lane == 0) at = atomicAdd(&cnt[1], (unsigned long long)__popc(bc));
                at = __shfl_sync(FULL_MASK, at, 0);
                if (col) {
                    const uint64_t pos = at + __popc(bc & lanemask_lt());
                    if (pos < col_cap) {
                        key_hi[pos] = ~__float_as_uint(d);
                        key_lo[pos] = c;
                    }
                }
            }
        }
    }
    if (!write) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            n_all += __shfl_xor_sync(FULL_MASK, n_all, o);
            n_col += __shfl_xor_sync(FULL_MASK, n_col, o);
        }
        if (lane == 0) {
            if (n_all) atomicAdd(&cnt[0], n_all);
            if (n_col) atomicAdd(&cnt[1], n_col);
        }
    }
}

// The apparent-pair test (Alg. 3, as k_apparent) with the candidates taken
// from the neighbour list of the column's vertex of smallest degree, largest
// vertex first: a group of G lanes reads G consecutive list entries per block
// and U blocks per step.
template <int P, int G, int U>
__global__ void __launch_bounds__(256, 4) k_apparent_sparse(
    const float *__restrict__ D, int64_t ld, int64_t n, const uint64_t *__restrict__ B,
    const unsigned long long *__restrict__ off, const uint32_t *__restrict__ nbr,
    const uint32_t *__restrict__ key_hi, const uint64_t *__restrict__ key_lo, uint64_t ncols_cap,
    const unsigned long long *d_ncols, DevState *__restrict__ st, uint8_t *__restrict__ status,
    uint64_t *__restrict__ pivot, float *__restrict__ pdiam) {
    const float t = st->t;
    const uint64_t ncols = count_of(d_ncols, ncols_cap);
    unsigned long long scanned = 0;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, gl = lane % G;
    const unsigned gmask = (G == 32) ? FULL_MASK : (((1u << G) - 1u) << (grp * G));
    const uint64_t ngroups = ((uint64_t)gridDim.x * blockDim.x) / G;
    uint64_t c = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;

    bool have = false;
    int v[P + 1];
    const float *row[P + 1];
    const uint32_t *list = nullptr;
    float diam = 0.0f, best_d = 0.0f;
    int64_t scan = 0, len = 0;
    int best_v = -1;

    for (;;) {
        if (!have) {
            while (c < ncols && status[c] == COL_CLEARED) c += ngroups;
            if (c < ncols) {
                have = true;
                diam = __uint_as_float(~key_hi[c]);
                decode_simplex<P>(key_lo[c], B, n, v);
                int k = 0;
                unsigned long long kd = off[v[0] + 1] - off[v[0]];
#pragma unroll
                for (int i = 0; i <= P; ++i) {
                    row[i] = D + (int64_t)v[i] * ld;
                    const unsigned long long di = off[v[i] + 1] - off[v[i]];
                    if (di < kd) {
                        kd = di;
                        k = i;
                    }
                }
                list = nbr + off[v[k]];
                len = (int64_t)kd;
                scan = len - 1;
                best_d = __uint_as_float(0x7f800000u);
                best_v = -1;
            }
        }
        if (!__any_sync(FULL_MASK, have)) break;

        bool ok[U];
        float dv[U][P + 1];
        int xs[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ok[u] = false;
            xs[u] = -1;
            const int64_t j = scan - gl - u * G;
            if (have && j >= 0) {
                const int x = (int)list[j];
                xs[u] = x;
                bool member = false;
#pragma unroll
                for (int i = 0; i <= P; ++i) member |= (x == v[i]);
                if (!member) {
                    float m = 0.0f;
#pragma unroll
                    for (int i = 0; i <= P; ++i) {
                        dv[u][i] = row[i][x];
                        m = fmaxf(m, dv[u][i]);
                    }
                    ok[u] = m <= diam;
                    const float cd = fmaxf(m, diam);
                    if (cd <= t && cd < best_d) {
                        best_d = cd;
                        best_v = x;
                    }
                }
            }
        }
        unsigned gb[U];
#pragma unroll
        for (int u = 0; u < U; ++u) gb[u] = (__ballot_sync(FULL_MASK, ok[u]) & gmask) >> (grp * G);
        if (have) {
            int first = -1, fu = 0;
#pragma unroll
            for (int u = U - 1; u >= 0; --u)
                if (gb[u]) {
                    first = __ffs(gb[u]) - 1;
                    fu = u;
                }
            if (first >= 0) {
                if (gl == first) {
                    int x = xs[0];
                    float dx[P + 1];
#pragma unroll
                    for (int i = 0; i <= P; ++i) {
                        dx[i] = dv[0][i];
#pragma unroll
                        for (int u = 1; u < U; ++u)
                            if (fu == u) dx[i] = dv[u][i];
                    }
#pragma unroll
                    for (int u = 1; u < U; ++u)
                        if (fu == u) x = xs[u];
                    bool apparent = true;
#pragma unroll
                    for (int i = 0; i <= P; ++i) {
                        if (v[i] > x) {  // facet tau - {v_i} precedes sigma
                            float fd = 0.0f;
#pragma unroll
                            for (int k = 0; k <= P; ++k)
                                if (k != i) fd = fmaxf(fd, dx[k]);
#pragma unroll
                            for (int a = 0; a <= P; ++a)
#pragma unroll
                                for (int b = a + 1; b <= P; ++b)
                                    if (a != i && b != i) fd = fmaxf(fd, row[a][v[b]]);
                            if (fd == diam) apparent = false;
                        }
                    }
                    status[c] = apparent ? COL_APPARENT : COL_LEFTOVER;
                    pivot[c] = cofacet_index<P>(v, x, B, n);
                    pdiam[c] = diam;
                    scanned += (unsigned long long)(len - (scan - gl - fu * G));  // entries down to the hit
                }
                have = false;
                c += ngroups;
            } else if (scan - U * G < 0) {
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) {
                    const float od = __shfl_xor_sync(gmask, best_d, o);
                    const int ov = __shfl_xor_sync(gmask, best_v, o);
                    if (od < best_d || (od == best_d && ov > best_v)) {
                        best_d = od;
                        best_v = ov;
                    }
                }
                if (gl == 0) {
                    status[c] = COL_LEFTOVER;
                    pivot[c] = best_v >= 0 ? cofacet_index<P>(v, best_v, B, n) : NO_PIVOT;
                    pdiam[c] = best_d;
                    scanned += (unsigned long long)len;
                }
                have = false;
                c += ngroups;
            } else {
                scan -= U * G;
            }
        }
    }
    unsigned long long w = scanned;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(FULL_MASK, w, o);
    if (lane == 0 && w) atomicAdd(&st->scanned, w);
}

inline unsigned grid_for(uint64_t warps_needed) {
    uint64_t blocks = (warps_needed + 7) / 8;
    if (blocks > 152ull * 8) blocks = 152ull * 8;
    return (unsigned)(blocks ? blocks : 1);
}

template <int P>
void sparse_build_p(const float *D, int64_t ld, int64_t n, const uint64_t *binom,
                    const uint64_t *prev, uint64_t nprev, const unsigned long long *off,
                    const uint32_t *nbr, const DevState *st, const uint64_t *dead_a,
                    uint64_t ndead_a, const uint64_t *dead_b, uint64_t ndead_b, bool write,
                    unsigned long long *cnt, uint32_t *key_hi, uint64_t *key_lo, uint64_t col_cap,
                    uint64_t *all_out, uint64_t all_cap, cudaStream_t s) {
    ++g_launches;
    k_sparse_build<P><<<grid_for(nprev), 256, 0, s>>>(D, ld, n, binom, prev, nprev, off, nbr, st,
                                                      dead_a, ndead_a, dead_b, ndead_b, write, cnt,
                                                      key_hi, key_lo, col_cap, all_out, all_cap);
}

template <int P>
void apparent_sparse_p(const float *D, int64_t ld, int64_t n, const uint64_t *binom,
                       const unsigned long long *off, const uint32_t *nbr, const uint32_t *key_hi,
                       const uint64_t *key_lo, uint64_t ncols, const unsigned long long *d_ncols,
                       DevState *st, uint8_t *status, uint64_t *pivot, float *pdiam, int sms,
                       cudaStream_t s) {
    constexpr int G = 4, U = 2;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apparent_sparse<P, G, U>, 256, 0);
    if (per_sm < 1) per_sm = 1;
    uint64_t blocks = (uint64_t)sms * per_sm;
    const uint64_t need = (ncols * G + 255) / 256;
    if (need < blocks) blocks = need;
    if (blocks == 0) return;
    ++g_launches;
    k_apparent_sparse<P, G, U><<<(unsigned)blocks, 256, 0, s>>>(
        D, ld, n, binom, off, nbr, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam);
}

}  // namespace

void launch_csr_build(const float *D, int64_t ld, int64_t n, const DevState *st,
                      unsigned long long *off, uint32_t *nbr, bool fill, cudaStream_t s) {
    if (n <= 0) return;
    const unsigned blocks = grid_for((uint64_t)n);
    if (!fill) {
        ++g_launches;
        k_csr_degree<<<blocks, 256, 0, s>>>(D, ld, n, st, off);
        ++g_launches;
        k_csr_offsets<<<1, 1024, 0, s>>>(off, n);
    } else {
        ++g_launches;
        k_csr_fill<<<blocks, 256, 0, s>>>(D, ld, n, st, off, nbr);
    }
}

void launch_sparse_build(const float *D, int64_t ld, int64_t n, int p, const uint64_t *binom,
                         const uint64_t *prev, uint64_t nprev, const unsigned long long *off,
                         const uint32_t *nbr, const DevState *st, const uint64_t *dead_a,
                         uint64_t ndead_a, const uint64_t *dead_b, uint64_t ndead_b, bool write,
                         unsigned long long *cnt, uint32_t *key_hi, uint64_t *key_lo,
                         uint64_t col_cap, uint64_t *all_out, uint64_t all_cap, cudaStream_t s) {
    if (nprev == 0) return;
    switch (p) {
        case 2: sparse_build_p<2>(D, ld, n, binom, prev, nprev, off, nbr, st, dead_a, ndead_a, dead_b, ndead_b, write, cnt, key_hi, key_lo, col_cap, all_out, all_cap, s); break;
        case 3: sparse_build_p<3>(D, ld, n, binom, prev, nprev, off, nbr, st, dead_a, ndead_a, dead_b, ndead_b, write, cnt, key_hi, key_lo, col_cap, all_out, all_cap, s); break;
        case 4: sparse_build_p<4>(D, ld, n, binom, prev, nprev, off, nbr, st, dead_a, ndead_a, dead_b, ndead_b, write, cnt, key_hi, key_lo, col_cap, all_out, all_cap, s); break;
        default: break;
    }
}

void launch_apparent_sparse(const float *D, int64_t ld, int64_t n, int p, const uint64_t *binom,
                            const unsigned long long *off, const uint32_t *nbr,
                            const uint32_t *key_hi, const uint64_t *key_lo, uint64_t ncols,
                            const unsigned long long *d_ncols, DevState *st, uint8_t *status,
                            uint64_t *pivot, float *pdiam, int sms, cudaStream_t s) {
    if (ncols == 0) return;
    switch (p) {
        case 2: apparent_sparse_p<2>(D, ld, n, binom, off, nbr, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, sms, s); break;
        case 3: apparent_sparse_p<3>(D, ld, n, binom, off, nbr, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, sms, s); break;
        case 4: apparent_sparse_p<4>(D, ld, n, binom, off, nbr, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, sms, s); break;
        default: break;
    }
}

}  // namespace rpp
