// apparent.cu -- the apparent-pair pass (Alg. 3, the Apparent Pairs Lemma and
// Corollary "massively parallel") and the partition of its output (Fig.
// "post-apparent", Sec. "Core System Optimizations").
//
// Column sigma (a p-simplex, vertices v_0 > ... > v_p) is tested on its own:
//  (1) tau = sigma + {w*} where w* is the LARGEST vertex outside sigma with
//      max_i D[v_i][w*] <= diam(sigma). Cofacet indices grow with the added
//      vertex, so tau is the lexicographically greatest cofacet of equal
//      diameter, i.e. the oldest cofacet (condition 1 of the lemma). If no
//      such vertex exists sigma is not apparent.
//  (2) The facets of tau in increasing index order drop its vertices in
//      decreasing order (Alg. 5); the facets before sigma drop a vertex
//      w > w*. sigma is apparent iff none of them has diam == diam(sigma)
//      (condition 2; Proposition "apparent-support").
// The kernel is bound by the latency of its L1/L2 loads and by issue. It is
// compiled for up to 64 registers a thread (dimension 1 takes 48: five
// 256-thread blocks per SM); squeezed into 32 registers for eight blocks, the
// test spilled to local memory and ran 4-30% slower depending on the shape. The paper runs one thread per column. Here a group of G
// lanes owns a column and tests U blocks of G candidate vertices per step,
// lane l taking w = scan - l - u G for u < U: the reads D[v_i][w] of a block
// are contiguous, so a step is U coalesced loads of (p+1) short row segments
// (the rows are L2-resident), all in flight before any test, and one warp
// ballot per block picks the largest qualifying w (first block, lowest
// lane). Groups of one warp advance independently: a group that finishes
// takes its next column in the same iteration, so no lane idles while a
// neighbour scans a long column.
// While scanning, each lane also tracks the smallest max_i D[v_i][w] it has
// seen (the largest w among equals). It is needed only for a column with no
// equal-diameter cofacet: there the scan covers every vertex, every such
// value exceeds diam(sigma) and is the diameter of the cofacet sigma + {w},
// so the group's minimum is the column's oldest cofacet (its unreduced
// pivot, kept if it lies inside the threshold), which the host reduction
// uses to skip columns whose pivot nobody owns. Tracking that value rather
// than max(diam, value) under the threshold test saves two instructions per
// candidate.
#include "device_common.cuh"
#include "internal.h"

namespace rpp {

namespace {

#define INF_F __uint_as_float(0x7f800000u)

template <int P, int G, int U>
__global__ void __launch_bounds__(256, 4) k_apparent(
    const float *__restrict__ D, int64_t ld, int64_t n, const uint64_t *__restrict__ gB,
    bool smem_table, const uint32_t *__restrict__ key_hi, const uint64_t *__restrict__ key_lo,
    uint64_t ncols_cap, const unsigned long long *d_ncols, DevState *__restrict__ st,
    uint8_t *__restrict__ status, uint64_t *__restrict__ pivot, float *__restrict__ pdiam,
    uint16_t *__restrict__ aw, bool app_piv) {
    extern __shared__ uint64_t sB[];
    const uint64_t *B = stage_binomial(gB, n, P + 2, sB, smem_table);
    const float t = st->t;
    const uint64_t ncols = count_of(d_ncols, ncols_cap);
    // candidate vertices a sequential scan examines before its exit (the
    // algorithmic count, independent of the lanes' and blocks' over-reads)
    unsigned long long scanned = 0;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, gl = lane % G;
    const unsigned gmask = (G == 32) ? FULL_MASK : (((1u << G) - 1u) << (grp * G));
    const uint64_t ngroups = ((uint64_t)gridDim.x * blockDim.x) / G;
    uint64_t c = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;

    bool have = false;
    int v[P + 1];
    const float *row[P + 1];
    uint64_t cidx = 0;  // the column's simplex index
    float diam = 0.0f, best_d = 0.0f;
    int scan = 0, best_v = -1;

    for (;;) {
        if (!have) {
            while (c < ncols && status[c] == COL_CLEARED) c += ngroups;
            if (c < ncols) {
                have = true;
                diam = __uint_as_float(~key_hi[c]);
                cidx = key_lo[c];
                decode_simplex<P>(cidx, B, n, v);
#pragma unroll
                for (int i = 0; i <= P; ++i) row[i] = D + (int64_t)v[i] * ld;
                scan = (int)n - 1;
                best_d = INF_F;
                best_v = -1;
            }
        }
        if (!__any_sync(FULL_MASK, have)) break;

        // U blocks of G candidates per step: lane gl tests scan - gl - u G
        bool ok[U];
        float dv[U][P + 1];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ok[u] = false;
            const int x = scan - gl - u * G;
            if (have && x >= 0) {
                bool member = false;
#pragma unroll
                for (int i = 0; i <= P; ++i) member |= (x == v[i]);
                // x <= n - 1: a vertex of sigma is read too (in bounds) and
                // then excluded by an infinite m
                float m = dv[u][0] = row[0][x];
#pragma unroll
                for (int i = 1; i <= P; ++i) {
                    dv[u][i] = row[i][x];
                    m = fmaxf(m, dv[u][i]);
                }
                if (member) m = INF_F;
                ok[u] = m <= diam;
                // the oldest cofacet if no candidate qualifies: then every m
                // exceeds diam and is the cofacet's diameter, so the smallest
                // m (the largest vertex among equals: the scan descends) is
                // it; the threshold is applied once, at the end
                if (m < best_d) {
                    best_d = m;
                    best_v = x;
                }
            }
        }
        unsigned gb[U];
#pragma unroll
        for (int u = 0; u < U; ++u) gb[u] = (__ballot_sync(FULL_MASK, ok[u]) & gmask) >> (grp * G);
        if (have) {
            int first = -1, fu = 0;  // the largest qualifying vertex: first block, lowest lane
#pragma unroll
            for (int u = U - 1; u >= 0; --u)
                if (gb[u]) {
                    first = __ffs(gb[u]) - 1;
                    fu = u;
                }
            if (first >= 0) {
                if (gl == first) {
                    const int x = scan - gl - fu * G;
                    float dx[P + 1];
#pragma unroll
                    for (int i = 0; i <= P; ++i) {
                        dx[i] = dv[0][i];
#pragma unroll
                        for (int u = 1; u < U; ++u)
                            if (fu == u) dx[i] = dv[u][i];
                    }
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
                                    if (a != i && b != i)
                                        fd = fmaxf(fd, row[a][v[b]]);
                            if (fd == diam) apparent = false;
                        }
                    }
                    status[c] = apparent ? COL_APPARENT : COL_LEFTOVER;
                    if (!apparent || app_piv) {  // see launch_apparent
                        pivot[c] = cofacet_index<P>(v, x, B, n);
                        pdiam[c] = diam;
                    }
                    if (P == 1 && aw && apparent) aw[cidx] = (uint16_t)x;
                    int above = 0;  // vertices of sigma above x
#pragma unroll
                    for (int i = 0; i <= P; ++i) above += v[i] > x;
                    scanned += (unsigned long long)(n - x - above);
                }
                have = false;
                c += ngroups;
            } else if (scan - U * G < 0) {
                // every vertex seen, none of equal diameter: reduce the oldest cofacet
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
                    const bool inside = best_v >= 0 && best_d <= t;
                    status[c] = COL_LEFTOVER;
                    pivot[c] = inside ? cofacet_index<P>(v, best_v, B, n) : NO_PIVOT;
                    pdiam[c] = inside ? best_d : INF_F;
                    scanned += (unsigned long long)(n - (P + 1));
                }
                have = false;
                c += ngroups;
            } else {
                scan -= U * G;
            }
        }
    }
    // one atomic per warp for the work counter
    unsigned long long w = scanned;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(FULL_MASK, w, o);
    if (lane == 0 && w) atomicAdd(&st->scanned, w);
}

// The same test with vectorised reads: a group of G lanes scans windows of
// 4 G consecutive candidates, lane l reading the four candidates
// x0 + 4 (G - 1 - l) .. + 3 of every row of sigma as one aligned float4
// (rows start on 128-byte boundaries and hold ld = n rounded up to 32 floats,
// so a window never leaves its row). The group reads 16 G contiguous bytes of
// each row per window and U windows per step, every load in flight before any
// test. The largest qualifying candidate is the first lane of the ballot with
// a hit, and the largest of that lane's hits; the rest is the scalar kernel's.
template <int P, int G, int U>
__global__ void __launch_bounds__(256, 4) k_apparent_vec(
    const float *__restrict__ D, int64_t ld, int64_t n, const uint64_t *__restrict__ gB,
    bool smem_table, const uint32_t *__restrict__ key_hi, const uint64_t *__restrict__ key_lo,
    uint64_t ncols_cap, const unsigned long long *d_ncols, DevState *__restrict__ st,
    uint8_t *__restrict__ status, uint64_t *__restrict__ pivot, float *__restrict__ pdiam,
    uint16_t *__restrict__ aw, bool app_piv) {
    static_assert(4 * G <= 32, "a window must stay inside the 32-float row padding");
    extern __shared__ uint64_t sB[];
    const uint64_t *B = stage_binomial(gB, n, P + 2, sB, smem_table);
    const float t = st->t;
    const uint64_t ncols = count_of(d_ncols, ncols_cap);
    constexpr int W = 4 * G;  // candidates per window
    const int x_top = (int)(((n - 1) / W) * W);  // a column's first window
    unsigned long long scanned = 0;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, gl = lane % G;
    const unsigned gmask = (G == 32) ? FULL_MASK : (((1u << G) - 1u) << (grp * G));
    const uint64_t ngroups = ((uint64_t)gridDim.x * blockDim.x) / G;
    uint64_t c = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;

    bool have = false;
    int v[P + 1];
    const float *row[P + 1];
    uint64_t cidx = 0;  // the column's simplex index
    float diam = 0.0f, best_d = 0.0f;
    int x0 = 0, best_v = -1;  // x0: lowest candidate of the current step's first window

    for (;;) {
        if (!have) {
            while (c < ncols && status[c] == COL_CLEARED) c += ngroups;
            if (c < ncols) {
                have = true;
                diam = __uint_as_float(~key_hi[c]);
                cidx = key_lo[c];
                decode_simplex<P>(cidx, B, n, v);
#pragma unroll
                for (int i = 0; i <= P; ++i) row[i] = D + (int64_t)v[i] * ld;
                x0 = x_top;
                best_d = INF_F;
                best_v = -1;
            }
        }
        if (!__any_sync(FULL_MASK, have)) break;

        float4 f[U][P + 1];
        int xb[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            xb[u] = x0 - u * W + 4 * (G - 1 - gl);  // this lane's lowest candidate
            if (have && xb[u] >= 0) {
#pragma unroll
                for (int i = 0; i <= P; ++i)
                    f[u][i] = __ldg(reinterpret_cast<const float4 *>(row[i] + xb[u]));
            }
        }
        unsigned hit[U];  // bit k: candidate xb + k qualifies
#pragma unroll
        for (int u = 0; u < U; ++u) {
            hit[u] = 0;
            if (have && xb[u] >= 0) {
                // bit k set: xb + k is no candidate (the row padding past n - 1,
                // or a vertex of sigma), one mask per window
                const int lim = (int)n - xb[u];
                unsigned skip = lim >= 4 ? 0u : (lim <= 0 ? 0xfu : (0xfu << lim) & 0xfu);
#pragma unroll
                for (int i = 0; i <= P; ++i) {
                    const unsigned d = (unsigned)(v[i] - xb[u]);
                    if (d < 4u) skip |= 1u << d;
                }
#pragma unroll
                for (int k = 3; k >= 0; --k) {
                    float m = 0.0f;
#pragma unroll
                    for (int i = 0; i <= P; ++i) {
                        const float e = k == 0 ? f[u][i].x : k == 1 ? f[u][i].y
                                                   : k == 2 ? f[u][i].z : f[u][i].w;
                        m = i == 0 ? e : fmaxf(m, e);
                    }
                    if ((skip >> k) & 1u) m = INF_F;
                    if (m <= diam) hit[u] |= 1u << k;
                    // the oldest cofacet if no candidate qualifies (as in k_apparent)
                    if (m < best_d) {
                        best_d = m;
                        best_v = xb[u] + k;
                    }
                }
            }
        }
        unsigned gb[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            gb[u] = (__ballot_sync(FULL_MASK, hit[u] != 0) & gmask) >> (grp * G);
        if (have) {
            int first = -1, fu = 0;  // first window with a hit, its lowest lane
#pragma unroll
            for (int u = U - 1; u >= 0; --u)
                if (gb[u]) {
                    first = __ffs(gb[u]) - 1;
                    fu = u;
                }
            if (first >= 0) {
                if (gl == first) {
                    unsigned h = hit[0];
                    float4 fx[P + 1];
#pragma unroll
                    for (int i = 0; i <= P; ++i) fx[i] = f[0][i];
                    int xl = xb[0];
#pragma unroll
                    for (int u = 1; u < U; ++u)
                        if (fu == u) {
                            h = hit[u];
                            xl = xb[u];
#pragma unroll
                            for (int i = 0; i <= P; ++i) fx[i] = f[u][i];
                        }
                    const int k = 31 - __clz(h);  // the largest qualifying candidate
                    const int x = xl + k;
                    float dx[P + 1];
#pragma unroll
                    for (int i = 0; i <= P; ++i)
                        dx[i] = k == 0 ? fx[i].x : k == 1 ? fx[i].y : k == 2 ? fx[i].z : fx[i].w;
                    bool apparent = true;
#pragma unroll
                    for (int i = 0; i <= P; ++i) {
                        if (v[i] > x) {  // facet tau - {v_i} precedes sigma
                            float fd = 0.0f;
#pragma unroll
                            for (int kk = 0; kk <= P; ++kk)
                                if (kk != i) fd = fmaxf(fd, dx[kk]);
#pragma unroll
                            for (int a = 0; a <= P; ++a)
#pragma unroll
                                for (int b = a + 1; b <= P; ++b)
                                    if (a != i && b != i) fd = fmaxf(fd, row[a][v[b]]);
                            if (fd == diam) apparent = false;
                        }
                    }
                    status[c] = apparent ? COL_APPARENT : COL_LEFTOVER;
                    if (!apparent || app_piv) {  // see launch_apparent
                        pivot[c] = cofacet_index<P>(v, x, B, n);
                        pdiam[c] = diam;
                    }
                    if (P == 1 && aw && apparent) aw[cidx] = (uint16_t)x;
                    int above = 0;  // vertices of sigma above x
#pragma unroll
                    for (int i = 0; i <= P; ++i) above += v[i] > x;
                    scanned += (unsigned long long)(n - x - above);
                }
                have = false;
                c += ngroups;
            } else if (x0 - U * W < 0) {
                // every vertex seen, none of equal diameter: reduce the oldest cofacet
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
                    const bool inside = best_v >= 0 && best_d <= t;
                    status[c] = COL_LEFTOVER;
                    pivot[c] = inside ? cofacet_index<P>(v, best_v, B, n) : NO_PIVOT;
                    pdiam[c] = inside ? best_d : INF_F;
                    scanned += (unsigned long long)(n - (P + 1));
                }
                have = false;
                c += ngroups;
            } else {
                x0 -= U * W;
            }
        }
    }
    unsigned long long w = scanned;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(FULL_MASK, w, o);
    if (lane == 0 && w) atomicAdd(&st->scanned, w);
}

__global__ void __launch_bounds__(256) k_partition(
    const uint8_t *__restrict__ status, const uint32_t *__restrict__ key_hi,
    const uint64_t *__restrict__ key_lo, const uint64_t *__restrict__ pivot,
    const float *__restrict__ pdiam, uint64_t ncols_cap, const unsigned long long *d_ncols,
    uint64_t *__restrict__ app_tau, uint64_t *__restrict__ app_sigma, Leftover *__restrict__ left,
    DevState *st) {
    const int lane = threadIdx.x & 31;
    const uint64_t ncols = count_of(d_ncols, ncols_cap);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < ncols;
         base += stride) {
        const uint64_t c = base + lane;
        const uint8_t s = c < ncols ? status[c] : (uint8_t)COL_CLEARED;
        const bool a = s == COL_APPARENT, l = s == COL_LEFTOVER;
        const unsigned ba = __ballot_sync(FULL_MASK, a), bl = __ballot_sync(FULL_MASK, l);
        if (ba) {
            unsigned long long off = 0;
            if (lane == 0) off = atomicAdd(&st->napp, (unsigned long long)__popc(ba));
            off = __shfl_sync(FULL_MASK, off, 0);
            if (a && app_tau) {  // no pair arrays: the apparent pairs are only counted
                const uint64_t pos = off + __popc(ba & lanemask_lt());
                app_tau[pos] = pivot[c];
                app_sigma[pos] = key_lo[c];
            }
        }
        if (bl) {
            unsigned long long off = 0;
            if (lane == 0) off = atomicAdd(&st->nleft, (unsigned long long)__popc(bl));
            off = __shfl_sync(FULL_MASK, off, 0);
            if (l) {
                const uint64_t pos = off + __popc(bl & lanemask_lt());
                Leftover L;
                L.sigma = key_lo[c];
                L.pivot = pivot[c];
                L.diam = __uint_as_float(~key_hi[c]);
                L.pdiam = pdiam[c];
                L.index = c;
                left[pos] = L;
            }
        }
    }
}

template <int P, int G, int U>
void apparent_pg(const float *D, int64_t ld, int64_t n, const uint64_t *binom,
                 const uint32_t *key_hi, const uint64_t *key_lo, uint64_t ncols,
                 const unsigned long long *d_ncols, DevState *st, uint8_t *status,
                 uint64_t *pivot, float *pdiam, uint16_t *aw, bool app_piv, int sms,
                  cudaStream_t s) {
    const size_t table = (size_t)(P + 3) * (n + 1) * sizeof(uint64_t);
    const bool smem = table <= 48 * 1024;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apparent<P, G, U>, 256,
                                                  smem ? table : 0);
    if (per_sm < 1) per_sm = 1;
    uint64_t blocks = (uint64_t)sms * per_sm;
    const uint64_t need = (ncols * G + 255) / 256;
    if (need < blocks) blocks = need;
    if (blocks == 0) return;
    ++g_launches;
    k_apparent<P, G, U><<<(unsigned)blocks, 256, smem ? table : 0, s>>>(
        D, ld, n, binom, smem, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw,
        app_piv);
}

template <int P, int G, int U>
void apparent_vec(const float *D, int64_t ld, int64_t n, const uint64_t *binom,
                  const uint32_t *key_hi, const uint64_t *key_lo, uint64_t ncols,
                  const unsigned long long *d_ncols, DevState *st, uint8_t *status,
                  uint64_t *pivot, float *pdiam, uint16_t *aw, bool app_piv, int sms,
                  cudaStream_t s) {
    const size_t table = (size_t)(P + 3) * (n + 1) * sizeof(uint64_t);
    const bool smem = table <= 48 * 1024;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apparent_vec<P, G, U>, 256,
                                                  smem ? table : 0);
    if (per_sm < 1) per_sm = 1;
    uint64_t blocks = (uint64_t)sms * per_sm;
    const uint64_t need = (ncols * G + 255) / 256;
    if (need < blocks) blocks = need;
    if (blocks == 0) return;
    ++g_launches;
    k_apparent_vec<P, G, U><<<(unsigned)blocks, 256, smem ? table : 0, s>>>(
        D, ld, n, binom, smem, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw,
        app_piv);
}

// group: lanes per column G (4, 8, 16, 32) for one candidate block per step,
// or 10 G + U for U blocks (42, 44, 82); 100 + 10 G + U for the vectorised
// test with U windows of 4 G candidates a step (121, 122, 141-144, 181).
template <int P>
void apparent_p(int group, const float *D, int64_t ld, int64_t n, const uint64_t *binom,
                const uint32_t *key_hi, const uint64_t *key_lo, uint64_t ncols,
                const unsigned long long *d_ncols, DevState *st, uint8_t *status,
                uint64_t *pivot, float *pdiam, uint16_t *aw, bool app_piv, int sms,
                  cudaStream_t s) {
    switch (group) {
        case 4: apparent_pg<P, 4, 1>(D, ld, n, binom, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw, app_piv, sms, s); break;
        case 16: apparent_pg<P, 16, 1>(D, ld, n, binom, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw, app_piv, sms, s); break;
        case 32: apparent_pg<P, 32, 1>(D, ld, n, binom, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw, app_piv, sms, s); break;
        case 42: apparent_pg<P, 4, 2>(D, ld, n, binom, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw, app_piv, sms, s); break;
        case 82: apparent_pg<P, 8, 2>(D, ld, n, binom, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw, app_piv, sms, s); break;
        case 44: apparent_pg<P, 4, 4>(D, ld, n, binom, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw, app_piv, sms, s); break;
        case 121: apparent_vec<P, 2, 1>(D, ld, n, binom, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw, app_piv, sms, s); break;
        case 141: apparent_vec<P, 4, 1>(D, ld, n, binom, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw, app_piv, sms, s); break;
        case 142: apparent_vec<P, 4, 2>(D, ld, n, binom, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw, app_piv, sms, s); break;
        case 181: apparent_vec<P, 8, 1>(D, ld, n, binom, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw, app_piv, sms, s); break;
        case 143: apparent_vec<P, 4, 3>(D, ld, n, binom, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw, app_piv, sms, s); break;
        case 144: apparent_vec<P, 4, 4>(D, ld, n, binom, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw, app_piv, sms, s); break;
        case 122: apparent_vec<P, 2, 2>(D, ld, n, binom, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw, app_piv, sms, s); break;
        default: apparent_pg<P, 8, 1>(D, ld, n, binom, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw, app_piv, sms, s); break;
    }
}

}  // namespace

void launch_apparent(const float *D, int64_t ld, int64_t n, int p, const uint64_t *binom,
                     const uint32_t *key_hi, const uint64_t *key_lo, uint64_t ncols,
                     const unsigned long long *d_ncols, DevState *st, uint8_t *status,
                     uint64_t *pivot, float *pdiam, uint16_t *aw, int group, int sms,
                     cudaStream_t s, bool app_piv) {
    if (ncols == 0) return;
    switch (p) {
        case 1: apparent_p<1>(group, D, ld, n, binom, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw, app_piv, sms, s); break;
        case 2: apparent_p<2>(group, D, ld, n, binom, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw, app_piv, sms, s); break;
        case 3: apparent_p<3>(group, D, ld, n, binom, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw, app_piv, sms, s); break;
        case 4: apparent_p<4>(group, D, ld, n, binom, key_hi, key_lo, ncols, d_ncols, st, status, pivot, pdiam, aw, app_piv, sms, s); break;
        default: break;
    }
}

void launch_partition(const uint8_t *status, const uint32_t *key_hi, const uint64_t *key_lo,
                      const uint64_t *pivot, const float *pdiam, uint64_t ncols,
                      const unsigned long long *d_ncols, uint64_t *app_tau,
                      uint64_t *app_sigma, Leftover *left, DevState *st, cudaStream_t s) {
    if (ncols == 0) return;
    uint64_t blocks = (ncols + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    ++g_launches;
    k_partition<<<(unsigned)blocks, 256, 0, s>>>(status, key_hi, key_lo, pivot, pdiam, ncols,
                                                  d_ncols, app_tau, app_sigma, left, st);
}

}  // namespace rpp
