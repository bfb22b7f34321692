// batch.cu -- the fused pass for batches of small clouds (dimensions 0 and 1).
//
// One block owns one cloud at a time (clouds are handed out largest first
// through an atomic counter, so the blocks stay busy until the end) and runs,
// without leaving the block:
//   1. the distance matrix with the library's fixed float32 formula (the same
//      operations as distance.cu, so every diameter is bit-identical to the
//      single-instance path), into the cloud's slot of a scratch buffer that
//      stays in L2;
//   2. the enclosing radius R = min_x max_y d(x, y) (Sec. "Filtering Out
//      Simplices by Diameter Equal to the Enclosing Radius") and the threshold
//      t = min(t_user, R), or min(R, the nearest-rank distance quantile) found
//      by a four-pass radix select over the C(n, 2) distances;
//   3. H0: the minimum spanning forest of the edges inside t by Boruvka's
//      algorithm under the filtration's total order of edges (diameter, then
//      larger index first). The order is strict, so the forest is the one that
//      Kruskal's algorithm builds (Sec. "Zero-Dimensional Persistence
//      Computation"); its edges are the H0 deaths and the dimension-1 columns
//      removed by the clearing lemma;
//   4. the apparent-pair test (Alg. 3, Apparent Pairs Lemma) of every other
//      edge inside t with the lane-group scan of apparent.cu; leftover columns
//      go to a global pool through warp-aggregated atomics.
// Apparent pairs are only counted: the host reduction recognises an apparent
// pivot by testing its youngest facet again, so no pair store leaves the GPU.
#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace rpp {

namespace {

constexpr int SMEM_POINTS = 8192;  // points staged in shared memory up to this many floats
constexpr uint32_t EDGE_CHUNK = 32;  // consecutive edges a lane group takes in the apparent test

__device__ __forceinline__ uint64_t edge_cidx(int a, int b) {  // a > b
    return (uint64_t)a * (uint64_t)(a - 1) / 2 + (uint64_t)b;
}

__device__ __forceinline__ uint64_t tri_cidx(int a, int b, int c) {  // a > b > c
    return (uint64_t)a * (uint64_t)(a - 1) * (uint64_t)(a - 2) / 6 +
           (uint64_t)b * (uint64_t)(b - 1) / 2 + (uint64_t)c;
}

// Edge (a, b), a > b, of index e.
__device__ __forceinline__ void edge_decode(uint32_t e, int *a, int *b) {
    int x = (int)((1.0f + sqrtf(8.0f * (float)e + 1.0f)) * 0.5f);
    while ((uint32_t)x * (uint32_t)(x - 1) / 2 > e) --x;
    while ((uint32_t)(x + 1) * (uint32_t)x / 2 <= e) ++x;
    *a = x;
    *b = (int)(e - (uint32_t)x * (uint32_t)(x - 1) / 2);
}

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t w = __shfl_xor_sync(FULL_MASK, v, o);
        v = w < v ? w : v;
    }
    return v;
}

__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL_MASK, v, o));
    return v;
}

// Dynamic shared memory of the fused kernel.
struct BatchSmem {
    uint64_t *best;   // [nmax] lightest outgoing edge key per component root
    int32_t *comp;    // [nmax] component root of each vertex
    int32_t *parent;  // [nmax] hooking of the roots in one Boruvka round
    int32_t *nxt;     // [nmax] new roots
    uint32_t *mst;    // [p2] MST edge indices, sorted
    uint32_t *hist;   // [256]
    float *X;         // staged points (or null)
    uint32_t *cleared;  // [C(nmax,2) / 32] forest edges as bits (null above CLEARED_BITS_NMAX)
};

// Buckets up to this many points keep the forest's edges as a bitmap in
// shared memory (16 KB at 512 points); larger ones search the sorted list.
constexpr int CLEARED_BITS_NMAX = 512;

__host__ __device__ inline size_t cleared_words(int nmax) {
    return nmax <= CLEARED_BITS_NMAX ? ((size_t)nmax * (nmax - 1) / 2 + 31) / 32 : 0;
}

__host__ __device__ inline int pow2_at_least(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

__host__ __device__ inline size_t batch_smem_bytes(int nmax, int points_floats) {
    const int p2 = pow2_at_least(nmax);
    size_t b = (size_t)nmax * 8 + 3 * (size_t)nmax * 4 + (size_t)p2 * 4 + 256 * 4;
    if (points_floats <= SMEM_POINTS) b += (size_t)points_floats * 4;
    return b + cleared_words(nmax) * 4;
}

template <int G, int U>
__global__ void __launch_bounds__(1024) k_batch_h1(
    const float *__restrict__ pts, const BatchCloud *__restrict__ clouds,
    const int32_t *__restrict__ order, BatchCtl *ctl, int nmax, int points_floats,
    float *__restrict__ Dbuf, uint64_t *__restrict__ mst_out, BatchOut *__restrict__ outs,
    Leftover *__restrict__ left, int32_t *__restrict__ left_cloud, uint64_t left_cap,
    uint16_t *__restrict__ app_w) {
    const int nclouds = ctl->nclouds;
    unsigned int *queue = &ctl->queue;
    unsigned long long *left_count = &ctl->left_count;
    extern __shared__ uint64_t smem_raw[];
    BatchSmem S;
    {
        char *p = (char *)smem_raw;
        const int p2 = pow2_at_least(nmax);
        S.best = (uint64_t *)p;
        p += (size_t)nmax * 8;
        S.comp = (int32_t *)p;
        p += (size_t)nmax * 4;
        S.parent = (int32_t *)p;
        p += (size_t)nmax * 4;
        S.nxt = (int32_t *)p;
        p += (size_t)nmax * 4;
        S.mst = (uint32_t *)p;
        p += (size_t)p2 * 4;
        S.hist = (uint32_t *)p;
        p += 256 * 4;
        S.X = points_floats <= SMEM_POINTS ? (float *)p : nullptr;
        if (S.X) p += (size_t)points_floats * 4;
        S.cleared = cleared_words(nmax) ? (uint32_t *)p : nullptr;
    }
    __shared__ int s_cloud;
    __shared__ unsigned int s_rbits, s_err, s_nm, s_changed, s_digit, s_rank;
    __shared__ unsigned long long s_ncols, s_napp, s_nleft, s_scanned;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned int q = atomicAdd(queue, 1u);
            s_cloud = q < (unsigned)nclouds ? order[q] : -1;
            s_rbits = 0x7f800000u;  // +inf
            s_err = 0;
            s_nm = 0;
            s_ncols = s_napp = s_nleft = s_scanned = 0;
        }
        __syncthreads();
        const int ci = s_cloud;
        if (ci < 0) return;
        const BatchCloud C = clouds[ci];
        const int n = C.n, dim = C.dim;
        const int64_t ld = C.ld;
        float *D = Dbuf + C.d_off;
        const float *Xg = pts + C.pt_off;

        // ---- 1. distances, enclosing radius ----
        const float *X = Xg;
        if (S.X && n * dim <= SMEM_POINTS) {
            for (int i = threadIdx.x; i < n * dim; i += blockDim.x) S.X[i] = Xg[i];
            X = S.X;
        }
        __syncthreads();
        for (int r = warp; r < n; r += nwarps) {
            float rmax = 0.0f;
            bool bad = false;
            for (int c = lane; c < n; c += 32) {
                float s = 0.0f;
                for (int k = 0; k < dim; ++k) {
                    const float d = __fsub_rn(X[r * dim + k], X[c * dim + k]);
                    s = __fadd_rn(s, __fmul_rn(d, d));
                }
                const float v = __fsqrt_rn(s);
                D[r * ld + c] = v;
                bad |= !(v <= 3.402823466e38f);
                rmax = fmaxf(rmax, v);
            }
            rmax = warp_max_f(rmax);
            bad = __any_sync(FULL_MASK, bad);
            if (lane == 0) {
                atomicMin(&s_rbits, __float_as_uint(rmax));
                if (bad) atomicOr(&s_err, (unsigned)ERR_NONFINITE);
            }
        }
        __syncthreads();
        const float R = __uint_as_float(s_rbits);
        float t = fminf(C.t_user, R);
        const uint32_t m = (uint32_t)n * (uint32_t)(n - 1) / 2;

        // ---- 2. nearest-rank quantile: radix select over the C(n, 2) distances ----
        if (C.qrank > 0 && m > 0 && s_err == 0) {
            uint64_t rk = C.qrank;
            rk = rk < 1 ? 1 : (rk > m ? m : rk);
            uint32_t prefix = 0, mask = 0, rank = (uint32_t)rk;
            for (int shift = 24; shift >= 0; shift -= 8) {
                for (int i = threadIdx.x; i < 256; i += blockDim.x) S.hist[i] = 0;
                __syncthreads();
                for (int a = 1 + warp; a < n; a += nwarps)
                    for (int b = lane; b < a; b += 32) {
                        const uint32_t v = __float_as_uint(D[a * ld + b]);
                        if ((v & mask) == prefix) atomicAdd(&S.hist[(v >> shift) & 255u], 1u);
                    }
                __syncthreads();
                if (warp == 0) {  // first digit whose running count reaches the rank
                    uint32_t h[8], run = 0;
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        h[k] = S.hist[lane * 8 + k];
                        run += h[k];
                    }
                    uint32_t incl = run;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(FULL_MASK, incl, o);
                        if (lane >= o) incl += y;
                    }
                    const uint32_t excl = incl - run;
                    if (excl < rank && rank <= incl) {
                        uint32_t acc = excl;
                        for (int k = 0; k < 8; ++k) {
                            if (rank <= acc + h[k]) {
                                s_digit = (uint32_t)(lane * 8 + k);
                                s_rank = rank - acc;
                                break;
                            }
                            acc += h[k];
                        }
                    }
                }
                __syncthreads();
                prefix |= s_digit << shift;
                mask |= 255u << shift;
                rank = s_rank;
            }
            t = fminf(R, __uint_as_float(prefix));
        }

        // edges inside t (the dimension-1 columns before clearing)
        {
            unsigned long long cnt = 0;
            for (int a = 1 + warp; a < n; a += nwarps)
                for (int b = lane; b < a; b += 32) cnt += D[a * ld + b] <= t;
            if (cnt) atomicAdd(&s_ncols, cnt);
        }

        // ---- 3. H0: minimum spanning forest inside t (Boruvka) ----
        for (int v = threadIdx.x; v < n; v += blockDim.x) S.comp[v] = v;
        __syncthreads();
        for (int round = 0; round < 64 && s_err == 0; ++round) {
            for (int v = threadIdx.x; v < n; v += blockDim.x) S.best[v] = ~0ull;
            if (threadIdx.x == 0) s_changed = 0;
            __syncthreads();
            for (int u = warp; u < n; u += nwarps) {
                const int cu = S.comp[u];
                uint64_t bk = ~0ull;
                for (int w0 = lane; w0 < n; w0 += 4 * 32) {
                    // four entries a lane, their loads issued before any test
                    float d[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int w = w0 + 32 * i;
                        d[i] = w < n ? D[u * ld + w] : 0.0f;
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int w = w0 + 32 * i;
                        if (w >= n || w == u || S.comp[w] == cu || d[i] > t) continue;
                        const uint32_t e = (uint32_t)(u > w ? edge_cidx(u, w) : edge_cidx(w, u));
                        const uint64_t key =
                            ((uint64_t)__float_as_uint(d[i]) << 32) | (uint64_t)(~e);
                        bk = key < bk ? key : bk;
                    }
                }
                bk = warp_min_u64(bk);
                if (lane == 0 && bk != ~0ull) atomicMin((unsigned long long *)&S.best[cu], bk);
            }
            __syncthreads();
            for (int c = threadIdx.x; c < n; c += blockDim.x) {
                if (S.comp[c] != c) continue;
                S.parent[c] = c;
                const uint64_t bk = S.best[c];
                if (bk == ~0ull) continue;
                const uint32_t e = ~(uint32_t)bk;
                int a, b;
                edge_decode(e, &a, &b);
                const int ca = S.comp[a], cb = S.comp[b];
                const int o = ca == c ? cb : ca;
                const bool mutual = S.best[o] == bk;
                if (!(mutual && c < o)) S.parent[c] = o;
                if (!(mutual && c > o)) {  // each forest edge recorded once
                    const unsigned k = atomicAdd(&s_nm, 1u);
                    mst_out[C.mst_off + k] = (bk & 0xffffffff00000000ull) | (uint64_t)e;
                    S.mst[k] = e;
                }
                s_changed = 1;
            }
            __syncthreads();
            if (!s_changed) break;
            for (int v = threadIdx.x; v < n; v += blockDim.x) {
                // the hooking is a forest (keys are unique, mutual picks keep
                // the smaller root), so a root is at most n - 1 hops away
                int r = S.comp[v], hops = 0;
                while (S.parent[r] != r && hops < n) {
                    r = S.parent[r];
                    ++hops;
                }
                if (S.parent[r] != r) atomicOr(&s_err, (unsigned)ERR_INTERNAL);
                S.nxt[v] = r;
            }
            __syncthreads();
            for (int v = threadIdx.x; v < n; v += blockDim.x) S.comp[v] = S.nxt[v];
            __syncthreads();
        }
        // sort the forest's edge indices (bitonic, padded to a power of two)
        const int nm = (int)s_nm;
        const int p2 = pow2_at_least(nm > 0 ? nm : 1);
        for (int i = nm + threadIdx.x; i < p2; i += blockDim.x) S.mst[i] = 0xffffffffu;
        __syncthreads();
        for (int k = 2; k <= p2; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < p2; i += blockDim.x) {
                    const int l = i ^ j;
                    if (l > i) {
                        const uint32_t a = S.mst[i], b = S.mst[l];
                        if ((a > b) == ((i & k) == 0)) {
                            S.mst[i] = b;
                            S.mst[l] = a;
                        }
                    }
                }
                __syncthreads();
            }
        if (S.cleared) {  // the forest's edges as bits: one lookup per column
            for (uint32_t i = threadIdx.x; i < (m + 31) / 32; i += blockDim.x) S.cleared[i] = 0u;
            __syncthreads();
            for (int i = threadIdx.x; i < nm; i += blockDim.x)
                atomicOr(&S.cleared[S.mst[i] >> 5], 1u << (S.mst[i] & 31));
            __syncthreads();
        }

        // ---- 4. apparent-pair test of the other edges inside t ----
        if (s_err == 0 && C.max_dim >= 1) {
            const int gl = lane % G, grp = lane / G;
            const unsigned gmask = (G == 32) ? FULL_MASK : (((1u << G) - 1u) << (grp * G));
            const uint32_t ngroups = blockDim.x / G;
            // a group's edges: chunks of EDGE_CHUNK consecutive indices (chunk
            // g, g + ngroups, ...), walked with (u, w) updated in place, so
            // an edge is decoded once per chunk and its row is read in order
            uint32_t e = (threadIdx.x / G) * EDGE_CHUNK;
            int u = 0, w = 0;
            if (e < m) edge_decode(e, &u, &w);
            auto advance = [&]() {
                ++e;
                if ((e & (EDGE_CHUNK - 1)) == 0) {
                    e += (ngroups - 1) * EDGE_CHUNK;
                    if (e < m) edge_decode(e, &u, &w);
                } else if (++w == u) {
                    ++u;
                    w = 0;
                }
            };
            unsigned long long napp = 0, nleft = 0, scanned = 0;
            bool have = false;
            int scan = 0, best_v = -1;
            float diam = 0.0f, best_d = 0.0f;
            uint16_t *aw = app_w + C.aw_off;
            for (;;) {
                while (!have && e < m) {
                    diam = D[u * ld + w];
                    if (diam <= t) {
                        bool cleared;  // a forest (cleared) column?
                        if (S.cleared) {
                            cleared = (S.cleared[e >> 5] >> (e & 31)) & 1u;
                        } else {
                            int lo = 0, hi = nm;
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if (S.mst[mid] < e) lo = mid + 1;
                                else hi = mid;
                            }
                            cleared = lo < nm && S.mst[lo] == e;
                        }
                        if (cleared) {
                            if (gl == 0) aw[e] = 0xFFFFu;
                            advance();
                            continue;
                        }
                        have = true;
                        scan = n - 1;
                        best_d = __uint_as_float(0x7f800000u);
                        best_v = -1;
                    } else {
                        if (gl == 0) aw[e] = 0xFFFFu;
                        advance();
                    }
                }
                if (!__any_sync(FULL_MASK, have)) break;

                // U blocks of G candidates per step: lane gl tests scan - gl - j G,
                // every block's loads in flight before any test
                bool ok[U];
                float du[U], dw[U];
#pragma unroll
                for (int j = 0; j < U; ++j) {
                    ok[j] = false;
                    du[j] = dw[j] = 0.0f;
                    const int x = scan - gl - j * G;
                    if (have && x >= 0 && x != u && x != w) {
                        du[j] = D[u * ld + x];
                        dw[j] = D[w * ld + x];
                        const float mx = fmaxf(du[j], dw[j]);
                        ok[j] = mx <= diam;
                        const float cd = fmaxf(mx, diam);
                        if (cd <= t && cd < best_d) {
                            best_d = cd;
                            best_v = x;
                        }
                    }
                }
                unsigned gbs[U];
#pragma unroll
                for (int j = 0; j < U; ++j) gbs[j] = (__ballot_sync(FULL_MASK, ok[j]) & gmask) >> (grp * G);
                bool emit = false;  // this lane writes a leftover column
                Leftover L;
                if (have) {
                    int first = -1, fj = 0;  // the largest qualifying vertex
#pragma unroll
                    for (int j = U - 1; j >= 0; --j)
                        if (gbs[j]) {
                            first = __ffs(gbs[j]) - 1;
                            fj = j;
                        }
                    if (first >= 0) {
                        if (gl == first) {
                            const int x = scan - gl - fj * G;
                            float dux = du[0], dwx = dw[0];
#pragma unroll
                            for (int j = 1; j < U; ++j)
                                if (fj == j) {
                                    dux = du[j];
                                    dwx = dw[j];
                                }
                            // candidates a sequential scan examines up to x
                            scanned += (unsigned long long)(n - x - (u > x) - (w > x));
                            // facets of tau = {u, w, x} before sigma drop a vertex above x
                            bool apparent = true;
                            if (u > x && dwx == diam) apparent = false;  // facet {w, x}
                            if (w > x && dux == diam) apparent = false;  // facet {u, x}
                            aw[e] = apparent ? (uint16_t)x : (uint16_t)0xFFFFu;
                            if (apparent) {
                                ++napp;
                            } else {
                                emit = true;
                                L.sigma = edge_cidx(u, w);
                                const int a = max(u, x), c = min(w, x);
                                const int b = u + w + x - a - c;
                                L.pivot = tri_cidx(a, b, c);
                                L.pdiam = diam;
                            }
                        }
                        have = false;
                        advance();
                    } else if (scan - U * G < 0) {
                        // no cofacet of equal diameter: the oldest cofacet inside t
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
                            scanned += (unsigned long long)(n - 2);
                            emit = true;
                            L.sigma = edge_cidx(u, w);
                            aw[e] = 0xFFFFu;
                            if (best_v >= 0) {
                                const int x2 = best_v;
                                const int a = max(u, x2), c = min(w, x2);
                                const int b = u + w + x2 - a - c;
                                L.pivot = tri_cidx(a, b, c);
                            } else {
                                L.pivot = NO_PIVOT;
                            }
                            L.pdiam = best_d;
                        }
                        have = false;
                        advance();
                    } else {
                        scan -= U * G;
                    }
                }
                if (emit) {  // L.sigma was set before the group moved on
                    L.diam = diam;
                    L.index = ((uint64_t)(~__float_as_uint(diam)) << 32) | (uint64_t)L.sigma;
                }
                const unsigned be = __ballot_sync(FULL_MASK, emit);
                if (be) {
                    unsigned long long off = 0;
                    if (lane == 0) off = atomicAdd(left_count, (unsigned long long)__popc(be));
                    off = __shfl_sync(FULL_MASK, off, 0);
                    if (emit) {
                        ++nleft;
                        const uint64_t pos = off + __popc(be & lanemask_lt());
                        if (pos < left_cap) {
                            left[pos] = L;
                            left_cloud[pos] = ci;
                        }
                    }
                }
            }
            atomicAdd(&s_napp, napp);
            atomicAdd(&s_nleft, nleft);
            atomicAdd(&s_scanned, scanned);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            BatchOut o;
            o.R = R;
            o.t = t;
            o.nmst = s_nm;
            o.err = s_err;
            o.ncols = s_ncols;
            o.napp = s_napp;
            o.nleft = s_nleft;
            o.scanned = s_scanned;
            outs[ci] = o;
        }
    }
}

// Rows of the selected clouds: the distance row copied out and sorted into
// neighbour keys (bits(D[v][w]) << 32) | w, as in neighbors.cu.
__global__ void __launch_bounds__(512) k_batch_rows(const float *__restrict__ Dbuf,
                                                    const BatchCloud *__restrict__ clouds,
                                                    const int32_t *__restrict__ jobs,
                                                    const int64_t *__restrict__ out_off, int njobs,
                                                    float *__restrict__ Dout,
                                                    uint64_t *__restrict__ nbr,
                                                    const uint16_t *__restrict__ app_w,
                                                    uint16_t *__restrict__ aw_out) {
    extern __shared__ unsigned long long keys[];
    const int j = blockIdx.y;
    const BatchCloud C = clouds[jobs[j]];
    const int n = C.n, row = blockIdx.x;
    if (row >= n) return;
    {  // this row's edges {row, w}, w < row: indices C(row, 2) .. C(row, 2) + row - 1
        const int64_t e0 = (int64_t)row * (row - 1) / 2;
        const uint16_t *src = app_w + C.aw_off + e0;
        uint16_t *dst = aw_out + out_off[njobs + j] + e0;
        for (int i = threadIdx.x; i < row; i += blockDim.x) dst[i] = src[i];
    }
    const int p2 = pow2_at_least(n);
    const float *src = Dbuf + C.d_off + (int64_t)row * C.ld;
    float *drow = Dout + out_off[j] + (int64_t)row * n;
    uint64_t *nrow = nbr + out_off[j] + (int64_t)row * n;
    for (int i = threadIdx.x; i < p2; i += blockDim.x) {
        if (i < n) {
            const float v = src[i];
            drow[i] = v;
            keys[i] = ((unsigned long long)__float_as_uint(v) << 32) | (unsigned)i;
        } else {
            keys[i] = ~0ull;
        }
    }
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1)
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int i = threadIdx.x; i < p2; i += blockDim.x) {
                const int l = i ^ jj;
                if (l > i) {
                    const unsigned long long a = keys[i], b = keys[l];
                    if ((a > b) == ((i & k) == 0)) {
                        keys[i] = b;
                        keys[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < n; i += blockDim.x) nrow[i] = keys[i];
}

__global__ void k_gather_points(const float *const *__restrict__ src,
                                const BatchCloud *__restrict__ clouds, float *__restrict__ pts) {
    const BatchCloud C = clouds[blockIdx.x];
    const float *s = src[blockIdx.x];
    if (!s) return;  // a host cloud, already copied
    const int64_t cnt = (int64_t)C.n * C.dim;
    for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) pts[C.pt_off + i] = s[i];
}

template <int G, int U>
BatchPlan plan_g(int nmax, int dimcap, BatchConfig cfg, int sms) {
    BatchPlan P;
    P.nmax = nmax;
    P.dimcap = dimcap;
    P.cfg = cfg;
    P.smem = batch_smem_bytes(nmax, nmax * dimcap);
    allow_dynamic_smem((const void *)k_batch_h1<G, U>, P.smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_h1<G, U>, cfg.threads, P.smem);
    if (cfg.per_sm > 0 && cfg.per_sm < per_sm) per_sm = cfg.per_sm;
    P.blocks = std::max(1, sms * std::max(1, per_sm));
    return P;
}

template <int G, int U>
void launch_g(const BatchPlan &P, const float *pts, const BatchCloud *clouds, const int32_t *order,
              BatchCtl *ctl, float *Dbuf, uint64_t *mst_out, BatchOut *outs, Leftover *left,
              int32_t *left_cloud, uint64_t left_cap, uint16_t *app_w, cudaStream_t s) {
    ++g_launches;
    k_batch_h1<G, U><<<P.blocks, P.cfg.threads, P.smem, s>>>(pts, clouds, order, ctl, P.nmax,
                                                          P.nmax * P.dimcap, Dbuf, mst_out, outs,
                                                          left, left_cloud, left_cap, app_w);
}

}  // namespace

BatchPlan plan_batch_h1(int nmax, int dimcap, BatchConfig cfg, int sms) {
    switch (cfg.group) {  // G lanes, or 10 G + U for U candidate blocks a step
        case 4: return plan_g<4, 1>(nmax, dimcap, cfg, sms);
        case 16: return plan_g<16, 1>(nmax, dimcap, cfg, sms);
        case 32: return plan_g<32, 1>(nmax, dimcap, cfg, sms);
        case 42: return plan_g<4, 2>(nmax, dimcap, cfg, sms);
        case 44: return plan_g<4, 4>(nmax, dimcap, cfg, sms);
        case 82: return plan_g<8, 2>(nmax, dimcap, cfg, sms);
        default: cfg.group = 8; return plan_g<8, 1>(nmax, dimcap, cfg, sms);
    }
}

void launch_batch_h1(const BatchPlan &P, const float *pts, const BatchCloud *clouds,
                     const int32_t *order, BatchCtl *ctl, float *Dbuf, uint64_t *mst_out,
                     BatchOut *outs, Leftover *left, int32_t *left_cloud, uint64_t left_cap,
                     uint16_t *app_w, cudaStream_t s) {
    switch (P.cfg.group) {
        case 4: launch_g<4, 1>(P, pts, clouds, order, ctl, Dbuf, mst_out, outs, left, left_cloud, left_cap, app_w, s); break;
        case 16: launch_g<16, 1>(P, pts, clouds, order, ctl, Dbuf, mst_out, outs, left, left_cloud, left_cap, app_w, s); break;
        case 32: launch_g<32, 1>(P, pts, clouds, order, ctl, Dbuf, mst_out, outs, left, left_cloud, left_cap, app_w, s); break;
        case 42: launch_g<4, 2>(P, pts, clouds, order, ctl, Dbuf, mst_out, outs, left, left_cloud, left_cap, app_w, s); break;
        case 44: launch_g<4, 4>(P, pts, clouds, order, ctl, Dbuf, mst_out, outs, left, left_cloud, left_cap, app_w, s); break;
        case 82: launch_g<8, 2>(P, pts, clouds, order, ctl, Dbuf, mst_out, outs, left, left_cloud, left_cap, app_w, s); break;
        default: launch_g<8, 1>(P, pts, clouds, order, ctl, Dbuf, mst_out, outs, left, left_cloud, left_cap, app_w, s);
    }
}

void launch_batch_rows(const float *Dbuf, const BatchCloud *clouds, const int32_t *jobs, int njobs,
                       const int64_t *out_off, int nmax, float *Dout, uint64_t *nbr,
                       const uint16_t *app_w, uint16_t *aw_out, cudaStream_t s) {
    if (njobs <= 0) return;
    const size_t smem = (size_t)pow2_at_least(nmax) * 8;
    allow_dynamic_smem((const void *)k_batch_rows, smem);
    ++g_launches;
    k_batch_rows<<<dim3((unsigned)nmax, (unsigned)njobs), 256, smem, s>>>(
        Dbuf, clouds, jobs, out_off, njobs, Dout, nbr, app_w, aw_out);
}

void launch_gather_points(const float *const *src, const BatchCloud *clouds, int nclouds,
                          float *pts, cudaStream_t s) {
    if (nclouds <= 0) return;
    ++g_launches;
    k_gather_points<<<nclouds, 256, 0, s>>>(src, clouds, pts);
}

}  // namespace rpp
