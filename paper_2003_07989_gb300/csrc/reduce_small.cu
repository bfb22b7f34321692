// reduce_small.cu -- the submatrix reduction of dimension 1 (Alg. 1 on the
// leftover columns, Sec. "Core System Optimizations") on the device, for the
// clouds of up to 512 points of a fused batch.
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
//     earlier leftover column whose final pivot is tau (a shared-memory hash
//     from final pivots to columns); otherwise the pivot is free and the
//     column is paired with it.
//   * After an addition every entry up to and including the old pivot is
//     zero (the owner's column has that pivot and nothing older), so the next
//     pivot is the oldest nonzero triangle younger than it.
// Two ways to find that next pivot:
//   * Cursors (short walks): each edge of V keeps a lazy cursor, its oldest
//     cofacet inside the threshold that the column has not passed (a warp
//     scan of the third vertices). The smallest head is a nonzero entry when
//     an odd number of V's edges hold it (a triangle's edges in V all have it
//     as their head); an even one cancels, and those cursors move on.
//   * Level sweep (long walks, V large): the triangles themselves in age
//     order, one diameter level of edges at a time. The triangles whose
//     longest edge is {a, b} (diameter d) are {a, b, w} with w within d of a
//     and of b; with P[a] the set of vertices within the current level's
//     diameter of a, they are the bits of P[a] & P[b], and their coefficients
//     the bits of adj[a] ^ adj[b] ^ [ab in V]. A level whose edges touch no
//     edge of V holds only zero entries; the warp passes 32 edges of such
//     levels at a time. The levels come from the cloud's edges inside the
//     threshold sorted by diameter (one radix sort over every cloud that needs
//     them), and P is moved along them.
// The first phase runs every cloud with cursors only and hands a cloud whose
// column needs more than RS_BUDGET additions, or whose V grows past RS_VMAX
// edges, to the second phase; the second phase redoes those clouds and lets
// such a column continue as a level sweep. A cloud whose level holds more
// than RS_LEVMAX edges of one diameter, or whose final edge sets outgrow the
// cloud's share of the pool, goes back to the host (status 1).
#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace rpp {

namespace {

constexpr int RS_VMAX = 64;     // edges of V per column with cursors
constexpr int RS_BUDGET = 64;   // additions per column with cursors (first phase)
constexpr int RS_SWEEP_AFTER = 8;  // second phase: additions with cursors before sweeping
constexpr int RS_LEVMAX = 32;   // edges of one diameter level in the sweep
constexpr int RS_HASH = 1024;   // slots of the final-pivot -> column table
constexpr int RS_ADDS_MAX = 1 << 22;  // additions per column (a bound on the walk)
constexpr uint32_t HASH_EMPTY = 0xffffffffu;

// Sorted edge keys of the second phase: b in bits [0, 9), a in [9, 18), the
// diameter's bits in [18, 50), the job in [50, 62).
constexpr int EK_BITS = 62;
__device__ __forceinline__ uint64_t edge_key(int job, float d, int a, int b) {
    return ((uint64_t)job << 50) | ((uint64_t)__float_as_uint(d) << 18) | ((uint64_t)a << 9) |
           (uint64_t)b;
}
__device__ __forceinline__ uint32_t ek_diam(uint64_t k) { return (uint32_t)(k >> 18); }
__device__ __forceinline__ int ek_a(uint64_t k) { return (int)((k >> 9) & 511u); }
__device__ __forceinline__ int ek_b(uint64_t k) { return (int)(k & 511u); }

// Age key of a triangle: diameter bits over the complemented index; ascending
// key is the filtration order (older first: smaller diameter, then larger index).
__device__ __forceinline__ uint64_t tri_key(float d, uint32_t idx) {
    return ((uint64_t)__float_as_uint(d) << 32) | (uint64_t)(0xffffffffu - idx);
}

__device__ __forceinline__ uint32_t c3(uint32_t v) {
    return (uint32_t)((uint64_t)v * (v - 1) * (v - 2) / 6);
}
__device__ __forceinline__ uint32_t c2(uint32_t v) { return v * (v - 1) / 2; }

// Index of the triangle with vertices a, b, c (any order). For fixed a > b it
// increases with c (also through c = a or c = b, which name no triangle).
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
// above `after` (~0 if none): the warp scans the third vertices, every lane
// loading its share of both distance rows before comparing.
constexpr int RS_WPL = REDUCE_SMALL_NMAX / 32;  // third vertices per lane
__device__ uint64_t cursor_next(const float *D, int n, float t, uint32_t e, uint64_t after) {
    int xy[2];
    decode_edge((uint64_t)e, xy);
    const int x = xy[0], y = xy[1];
    const int lane = threadIdx.x & 31;
    const float dxy = D[x * n + y];
    const float *rx = D + (int64_t)x * n, *ry = D + (int64_t)y * n;
    float fx[RS_WPL], fy[RS_WPL];
#pragma unroll
    for (int i = 0; i < RS_WPL; ++i) {
        const int w = lane + 32 * i;
        fx[i] = w < n ? rx[w] : 0.0f;
        fy[i] = w < n ? ry[w] : 0.0f;
    }
    uint64_t best = ~0ull;
#pragma unroll
    for (int i = 0; i < RS_WPL; ++i) {
        const int w = lane + 32 * i;
        if (w >= n || w == x || w == y) continue;
        const float d = fmaxf(dxy, fmaxf(fx[i], fy[i]));
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

// The cloud a warp reduces, and V: an adjacency bitset (both directions of
// every edge), with each vertex's degree in V in the second phase.
struct Cloud {
    const float *D;  // row stride n
    const uint16_t *aw;
    int n, w32;
    float t;
    uint32_t *adj;   // n x w32
    int32_t *deg;    // n (second phase; nullptr in the first)
    __device__ bool in(int a, int b) const { return (adj[a * w32 + (b >> 5)] >> (b & 31)) & 1u; }
    // One lane flips the edge {x, y}.
    __device__ void flip1(int x, int y) {
        const uint32_t was = adj[x * w32 + (y >> 5)] & (1u << (y & 31));
        adj[x * w32 + (y >> 5)] ^= 1u << (y & 31);
        adj[y * w32 + (x >> 5)] ^= 1u << (x & 31);
        if (deg) {
            deg[x] += was ? -1 : 1;
            deg[y] += was ? -1 : 1;
        }
    }
    // Any number of lanes flip distinct edges at once.
    __device__ void flip_atomic(int x, int y) {
        const uint32_t was = atomicXor(&adj[x * w32 + (y >> 5)], 1u << (y & 31)) & (1u << (y & 31));
        atomicXor(&adj[y * w32 + (x >> 5)], 1u << (x & 31));
        if (deg) {
            atomicAdd(&deg[x], was ? -1 : 1);
            atomicAdd(&deg[y], was ? -1 : 1);
        }
    }
};

// V's edge list with one lazy cursor per edge (cursor mode). Lane 0 writes
// the shared arrays; every lane keeps vcount.
struct VList {
    uint32_t *edge;
    uint64_t *head;
    int vcount;
    // Toggle e in V (its bits and, when it enters, a cursor past `after`).
    // False when the list would overflow (nothing changed then).
    __device__ bool toggle(Cloud &C, uint32_t e, uint64_t after) {
        int xy[2];
        decode_edge((uint64_t)e, xy);
        const int lane = threadIdx.x & 31;
        if (C.in(xy[0], xy[1])) {  // leaves V: swap-remove
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
                C.flip1(xy[0], xy[1]);
            }
            --vcount;
        } else {
            if (vcount >= RS_VMAX) return false;
            const uint64_t h = cursor_next(C.D, C.n, C.t, e, after);
            if (lane == 0) {
                edge[vcount] = e;
                head[vcount] = h;
                C.flip1(xy[0], xy[1]);
            }
            ++vcount;
        }
        __syncwarp();
        return true;
    }
    // Every cursor at or before k moves past k.
    __device__ void pass(Cloud &C, uint64_t k) {
        for (int q = 0; q < vcount; ++q) {
            const uint64_t h = head[q];
            if (h <= k) {
                const uint64_t nh = cursor_next(C.D, C.n, C.t, edge[q], k);
                if ((threadIdx.x & 31) == 0) head[q] = nh;
                __syncwarp();
            }
        }
    }
    // The oldest nonzero entry of the working column past the cursors: the
    // smallest head held by an odd number of V's edges; even ones cancel and
    // their cursors move on. ~0 if the column is zero.
    __device__ uint64_t pivot(Cloud &C) {
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
            pass(C, m);
        }
    }
};
// The level sweep of one cloud (second phase). P holds exactly the edges at
// sorted positions below `pos`; while a column sweeps, pos == f1, the first
// position after the current level. The sorted edges are read through a
// window of 64 positions held in registers (lane l: positions wbase + l and
// wbase + 32 + l, with each edge's apparent vertex), the second half loaded
// ahead while the first is in use.
struct Sweep {
    const uint64_t *keys;  // the cloud's edges inside the threshold, by diameter
    const uint16_t *kaw;   // the apparent vertex of each of those edges
    int64_t m;
    int64_t pos, f1;
    uint32_t *P;           // n x w32
    float lvl_d;
    int levn;
    int *la, *lb, *lw;     // level edges {a > b}; triangles {a, b, w} with w < lw are to come
    uint32_t *li;          // level edges' indices
    uint16_t *law;         // level edges' apparent vertices
    int *ba, *bb;          // a batch of single-edge levels: their edges
    int pa, pb, pw, pi;    // the last pivot's triangle, {pa > pb} its level edge (number pi)
    int64_t wbase;         // window: a multiple of 32
    uint64_t k0, k1;       // keys at wbase + lane, wbase + 32 + lane (~0 past m)
    uint16_t a0, a1;

    __device__ void load_half(int64_t base, uint64_t &k, uint16_t &a) const {
        const int64_t q = base + (threadIdx.x & 31);
        k = q < m ? keys[q] : ~0ull;
        a = q < m ? kaw[q] : (uint16_t)0xffffu;
    }
    // Window covering position p.
    __device__ void window_at(int64_t p) {
        wbase = p & ~(int64_t)31;
        load_half(wbase, k0, a0);
        load_half(wbase + 32, k1, a1);
    }
    // Move the window forward so that it covers p (p >= wbase).
    __device__ void advance(int64_t p) {
        if (p >= wbase + 64) {
            window_at(p);
        } else if (p >= wbase + 32) {
            wbase += 32;
            k0 = k1;
            a0 = a1;
            load_half(wbase + 32, k1, a1);
        }
    }
    // Key and apparent vertex at p + lane (p within the window's first half).
    __device__ void fetch(int64_t p, uint64_t &k, uint16_t &a) {
        advance(p);
        const int lane = threadIdx.x & 31;
        const int off = (int)(p - wbase) + lane;  // 0 .. 62
        const uint64_t x0 = __shfl_sync(FULL_MASK, k0, off & 31);
        const uint64_t x1 = __shfl_sync(FULL_MASK, k1, off & 31);
        const uint16_t y0 = (uint16_t)__shfl_sync(FULL_MASK, (int)a0, off & 31);
        const uint16_t y1 = (uint16_t)__shfl_sync(FULL_MASK, (int)a1, off & 31);
        k = off < 32 ? x0 : x1;
        a = off < 32 ? y0 : y1;
    }

    __device__ void p_flip(Cloud &C, int a, int b) {
        atomicXor(&P[a * C.w32 + (b >> 5)], 1u << (b & 31));
        atomicXor(&P[b * C.w32 + (a >> 5)], 1u << (a & 31));
    }
    // Flip the P bits of the edges at positions [lo, hi), eight loads in
    // flight per lane.
    __device__ void p_flip_range(Cloud &C, int64_t lo, int64_t hi) {
        const int lane = threadIdx.x & 31;
        for (int64_t q0 = lo; q0 < hi; q0 += 256) {
            uint64_t k[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int64_t q = q0 + i * 32 + lane;
                k[i] = q < hi ? keys[q] : 0;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (q0 + i * 32 + lane < hi) p_flip(C, ek_a(k[i]), ek_b(k[i]));
        }
        __syncwarp();
    }
    __device__ void move_p(Cloud &C, int64_t target) {
        if (target > pos) p_flip_range(C, pos, target);
        else if (target < pos) p_flip_range(C, target, pos);
        pos = target;
    }
    // First position whose diameter's bits are >= db.
    __device__ int64_t lower_bound(uint32_t db) const {
        const int lane = threadIdx.x & 31;
        int64_t lo = 0, hi = m;
        while (hi - lo > 32) {  // 32-way steps: every lane probes one split
            const int64_t q = lo + (hi - lo) * (lane + 1) / 33;
            const bool below = ek_diam(keys[q]) < db;
            const int c = __popc(__ballot_sync(FULL_MASK, below));  // a prefix
            const int64_t nlo = c ? lo + (hi - lo) * c / 33 + 1 : lo;
            const int64_t nhi = c < 32 ? lo + (hi - lo) * (c + 1) / 33 : hi;
            lo = nlo;
            hi = nhi;
        }
        const int64_t q = lo + lane;
        const bool below = q < hi && ek_diam(keys[q]) < db;
        return lo + __popc(__ballot_sync(FULL_MASK, below));
    }
    // Enter the level of equal diameter starting at `start` (== pos): list its
    // edges and set their bits in P. False when it holds more than RS_LEVMAX.
    __device__ bool load_level(Cloud &C, int64_t start) {
        const int lane = threadIdx.x & 31;
        uint64_t k;
        uint16_t aw;
        fetch(start, k, aw);
        const uint32_t d0 = ek_diam(__shfl_sync(FULL_MASK, k, 0));
        int cnt_all = 0;
        int64_t q = start;
        for (;;) {
            if (q != start) fetch(q, k, aw);
            const bool inl = q + lane < m && ek_diam(k) == d0;
            const int cnt = __popc(__ballot_sync(FULL_MASK, inl));  // a prefix (sorted keys)
            if (cnt_all + cnt > RS_LEVMAX) return false;
            if (inl) {
                const int a = ek_a(k), b = ek_b(k);
                la[cnt_all + lane] = a;
                lb[cnt_all + lane] = b;
                li[cnt_all + lane] = c2((uint32_t)a) + (uint32_t)b;
                law[cnt_all + lane] = aw;
                lw[cnt_all + lane] = C.n;
                p_flip(C, a, b);
            }
            cnt_all += cnt;
            q += cnt;
            if (cnt < 32) break;
        }
        __syncwarp();
        levn = cnt_all;
        f1 = pos = q;
        lvl_d = __uint_as_float(d0);
        return true;
    }
    // Is a triangle {a, b, w} of the edge {a > b} at batch position i nonzero
    // at its level? Its level's P is P with the batch edges before i added
    // (lane j holds batch edge j; ba/bb hold them too): w is inside when
    // {a, w} and {b, w} are both among those edges, and the entry is nonzero
    // when an odd number of {a, w}, {b, w}, {a, b} are in V. Every lane calls
    // it; lanes at i >= nb answer false.
    __device__ bool batch_test(const Cloud &C, int a, int b, int i, int nb) const {
        const int lane = threadIdx.x & 31;
        const int w32 = C.w32;
        const bool live = i < nb && (C.deg[a] | C.deg[b]) != 0;
        // the earlier batch edges sharing a vertex with this one
        unsigned inc = 0;
#pragma unroll 8
        for (int j = 0; j < 31; ++j) {
            const int aj = __shfl_sync(FULL_MASK, a, j), bj = __shfl_sync(FULL_MASK, b, j);
            if (j < i && (aj == a || aj == b || bj == a || bj == b)) inc |= 1u << j;
        }
        if (!live) return false;
        const uint32_t flip = C.in(a, b) ? ~0u : 0u;
        const uint32_t *Pa = P + a * w32, *Pb = P + b * w32;
        const uint32_t *Aa = C.adj + a * w32, *Ab = C.adj + b * w32;
        const int r = lane % w32;  // lanes start at different words: fewer bank conflicts
        uint32_t any = 0;
        for (int k0 = 0; k0 < w32; k0 += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int kk = k0 + u;
                int q = r + kk;
                if (q >= w32) q -= w32;
                if (kk < w32) any |= Pa[q] & Pb[q] & (Aa[q] ^ Ab[q] ^ flip);
            }
        }
        if (any) return true;
        // third vertices w brought in by the batch edges before i
        while (inc) {
            const int j = __ffs(inc) - 1;
            inc &= inc - 1;
            const int aj = ba[j], bj = bb[j];
            const int x = (aj == a || aj == b) ? aj : bj;  // {x, w} is in
            const int w = x == aj ? bj : aj;
            const int y = x == a ? b : a;                  // {y, w} must be too
            bool in_y = (P[y * w32 + (w >> 5)] >> (w & 31)) & 1u;
            for (int j2 = 0; j2 < i && !in_y; ++j2)
                in_y = (ba[j2] == y && bb[j2] == w) || (ba[j2] == w && bb[j2] == y);
            if (in_y && ((C.in(a, w) ^ C.in(b, w) ^ (flip & 1u)) & 1u)) return true;
        }
        return false;
    }
    // Move past every level whose entries are all zero, setting their bits in
    // P, and enter the next one. Runs of single-edge levels are tested 32 at
    // a time (one per lane); a level of several equal edges is passed whole
    // when none of its edges touches V and entered otherwise. 1: entered; 0:
    // no edge left; -1: a level too large to list.
    __device__ int next_level(Cloud &C) {
        const int lane = threadIdx.x & 31;
        for (;;) {
            if (f1 >= m) {
                levn = 0;
                return 0;
            }
            uint64_t k;
            uint16_t aw;
            fetch(f1, k, aw);
            const bool valid = f1 + lane < m;
            const uint32_t db = valid ? ek_diam(k) : 0xffffffffu;
            // the diameter at f1 + 32 (the window holds it: f1 - wbase < 32)
            const uint64_t kn = __shfl_sync(FULL_MASK, k1, (int)(f1 - wbase));
            const uint32_t dn = f1 + 32 < m ? ek_diam(kn) : 0xffffffffu;
            const uint32_t up = __shfl_up_sync(FULL_MASK, db, 1);
            const uint32_t down = __shfl_down_sync(FULL_MASK, db, 1);
            const uint32_t dprev = lane == 0 ? 0xfffffffeu : up;  // f1 starts a level
            const uint32_t dnext = lane == 31 ? dn : down;
            const bool single = valid && db != dprev && db != dnext;
            const unsigned ns = __ballot_sync(FULL_MASK, !single);
            const int nb = ns ? __ffs(ns) - 1 : 32;  // lanes [0, nb): single-edge levels
            const int a = ek_a(k), b = ek_b(k);
            if (nb == 0) {
                // several equal edges from f1 on: pass them if none touches V
                const uint32_t d0 = __shfl_sync(FULL_MASK, db, 0);
                int64_t q = f1;
                bool idle = true;
                for (;;) {
                    uint64_t k2;
                    uint16_t aw2;
                    fetch(q, k2, aw2);
                    const bool inl = q + lane < m && ek_diam(k2) == d0;
                    if (__ballot_sync(FULL_MASK, inl && (C.deg[ek_a(k2)] | C.deg[ek_b(k2)]) != 0))
                        idle = false;
                    const int cnt = __popc(__ballot_sync(FULL_MASK, inl));
                    q += cnt;
                    if (cnt < 32 || !idle) break;
                }
                if (!idle) {
                    window_at(f1);
                    return load_level(C, f1) ? 1 : -1;
                }
                p_flip_range(C, f1, q);
                f1 = pos = q;
                continue;
            }
            if (lane < nb) {
                ba[lane] = a;
                bb[lane] = b;
            }
            __syncwarp();
            const unsigned hb = __ballot_sync(FULL_MASK, batch_test(C, a, b, lane, nb));
            const int first = hb ? __ffs(hb) - 1 : nb;
            if (lane < first) p_flip(C, a, b);
            __syncwarp();
            f1 = pos = f1 + first;
            if (hb) return load_level(C, f1) ? 1 : -1;
        }
    }
    // Does the triangle {a, b, w} of level edge i belong to another edge of
    // the level (one of its other edges has the level's diameter and a
    // larger index)?
    __device__ bool taken_by_other(const Cloud &C, int i, int w) const {
        const int a = la[i], b = lb[i];
        if (C.D[a * C.n + w] == lvl_d) {
            const uint32_t o = a > w ? c2((uint32_t)a) + (uint32_t)w : c2((uint32_t)w) + (uint32_t)a;
            if (o > li[i]) return true;
        }
        if (C.D[b * C.n + w] == lvl_d) {
            const uint32_t o = b > w ? c2((uint32_t)b) + (uint32_t)w : c2((uint32_t)w) + (uint32_t)b;
            if (o > li[i]) return true;
        }
        return false;
    }
    // Oldest triangle of level edge i still to come that is nonzero now: the
    // largest such w (the index grows with w), or -1.
    __device__ int level_head(const Cloud &C, int i, bool shared) const {
        const int a = la[i], b = lb[i];
        if (C.deg[a] == 0 && C.deg[b] == 0) return -1;
        const int top = lw[i] - 1;
        if (top < 0) return -1;
        const int lane = threadIdx.x & 31;
        const int w32 = C.w32;
        const uint32_t flip = C.in(a, b) ? ~0u : 0u;
        uint32_t mk = 0;
        if (lane < w32 && lane * 32 <= top) {
            mk = P[a * w32 + lane] & P[b * w32 + lane] &
                 (C.adj[a * w32 + lane] ^ C.adj[b * w32 + lane] ^ flip);
            if (lane == (top >> 5) && (top & 31) < 31) mk &= (2u << (top & 31)) - 1u;
        }
        for (;;) {
            const unsigned bal = __ballot_sync(FULL_MASK, mk != 0);
            if (!bal) return -1;
            const int hl = 31 - __clz(bal);
            const uint32_t mm = __shfl_sync(FULL_MASK, mk, hl);
            const int w = hl * 32 + 31 - __clz(mm);
            if (!shared || !taken_by_other(C, i, w)) return w;
            if (lane == hl) mk &= ~(1u << (w & 31));
        }
    }
    // The oldest nonzero entry from the current position on; the sweep moves
    // past it. ~0: the column is zero; *bail: a level too large to list.
    __device__ uint64_t pivot(Cloud &C, bool *bail) {
        for (;;) {
            if (levn == 1) {
                const int w = level_head(C, 0, false);
                if (w >= 0) {
                    if ((threadIdx.x & 31) == 0) lw[0] = w;
                    __syncwarp();
                    pa = la[0], pb = lb[0], pw = w, pi = 0;
                    return tri_key(lvl_d, tri_index(pa, pb, w));
                }
            } else if (levn > 1) {
                int best = -1, bw = -1;
                uint32_t bidx = 0;
                for (int i = 0; i < levn; ++i) {
                    const int w = level_head(C, i, true);
                    if (w < 0) continue;
                    const uint32_t ti = tri_index(la[i], lb[i], w);
                    if (best < 0 || ti > bidx) {
                        best = i;
                        bw = w;
                        bidx = ti;
                    }
                }
                if (best >= 0) {
                    // every entry with index >= bidx at this level has been passed
                    const int i = threadIdx.x & 31;
                    if (i < levn) {
                        if (i == best) lw[i] = bw;
                        else
                            while (lw[i] > 0 && tri_index(la[i], lb[i], lw[i] - 1) > bidx) --lw[i];
                    }
                    __syncwarp();
                    pa = la[best], pb = lb[best], pw = bw, pi = best;
                    return tri_key(lvl_d, bidx);
                }
            }
            const int r = next_level(C);
            if (r == 0) return ~0ull;
            if (r < 0) {
                *bail = true;
                return ~0ull;
            }
        }
    }
    // Start sweeping just past the entry k, which has just been cancelled (the
    // column is zero up to and including k). False: a level too large.
    __device__ bool enter(Cloud &C, uint64_t k) {
        const uint32_t db = (uint32_t)(k >> 32);
        const uint32_t kidx = 0xffffffffu - (uint32_t)k;
        const int64_t f = lower_bound(db);
        move_p(C, f);
        if (f >= m || ek_diam(keys[f]) != db) return false;  // k is inside: never
        window_at(f);
        if (!load_level(C, f)) return false;
        // triangles of index below kidx are still to come
        const int lane = threadIdx.x & 31;
        for (int i = 0; i < levn; ++i) {
            int wpos = C.n;
            for (int w0 = 0; w0 < C.n; w0 += 32) {
                const int w = w0 + lane;
                const unsigned bal =
                    __ballot_sync(FULL_MASK, w < C.n && tri_index(la[i], lb[i], w) >= kidx);
                if (bal) {
                    wpos = w0 + __ffs(bal) - 1;
                    break;
                }
            }
            if (lane == 0) lw[i] = wpos;
        }
        __syncwarp();
        return true;
    }
};

// The column whose final pivot is tau among the first j columns (-1: none):
// the shared hash when the cloud's columns fit it, else a scan of death[].
__device__ int64_t find_owner(const uint32_t *hkey, const uint16_t *hval, bool use_hash,
                              const uint64_t *death, int64_t j, uint32_t tau) {
    const int lane = threadIdx.x & 31;
    if (use_hash) {
        uint32_t h = (tau * 2654435761u) & (RS_HASH - 1);
        for (int round = 0; round < RS_HASH / 32; ++round) {
            const uint32_t slot = (h + lane) & (RS_HASH - 1);
            const uint32_t k = hkey[slot];
            const unsigned hit = __ballot_sync(FULL_MASK, k == tau);
            const unsigned empty = __ballot_sync(FULL_MASK, k == HASH_EMPTY);
            if (hit) {
                const int f = __ffs(hit) - 1;
                if (!(empty & ((1u << f) - 1u))) return hval[(h + f) & (RS_HASH - 1)];
                return -1;
            }
            if (empty) return -1;
            h += 32;
        }
        return -1;
    }
    int64_t oi = -1;
    for (int64_t i = lane; i < j; i += 32)
        if (death[i] == (uint64_t)tau) oi = i;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int64_t x = __shfl_xor_sync(FULL_MASK, oi, o);
        oi = x > oi ? x : oi;
    }
    return oi;
}

// V's final edges ({a > b}, as edge indices) from the adjacency bits, into
// out[0, cap); returns how many there are (all written only when <= cap).
__device__ int64_t extract_v(const Cloud &C, uint32_t *out, int64_t cap) {
    const int lane = threadIdx.x & 31;
    const int nw = C.n * C.w32;
    int64_t total = 0;
    for (int base = 0; base < nw; base += 32) {
        const int idx = base + lane;
        uint32_t word = 0;
        int a = 0, lo = 0;
        if (idx < nw) {
            a = idx / C.w32;
            lo = (idx - a * C.w32) * 32;
            word = C.adj[idx];
            if (lo >= a) word = 0;
            else if (a - lo < 32) word &= (1u << (a - lo)) - 1u;
        }
        const int cnt = __popc(word);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += x;
        }
        int64_t at = total + incl - cnt;
        while (word) {
            const int b = lo + __ffs(word) - 1;
            word &= word - 1;
            if (at < cap) out[at] = c2((uint32_t)a) + (uint32_t)b;
            ++at;
        }
        total += __shfl_sync(FULL_MASK, incl, 31);
    }
    __syncwarp();
    return total;
}

// One job (a cloud) of either phase, by one warp.
template <bool SWEEP>
__device__ void reduce_job(
    const int job, const float *__restrict__ Dall, const uint16_t *__restrict__ awall,
    const ReduceJob *__restrict__ jobs, const Leftover *__restrict__ left,
    const uint64_t *__restrict__ ekeys, const uint16_t *__restrict__ ekaw,
    const unsigned long long *__restrict__ ecount, const unsigned *__restrict__ eerr,
    uint32_t *__restrict__ vpool, uint32_t *__restrict__ vstart,
    uint32_t *__restrict__ vcnt, uint64_t *__restrict__ death_all, float *__restrict__ ddiam_all,
    const int32_t *__restrict__ status_in, int32_t *__restrict__ status,
    int32_t *__restrict__ adds_out, const unsigned *cancel) {
    extern __shared__ uint32_t dyn[];
    __shared__ uint32_t s_edge[RS_VMAX];
    __shared__ uint64_t s_head[RS_VMAX];
    __shared__ uint32_t hkey[RS_HASH];
    __shared__ uint16_t hval[RS_HASH];
    __shared__ int s_la[SWEEP ? RS_LEVMAX : 1], s_lb[SWEEP ? RS_LEVMAX : 1],
        s_lw[SWEEP ? RS_LEVMAX : 1];
    __shared__ uint32_t s_li[SWEEP ? RS_LEVMAX : 1];
    __shared__ uint16_t s_law[SWEEP ? RS_LEVMAX : 1];
    __shared__ int s_ba[SWEEP ? 32 : 1], s_bb[SWEEP ? 32 : 1];
    const int lane = threadIdx.x & 31;
    if (SWEEP && status_in[job] != 1) {  // the first phase finished it
        if (lane == 0) {
            status[job] = 0;
            adds_out[job] = 0;
        }
        return;
    }
    const ReduceJob J = jobs[job];
    const int n = J.n, w32 = (n + 31) >> 5;
    Cloud C;
    C.D = Dall + J.d_off;
    C.aw = awall + J.aw_off;
    C.n = n;
    C.w32 = w32;
    C.t = J.t;
    C.adj = dyn;
    C.deg = SWEEP ? (int32_t *)(dyn + 2 * n * w32) : nullptr;
    const Leftover *L = left + J.left_off;
    uint64_t *death = death_all + J.left_off;
    float *ddiam = ddiam_all + J.left_off;
    uint32_t *vs = vstart + J.left_off, *vc = vcnt + J.left_off;
    uint32_t *pool = vpool + J.v_off;
    const int64_t vcap = J.v_cap;
    int64_t vnext = 0;
    for (int i = lane; i < n * w32; i += 32) dyn[i] = 0;
    for (int i = lane; i < RS_HASH; i += 32) hkey[i] = HASH_EMPTY;
    Sweep S;
    S.levn = 0;
    if (SWEEP) {
        if (*eerr) {  // the edges did not all fit: the host reduces the cloud
            if (lane == 0) {
                status[job] = 1;
                adds_out[job] = 0;
            }
            return;
        }
        S.P = dyn + n * w32;
        for (int i = lane; i < n * w32; i += 32) S.P[i] = 0;
        for (int i = lane; i < n; i += 32) C.deg[i] = 0;
        S.la = s_la, S.lb = s_lb, S.lw = s_lw, S.li = s_li, S.law = s_law;
        S.ba = s_ba, S.bb = s_bb;
        S.pos = S.f1 = 0;
        // the cloud's segment of the sorted edges: keys of this job
        const int64_t cnt = (int64_t)*ecount;
        const uint64_t k0 = (uint64_t)job << 50, k1 = (uint64_t)(job + 1) << 50;
        int64_t a = 0, b = cnt;
        while (a < b) {
            const int64_t mid = (a + b) >> 1;
            if (ekeys[mid] < k0) a = mid + 1;
            else b = mid;
        }
        const int64_t lo = a;
        b = cnt;
        while (a < b) {
            const int64_t mid = (a + b) >> 1;
            if (ekeys[mid] < k1) a = mid + 1;
            else b = mid;
        }
        S.keys = ekeys + lo;
        S.kaw = ekaw + lo;
        S.m = a - lo;
        S.wbase = 0;
    }
    __syncwarp();
    const bool use_hash = J.nleft <= RS_HASH / 2;
    VList V{s_edge, s_head, 0};
    int total_adds = 0;
    bool bail = false;
    for (int64_t j = 0; j < J.nleft && !bail; ++j) {
        if (cancel && (j & 15) == 0 && *(volatile const unsigned *)cancel) {
            bail = true;  // the host no longer needs this cloud
            break;
        }
        bool have = L[j].pivot != NO_PIVOT;
        uint64_t k = have ? tri_key(L[j].pdiam, (uint32_t)L[j].pivot) : ~0ull;
        bool cursors = true;  // false: the column sweeps
        {
            int xy[2];
            decode_edge(L[j].sigma, xy);
            if (lane == 0) {
                s_edge[0] = (uint32_t)L[j].sigma;
                s_head[0] = k;  // the oldest cofacet of the column's edge
                C.flip1(xy[0], xy[1]);
            }
            V.vcount = 1;
        }
        __syncwarp();
        int adds = 0;
        while (have) {
            // the pivot's youngest facet s = {sa > sb} and the vertex vr it adds
            int sa, sb, vr;
            int saw = -1;  // s's apparent vertex when already at hand
            if (SWEEP && !cursors && S.levn == 1) {  // the level's one edge: no tie
                sa = S.pa, sb = S.pb, vr = S.pw;
                saw = S.law[0];
            } else {
                int v[3];
                if (cursors) {
                    tri_vertices(0xffffffffu - (uint32_t)k, v);
                } else {
                    v[0] = S.pa, v[1] = S.pb, v[2] = S.pw;
                    if (v[2] > v[0]) { const int x = v[0]; v[0] = v[2]; v[2] = v[1]; v[1] = x; }
                    else if (v[2] > v[1]) { const int x = v[1]; v[1] = v[2]; v[2] = x; }
                }
                const float fd[3] = {C.D[v[1] * n + v[2]], C.D[v[0] * n + v[2]],
                                     C.D[v[0] * n + v[1]]};
                int r = 0;  // facets in increasing index order: without v0, v1, v2
                for (int i = 1; i < 3; ++i)
                    if (fd[i] > fd[r]) r = i;
                sa = r == 0 ? v[1] : v[0];
                sb = r == 2 ? v[1] : v[2];
                vr = v[r];
            }
            const uint32_t s = c2((uint32_t)sa) + (uint32_t)sb;
            const uint32_t tau = 0xffffffffu - (uint32_t)k;
            int64_t oi = -1;  // -1: apparent owner; >= 0: a leftover column
            if ((saw >= 0 ? (uint16_t)saw : C.aw[s]) != (uint16_t)vr) {
                oi = find_owner(hkey, hval, use_hash, death, j, tau);
                if (oi < 0) break;  // free: the column is paired with k
            }
            if (++adds > RS_ADDS_MAX) {  // never expected: walks end by construction
                bail = true;
                break;
            }
            const int add_edges = oi < 0 ? 1 : (int)vc[oi];
            const bool enter =
                cursors && (adds > (SWEEP ? RS_SWEEP_AFTER : RS_BUDGET) ||
                            V.vcount + add_edges > RS_VMAX);
            if (enter) {
                if (!SWEEP) {
                    bail = true;
                    break;
                }
                cursors = false;  // this column goes on as a sweep
            }
            // the addition: every entry up to k is then zero
            if (cursors) {
                if (oi < 0) {
                    if (!V.toggle(C, s, k)) bail = true;
                } else {
                    const uint32_t *Vi = pool + vs[oi];
                    for (int q = 0; q < add_edges && !bail; ++q)
                        if (!V.toggle(C, Vi[q], k)) bail = true;
                }
                if (bail) break;
                V.pass(C, k);
                k = V.pivot(C);
            } else if (SWEEP) {
                if (oi < 0) {
                    if (lane == 0) C.flip1(sa, sb);
                } else {
                    const uint32_t *Vi = pool + vs[oi];
                    for (int q = lane; q < add_edges; q += 32) {
                        int xy[2];
                        decode_edge((uint64_t)Vi[q], xy);
                        C.flip_atomic(xy[0], xy[1]);
                    }
                }
                __syncwarp();
                if (enter && !S.enter(C, k)) {
                    bail = true;
                    break;
                }
                bool sb_bail = false;
                k = S.pivot(C, &sb_bail);
                if (sb_bail) {
                    bail = true;
                    break;
                }
            }
            if (k == ~0ull) have = false;  // zero column: an essential class
        }
        total_adds += adds;
        if (!bail) {
            // the pair, and V's final edges into the cloud's pool
            const uint32_t tau = 0xffffffffu - (uint32_t)k;
            int64_t cnt;
            if (cursors) {
                cnt = V.vcount;
                if (vnext + cnt <= vcap)
                    for (int q = lane; q < V.vcount; q += 32) pool[vnext + q] = s_edge[q];
            } else {
                cnt = extract_v(C, pool + vnext, vcap - vnext);
            }
            if (vnext + cnt > vcap) {
                bail = true;
            } else if (lane == 0) {
                death[j] = have ? (uint64_t)tau : NO_PIVOT;
                ddiam[j] = have ? __uint_as_float((uint32_t)(k >> 32)) : 0.0f;
                vs[j] = (uint32_t)vnext;
                vc[j] = (uint32_t)cnt;
                if (have && use_hash) {
                    uint32_t h = (tau * 2654435761u) & (RS_HASH - 1);
                    while (hkey[h] != HASH_EMPTY) h = (h + 1) & (RS_HASH - 1);
                    hkey[h] = tau;
                    hval[h] = (uint16_t)j;
                }
            }
            vnext += cnt;
        }
        __syncwarp();
        // clear V for the next column
        if (cursors) {
            for (int q = lane; q < V.vcount; q += 32) {
                int xy[2];
                decode_edge((uint64_t)s_edge[q], xy);
                C.flip_atomic(xy[0], xy[1]);
            }
        } else {
            for (int i = lane; i < n * w32; i += 32) dyn[i] = 0;
            for (int i = lane; i < n; i += 32) C.deg[i] = 0;
        }
        __syncwarp();
    }
    if (lane == 0) {
        status[job] = bail ? 1 : 0;
        adds_out[job] = total_adds;
    }
}

// The first phase: one block (warp) per job.
__global__ void __launch_bounds__(32) k_reduce_cursors(
    const float *__restrict__ Dall, const uint16_t *__restrict__ awall,
    const ReduceJob *__restrict__ jobs, const Leftover *__restrict__ left,
    uint32_t *__restrict__ vpool, uint32_t *__restrict__ vstart, uint32_t *__restrict__ vcnt,
    uint64_t *__restrict__ death, float *__restrict__ ddiam, int32_t *__restrict__ status,
    int32_t *__restrict__ adds, const unsigned *cancel) {
    reduce_job<false>((int)blockIdx.x, Dall, awall, jobs, left, nullptr, nullptr, nullptr, nullptr,
                      vpool, vstart, vcnt, death, ddiam, nullptr, status, adds, cancel);
}

// The second phase: a fixed number of blocks (one per SM by default) take
// jobs in the given order (the heaviest first) from a counter, so that the
// next launches' fused passes keep room on the SMs.
__global__ void __launch_bounds__(32) k_reduce_sweeps(
    const float *__restrict__ Dall, const uint16_t *__restrict__ awall,
    const ReduceJob *__restrict__ jobs, int njobs, const int32_t *__restrict__ order,
    unsigned *__restrict__ next, const Leftover *__restrict__ left,
    const uint64_t *__restrict__ ekeys, const uint16_t *__restrict__ ekaw,
    const unsigned long long *__restrict__ ecount, const unsigned *__restrict__ eerr,
    uint32_t *__restrict__ vpool, uint32_t *__restrict__ vstart, uint32_t *__restrict__ vcnt,
    uint64_t *__restrict__ death, float *__restrict__ ddiam, const int32_t *__restrict__ status_in,
    int32_t *__restrict__ status, int32_t *__restrict__ adds) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        int jj = 0;
        if (lane == 0) jj = (int)atomicAdd(next, 1u);
        jj = __shfl_sync(FULL_MASK, jj, 0);
        if (jj >= njobs) break;
        reduce_job<true>(order[jj], Dall, awall, jobs, left, ekeys, ekaw, ecount, eerr, vpool,
                         vstart, vcnt, death, ddiam, status_in, status, adds, nullptr);
        __syncwarp();
    }
}

// Sweep keys of the edges inside the threshold of every cloud the first phase
// handed on (status 1), appended through warp-aggregated atomics; a count
// beyond cap sets *err (the clouds then go to the host).
__global__ void __launch_bounds__(256) k_sweep_edges(const float *__restrict__ Dall,
                                                     const ReduceJob *__restrict__ jobs,
                                                     const int32_t *__restrict__ status,
                                                     uint64_t *__restrict__ keys, uint64_t cap,
                                                     unsigned long long *__restrict__ count,
                                                     unsigned *__restrict__ err) {
    const int job = blockIdx.x;
    if (status[job] != 1) return;
    const ReduceJob J = jobs[job];
    const int n = J.n;
    const float *D = Dall + J.d_off;
    const uint64_t ne = (uint64_t)n * (uint64_t)(n - 1) / 2;
    const int lane = threadIdx.x & 31;
    for (uint64_t base = 0; base < ne; base += blockDim.x) {
        const uint64_t e = base + threadIdx.x;
        bool keep = false;
        uint64_t key = 0;
        if (e < ne) {
            int xy[2];
            decode_edge(e, xy);
            const float d = D[xy[0] * n + xy[1]];
            keep = d <= J.t;
            key = edge_key(job, d, xy[0], xy[1]);
        }
        const unsigned bal = __ballot_sync(FULL_MASK, keep);
        if (!bal) continue;
        const int leader = __ffs(bal) - 1;
        unsigned long long at = 0;
        if (lane == leader) at = atomicAdd(count, (unsigned long long)__popc(bal));
        at = __shfl_sync(FULL_MASK, at, leader);
        if (keep) {
            const unsigned long long p = at + __popc(bal & ((1u << lane) - 1u));
            if (p < cap) keys[p] = key;
            else atomicOr(err, 1u);
        }
    }
}

// The apparent vertex of every sorted sweep edge (aw of its cloud at the
// edge's index), so that the sweep reads it beside the key.
__global__ void __launch_bounds__(256) k_sweep_aw(const uint64_t *__restrict__ keys,
                                                  const unsigned long long *__restrict__ count,
                                                  uint64_t cap, const uint16_t *__restrict__ aw,
                                                  const ReduceJob *__restrict__ jobs,
                                                  uint16_t *__restrict__ kaw) {
    const uint64_t m = count_of(count, cap);
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[q];
        const int job = (int)(k >> 50);
        const uint32_t e = c2((uint32_t)ek_a(k)) + (uint32_t)ek_b(k);
        kaw[q] = aw[jobs[job].aw_off + e];
    }
}

}  // namespace

// Pool words of a cloud: RS_VMAX edges per column, and room for a quarter of
// the cloud's edges besides (the final edge sets of columns that swept).
size_t reduce_small_vpool_words(uint64_t nleft, uint64_t n) {
    return (size_t)(nleft * RS_VMAX + n * (n - 1) / 8);
}

void launch_reduce_small(const ReduceSmallArgs &A, cudaStream_t s) {
    if (A.njobs <= 0) return;
    const size_t w32 = (size_t)(A.nmax + 31) / 32;
    const size_t smem_a = (size_t)A.nmax * w32 * 4;
    allow_dynamic_smem((const void *)k_reduce_cursors, smem_a);
    ++g_launches;
    k_reduce_cursors<<<(unsigned)A.njobs, 32, smem_a, s>>>(A.D, A.aw, A.jobs, A.left, A.vpool,
                                                          A.vstart, A.vcnt, A.death, A.ddiam,
                                                          A.status, A.adds, A.cancel);
}

void launch_reduce_small_sweep(const ReduceSmallArgs &A, cudaStream_t s) {
    if (A.njobs <= 0 || !A.ekeys || A.ecap == 0) return;
    const size_t w32 = (size_t)(A.nmax + 31) / 32;
    const size_t smem_b = 2 * (size_t)A.nmax * w32 * 4 + (size_t)A.nmax * 4;
    cudaMemsetAsync(A.ecount, 0, sizeof(unsigned long long), s);
    cudaMemsetAsync(A.eerr, 0, sizeof(unsigned), s);
    cudaMemsetAsync(A.next_b, 0, sizeof(unsigned), s);
    ++g_launches;
    k_sweep_edges<<<(unsigned)A.njobs, 256, 0, s>>>(A.D, A.jobs, A.status, A.ekeys, A.ecap,
                                                    A.ecount, A.eerr);
    radix_sort(nullptr, A.ekeys, nullptr, nullptr, A.etmp, nullptr, A.escratch, A.ecap, A.ecount,
               EK_BITS, A.eerr, s);
    ++g_launches;
    k_sweep_aw<<<152 * 4, 256, 0, s>>>(A.ekeys, A.ecount, A.ecap, A.aw, A.jobs, A.ekaw);
    allow_dynamic_smem((const void *)k_reduce_sweeps, smem_b);
    const int blocks = std::max(1, std::min(A.njobs, A.blocks_b > 0 ? A.blocks_b : 152));
    ++g_launches;
    k_reduce_sweeps<<<(unsigned)blocks, 32, smem_b, s>>>(
        A.D, A.aw, A.jobs, A.njobs, A.order_b, A.next_b, A.left, A.ekeys, A.ekaw, A.ecount,
        A.eerr, A.vpool, A.vstart, A.vcnt, A.death, A.ddiam, A.status, A.status_b, A.adds_b);
}

}  // namespace rpp
