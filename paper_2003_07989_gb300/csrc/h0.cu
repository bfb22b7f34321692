// h0.cu -- H0 of one instance on the GPU (Sec. "Zero-Dimensional Persistence
// Computation"): the minimum spanning forest of the edges inside the threshold,
// whose edges are the H0 deaths and the dimension-1 columns that the clearing
// lemma removes.
//
// The paper runs Kruskal's union-find on the host. Here Boruvka's rounds run
// on the device under the filtration's strict total order of edges (diameter,
// then larger index first; no two edges compare equal), so the forest is the
// unique minimum one, the forest Kruskal builds in that order. Every round at
// least halves the number of components that still have an edge inside the
// threshold, so ceil(log2 n) + 1 rounds always suffice and the host launches
// them without reading anything back; a round after one that hooked nothing
// returns at once (flags[r] records whether round r hooked). A round:
//   reset : best[c] = none for every vertex (only roots are used);
//   min   : warps scan the rows in chunks for each vertex u's lightest edge
//           to another component and fold it into best[comp[u]] (64-bit
//           atomicMin of the key (bits(d) << 32) | ~index; the index fits
//           32 bits since C(n, 2) < 2^32);
//   hook  : each root with an edge hooks onto the other endpoint's root; when
//           two roots picked the same edge, the smaller one stays a root, and
//           that edge is recorded once;
//   jump  : every vertex follows the hooks to its new root (a forest: at most
//           n - 1 hops; a longer chain sets ERR_INTERNAL instead of looping).
// Finally the forest's columns are found in the sorted dimension-1 array by
// binary search on (~bits(d), index) and marked cleared.
#include <algorithm>
#include <utility>

#include "device_common.cuh"
#include "internal.h"

namespace rpp {

namespace {

__global__ void k_h0_init(int32_t *__restrict__ comp, int64_t n, unsigned *__restrict__ nmst,
                          unsigned *__restrict__ flags, int rounds) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) comp[v] = (int32_t)v;
    if (v == 0) *nmst = 0u;
    if (v < rounds) flags[v] = 0u;
}

// Round r has work unless round r - 1 hooked nothing.
__device__ __forceinline__ bool h0_idle(const unsigned *flags, int r) {
    return r > 0 && flags[r - 1] == 0u;
}

__global__ void k_h0_reset(unsigned long long *__restrict__ best, int64_t n,
                           const unsigned *__restrict__ flags, int r) {
    if (h0_idle(flags, r)) return;
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) best[v] = ~0ull;
}

// A task is one chunk of H0_CHUNK entries of one row, taken by one warp: each
// lane loads its H0_CHUNK / 32 entries (and their components) before testing
// any, so the loads of a chunk are in flight together; many chunks per row
// keep the SMs busy however few rows there are.
constexpr int H0_CHUNK = 256;

__global__ void __launch_bounds__(256) k_h0_min(const float *__restrict__ D, int64_t ld, int64_t n,
                                                const DevState *__restrict__ st,
                                                const int32_t *__restrict__ comp,
                                                unsigned long long *__restrict__ best,
                                                const unsigned *__restrict__ flags, int r) {
    if (h0_idle(flags, r)) return;
    constexpr int PER = H0_CHUNK / 32;
    const float t = st->t;
    const int lane = threadIdx.x & 31;
    const int64_t chunks = (n + H0_CHUNK - 1) / H0_CHUNK;
    const int64_t tasks = n * chunks;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t task = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; task < tasks;
         task += warps) {
        const int64_t u = task / chunks;
        const int64_t w0 = (task - u * chunks) * H0_CHUNK + lane;
        const int32_t cu = comp[u];
        const float *row = D + u * ld;
        float d[PER];
        int32_t cw[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int64_t w = w0 + 32 * i;
            d[i] = w < n ? row[w] : 0.0f;
            cw[i] = w < n ? comp[w] : cu;
        }
        unsigned long long bk = ~0ull;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int64_t w = w0 + 32 * i;
            if (cw[i] == cu || !(d[i] <= t)) continue;  // also w == u and w >= n
            const uint64_t e = u > w ? (uint64_t)u * (uint64_t)(u - 1) / 2 + (uint64_t)w
                                     : (uint64_t)w * (uint64_t)(w - 1) / 2 + (uint64_t)u;
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(d[i]) << 32) | (unsigned long long)(~(uint32_t)e);
            bk = key < bk ? key : bk;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long x = __shfl_xor_sync(FULL_MASK, bk, o);
            bk = x < bk ? x : bk;
        }
        if (lane == 0 && bk != ~0ull) atomicMin(&best[cu], bk);
    }
}

__global__ void k_h0_hook(int64_t n, const int32_t *__restrict__ comp,
                          const unsigned long long *__restrict__ best, int32_t *__restrict__ parent,
                          unsigned long long *__restrict__ mst, unsigned *__restrict__ nmst,
                          unsigned *__restrict__ flags, int r) {
    if (h0_idle(flags, r)) return;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    parent[c] = (int32_t)c;
    if (comp[c] != c) return;
    const unsigned long long bk = best[c];
    if (bk == ~0ull) return;
    int v[2];
    decode_edge((uint64_t)(~(uint32_t)bk), v);
    const int32_t ca = comp[v[0]], cb = comp[v[1]];
    const int32_t o = ca == c ? cb : ca;
    const bool mutual = best[o] == bk;
    if (!(mutual && c < o)) parent[c] = o;
    if (!(mutual && c > o)) mst[atomicAdd(nmst, 1u)] = bk;  // each forest edge once
    flags[r] = 1u;
}

__global__ void k_h0_jump(int64_t n, const int32_t *__restrict__ comp,
                          const int32_t *__restrict__ parent, int32_t *__restrict__ next,
                          DevState *__restrict__ st, const unsigned *__restrict__ flags, int r) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    if (flags[r] == 0u) {  // nothing hooked: the components stay
        next[v] = comp[v];
        return;
    }
    int32_t root = comp[v];
    int64_t hops = 0;
    while (parent[root] != root && hops < n) {
        root = parent[root];
        ++hops;
    }
    if (parent[root] != root) atomicOr(&st->err, (unsigned)ERR_INTERNAL);
    next[v] = root;
}

// Position of each forest edge in the sorted dimension-1 array (ascending
// (key_hi, key_lo) = (~bits(d), index)); the column there is marked cleared.
__global__ void k_h0_clear(const unsigned long long *__restrict__ mst,
                           const unsigned *__restrict__ nmst, const uint32_t *__restrict__ key_hi,
                           const uint64_t *__restrict__ key_lo, uint64_t ncols_cap,
                           const unsigned long long *d_ncols, uint8_t *__restrict__ status,
                           uint32_t *__restrict__ pos) {
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *nmst) return;
    const uint64_t ncols = count_of(d_ncols, ncols_cap);
    const unsigned long long bk = mst[i];
    const uint32_t hi = ~(uint32_t)(bk >> 32);
    const uint64_t lo = (uint64_t)(~(uint32_t)bk);
    uint64_t a = 0, b = ncols;
    while (a < b) {
        const uint64_t m = (a + b) >> 1;
        if (key_hi[m] < hi || (key_hi[m] == hi && key_lo[m] < lo)) a = m + 1;
        else b = m;
    }
    pos[i] = (uint32_t)a;
    if (a < ncols && key_hi[a] == hi && key_lo[a] == lo) status[a] = COL_CLEARED;
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

void launch_h0_forest(const float *D, int64_t ld, int64_t n, DevState *st, int32_t *comp,
                      int32_t *parent, int32_t *next, unsigned long long *best,
                      unsigned long long *mst, unsigned *nmst, unsigned *flags, cudaStream_t s) {
    if (n < 1) return;
    int rounds = 1;
    while ((int64_t(1) << (rounds - 1)) < n) ++rounds;  // ceil(log2 n) + 1
    ++g_launches;
    k_h0_init<<<blocks_for(std::max<int64_t>(n, rounds), 256), 256, 0, s>>>(comp, n, nmst, flags,
                                                                          rounds);
    const int64_t tasks = n * ((n + H0_CHUNK - 1) / H0_CHUNK);  // one warp each
    int64_t warps = tasks;
    if (warps > 152 * 64) warps = 152 * 64;
    const unsigned min_blocks = (unsigned)((warps * 32 + 255) / 256);
    for (int r = 0; r < rounds; ++r) {
        g_launches += 4;
        k_h0_reset<<<blocks_for(n, 256), 256, 0, s>>>(best, n, flags, r);
        k_h0_min<<<min_blocks, 256, 0, s>>>(D, ld, n, st, comp, best, flags, r);
        k_h0_hook<<<blocks_for(n, 256), 256, 0, s>>>(n, comp, best, parent, mst, nmst, flags, r);
        k_h0_jump<<<blocks_for(n, 256), 256, 0, s>>>(n, comp, parent, next, st, flags, r);
        std::swap(comp, next);
    }
}

void launch_h0_clear(const unsigned long long *mst, const unsigned *nmst, int64_t n,
                     const uint32_t *key_hi, const uint64_t *key_lo, uint64_t ncols,
                     const unsigned long long *d_ncols, uint8_t *status, uint32_t *pos,
                     cudaStream_t s) {
    if (n < 2 || ncols == 0) return;
    ++g_launches;
    k_h0_clear<<<blocks_for(n, 256), 256, 0, s>>>(mst, nmst, key_hi, key_lo, ncols, d_ncols,
                                                  status, pos);
}

}  // namespace rpp
