// filtration.cu -- filtration construction with clearing (Alg. 6 and Alg. 7,
// Sec. "Filtration Construction with Clearing").
//
// Every index c in [0, C(n, p+1)) names one p-simplex. A thread decodes c with
// the binomial table staged in shared memory (once per run of indices that
// share all vertices but the lowest, see k_build_columns), takes the diameter
// (the largest of the C(p+1, 2) distances among its vertices, Sec. 2), and
// keeps the simplex when diam <= t and it was not paired as a death in
// dimension p-1 (the clearing lemma, Sec. "Clearing Lemma"; the previous
// dimension's deaths are a bitmap over indices). Instead of writing (-inf, +inf) sentinels for dropped
// simplices and sorting everything as Alg. 6/7 do, kept simplices are
// compacted with warp-aggregated atomics (Sec. "Warp-based Filtering"): one
// atomic per warp reserves space, lanes write at their ballot rank. The sort
// key is (~bits(diam), cidx): ascending key order is decreasing diameter, then
// increasing index, which is coboundary order.
#include "device_common.cuh"
#include "internal.h"

namespace rpp {

namespace {

// Indices c of one run share every vertex but the lowest: the p-simplex
// {v_0 > ... > v_p} has c = C(v_0, p+1) + ... + C(v_{p-1}, 2) + v_p, so for a
// fixed prefix (v_0, ..., v_{p-1}) the run c, c+1, ... walks v_p = 0, 1, ...,
// v_{p-1} - 1. A warp takes a chunk of consecutive indices, lane l index
// c0 + l + 32 k; a lane decodes its index once and then only adds 32 to v_p
// (decoding again when v_p runs past v_{p-1}, i.e. into the next prefix).
// Per index that leaves p distance reads, D[v_i][v_p] for i < p, which the
// lanes of a warp take from the same rows at consecutive columns (coalesced),
// and the prefix's own diameter, computed once per decode.
// One pass over a warp's chunk: decode once, then step v_p by 32 (decoding
// again when v_p runs into the next prefix). Calls f(k, c, keep, d) for
// iteration k (index c = c0 + lane + 32 k, valid when c < cend).
template <int P, class F>
__device__ __forceinline__ void chunk_pass(const float *__restrict__ D, int64_t ld, int64_t n,
                                           const uint64_t *B, const uint32_t *__restrict__ cleared,
                                           float t, uint64_t c0, uint64_t cend, int lane, F &&f) {
    int v[P + 1];
    const float *row[P];
    float pd = 0.0f;  // diameter of the prefix v_0 .. v_{p-1}
    bool fresh = true;
    int k = 0;
    for (uint64_t c = c0 + lane;; c += 32, ++k) {
        const bool valid = c < cend;
        if (!__any_sync(FULL_MASK, valid)) break;
        bool keep = false;
        float d = 0.0f;
        if (valid) {
            if (!fresh) v[P] += 32;
            if (fresh || v[P] >= v[P - 1]) {
                decode_simplex<P>(c, B, n, v);
                pd = 0.0f;
#pragma unroll
                for (int a = 0; a < P; ++a) {
                    row[a] = D + (int64_t)v[a] * ld;
#pragma unroll
                    for (int b = a + 1; b < P; ++b) pd = fmaxf(pd, row[a][v[b]]);
                }
                fresh = false;
            }
            if (!(cleared && ((cleared[c >> 5] >> (c & 31)) & 1u))) {
                d = pd;
#pragma unroll
                for (int a = 0; a < P; ++a) d = fmaxf(d, row[a][v[P]]);
                keep = d <= t;
            }
        }
        f(k, c, keep, d);
    }
}

// Indices c of one run share every vertex but the lowest: the p-simplex
// {v_0 > ... > v_p} has c = C(v_0, p+1) + ... + C(v_{p-1}, 2) + v_p, so for a
// fixed prefix (v_0, ..., v_{p-1}) the run c, c+1, ... walks v_p = 0, 1, ...,
// v_{p-1} - 1. A warp takes a chunk of at most 2048 consecutive indices, lane
// l index c0 + l + 32 k; a lane decodes its index once and then only adds 32
// to v_p. Per index that leaves p distance reads, D[v_i][v_p] for i < p,
// which the lanes of a warp take from the same rows at consecutive columns
// (coalesced), and the prefix's own diameter, computed once per decode.
// Compaction takes two passes over the chunk: the first records which
// indices are kept (one bit per lane and step) and reserves the chunk's
// output with ONE atomic (a warp-per-step atomic on the shared counter
// serialises once the candidates number in the billions); the second
// recomputes the kept diameters (their rows are in cache) and writes them at
// their ballot ranks.
// Ordered build (k_build_count, k_chunk_offsets, k_build_write): the same
// chunks and passes, split into three kernels. The first counts each chunk's
// kept indices, the second turns the counts into each chunk's output offset
// (an exclusive scan, in chunk order) and the column count, the third writes
// every chunk at its offset. The columns then leave in increasing index
// order, so the sort needs only the diameter digits (a stable sort keeps the
// index order within a diameter). No kernel waits on another block.
template <int P>
__global__ void __launch_bounds__(256) k_build_columns(const float *__restrict__ D, int64_t ld,
                                                        int64_t n, const uint64_t *__restrict__ gB,
                                                        bool smem_table, uint64_t total,
                                                        uint64_t chunk,
                                                        const uint32_t *__restrict__ cleared,
                                                        DevState *st, uint32_t *__restrict__ key_hi,
                                                        uint64_t *__restrict__ key_lo) {
    extern __shared__ uint64_t sB[];
    const uint64_t *B = stage_binomial(gB, n, P + 1, sB, smem_table);
    const float t = st->t;
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t c0 = warp * chunk; c0 < total; c0 += nwarps * chunk) {
        const uint64_t cend = c0 + chunk < total ? c0 + chunk : total;
        uint64_t kept = 0;  // bit k: this lane's index of step k is kept
        chunk_pass<P>(D, ld, n, B, cleared, t, c0, cend, lane,
                      [&](int k, uint64_t, bool keep, float) {
                          if (keep) kept |= 1ull << k;
                      });
        unsigned cnt = __popcll(kept);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL_MASK, cnt, o);
        if (cnt == 0) continue;
        unsigned long long at = 0;
        if (lane == 0) at = atomicAdd(&st->ncols, (unsigned long long)cnt);
        at = __shfl_sync(FULL_MASK, at, 0);
        chunk_pass<P>(D, ld, n, B, cleared, t, c0, cend, lane,
                      [&](int k, uint64_t c, bool keep, float d) {
                          const unsigned ball = __ballot_sync(FULL_MASK, keep);
                          if (keep) {
                              const uint64_t pos = at + __popc(ball & lanemask_lt());
                              key_hi[pos] = ~__float_as_uint(d);
                              key_lo[pos] = c;
                          }
                          at += __popc(ball);
                      });
    }
}

// Ordered build, first kernel: counts[chunk] = kept indices of the chunk.
template <int P>
__global__ void __launch_bounds__(256) k_build_count(const float *__restrict__ D, int64_t ld,
                                                      int64_t n, const uint64_t *__restrict__ gB,
                                                      bool smem_table, uint64_t total,
                                                      uint64_t chunk,
                                                      const uint32_t *__restrict__ cleared,
                                                      const DevState *st,
                                                      unsigned long long *__restrict__ counts) {
    extern __shared__ uint64_t sB[];
    const uint64_t *B = stage_binomial(gB, n, P + 1, sB, smem_table);
    const float t = st->t;
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t id = warp; id * chunk < total; id += nwarps) {
        const uint64_t c0 = id * chunk;
        const uint64_t cend = c0 + chunk < total ? c0 + chunk : total;
        unsigned cnt = 0;
        chunk_pass<P>(D, ld, n, B, cleared, t, c0, cend, lane,
                      [&](int, uint64_t, bool keep, float) { cnt += keep; });
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL_MASK, cnt, o);
        if (lane == 0) counts[id] = cnt;
    }
}

// Ordered build, second kernel (one block of 1024 threads): the counts
// become exclusive offsets in chunk order, tile by tile of 8192 with a
// running carry; their sum is the column count.
__global__ void __launch_bounds__(1024) k_chunk_offsets(unsigned long long *__restrict__ counts,
                                                        uint64_t nchunks, DevState *st) {
    constexpr int ITEMS = 8;
    __shared__ unsigned long long s_warp[32];
    __shared__ unsigned long long s_carry;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (uint64_t base = 0; base < nchunks; base += 1024 * ITEMS) {
        unsigned long long v[ITEMS], sum = 0;
        const uint64_t i0 = base + (uint64_t)tid * ITEMS;
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            v[k] = i0 + k < nchunks ? counts[i0 + k] : 0ull;
            sum += v[k];
        }
        unsigned long long incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_warp[w] = incl;
        __syncthreads();
        if (w == 0) {
            unsigned long long x = s_warp[lane], xi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(FULL_MASK, xi, o);
                if (lane >= o) xi += y;
            }
            s_warp[lane] = xi - x;  // exclusive over the warps
        }
        __syncthreads();
        unsigned long long at = s_carry + s_warp[w] + incl - sum;
#pragma unroll
        for (int k = 0; k < ITEMS; ++k)
            if (i0 + k < nchunks) {
                counts[i0 + k] = at;
                at += v[k];
            }
        __syncthreads();
        if (tid == 1023) s_carry = at;
        __syncthreads();
    }
    if (tid == 0) st->ncols = s_carry;
}

// Ordered build, third kernel: every chunk written at its offset.
template <int P>
__global__ void __launch_bounds__(256) k_build_write(const float *__restrict__ D, int64_t ld,
                                                      int64_t n, const uint64_t *__restrict__ gB,
                                                      bool smem_table, uint64_t total,
                                                      uint64_t chunk,
                                                      const uint32_t *__restrict__ cleared,
                                                      const DevState *st,
                                                      const unsigned long long *__restrict__ offs,
                                                      uint32_t *__restrict__ key_hi,
                                                      uint64_t *__restrict__ key_lo) {
    extern __shared__ uint64_t sB[];
    const uint64_t *B = stage_binomial(gB, n, P + 1, sB, smem_table);
    const float t = st->t;
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t id = warp; id * chunk < total; id += nwarps) {
        const uint64_t c0 = id * chunk;
        const uint64_t cend = c0 + chunk < total ? c0 + chunk : total;
        uint64_t at = offs[id];
        if (id + 1 < (total + chunk - 1) / chunk ? offs[id + 1] == at : st->ncols == at)
            continue;  // nothing kept
        chunk_pass<P>(D, ld, n, B, cleared, t, c0, cend, lane,
                      [&](int, uint64_t c, bool keep, float d) {
                          const unsigned ball = __ballot_sync(FULL_MASK, keep);
                          if (keep) {
                              const uint64_t pos = at + __popc(ball & lanemask_lt());
                              key_hi[pos] = ~__float_as_uint(d);
                              key_lo[pos] = c;
                          }
                          at += __popc(ball);
                      });
    }
}

// The vertices (a << 16) | b, a > b, of edge indices (n <= 65535).
__global__ void k_edge_pairs(const uint64_t *__restrict__ lo, uint64_t count,
                             uint32_t *__restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        int v[2];
        decode_edge(lo[i], v);
        out[i] = ((uint32_t)v[0] << 16) | (uint32_t)v[1];
    }
}

__global__ void k_invert_u32(const uint32_t *__restrict__ in, uint64_t count,
                             uint32_t *__restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        out[i] = ~in[i];
}

__global__ void k_bitmap_set(const uint64_t *__restrict__ idx, uint64_t count,
                             uint32_t *__restrict__ bitmap) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        const uint64_t c = idx[i];
        atomicOr(&bitmap[c >> 5], 1u << (c & 31));
    }
}

// First position i in [0, n) with a[i] >= key (a ascending), into *out.
__global__ void k_lower_bound_u32(const uint32_t *__restrict__ a, uint64_t n, uint32_t key,
                                  unsigned long long *out) {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    *out = lo;
}

// Grid and chunk of the build: chunks of consecutive indices per warp, long
// enough that a lane's single decode serves many indices, short enough to
// spread the work.
uint64_t build_grid(uint64_t total, uint64_t *chunk) {
    uint64_t blocks = (total + 255) / 256;
    const uint64_t cap = 152ull * 8;
    if (blocks > cap) blocks = cap;
    const uint64_t warps = blocks * 8;
    uint64_t c = warps ? (total + warps - 1) / warps : 32;
    c = (c + 31) / 32 * 32;
    if (c > 2048) c = 2048;
    if (c < 32) c = 32;
    *chunk = c;
    return blocks;
}

template <int P>
void build_p(const float *D, int64_t ld, int64_t n, const uint64_t *binom, uint64_t total,
             const uint32_t *cleared, DevState *st, uint32_t *key_hi, uint64_t *key_lo,
             unsigned long long *order, cudaStream_t s) {
    const size_t table = (size_t)(P + 2) * (n + 1) * sizeof(uint64_t);
    const bool smem = table <= 160 * 1024;
    uint64_t chunk;
    const uint64_t blocks = build_grid(total, &chunk);
    if (blocks == 0) return;
    const size_t sm = smem ? table : 0;
    if (!order) {
        if (smem) allow_dynamic_smem((const void *)k_build_columns<P>, table);
        ++g_launches;
        k_build_columns<P><<<(unsigned)blocks, 256, sm, s>>>(D, ld, n, binom, smem, total, chunk,
                                                             cleared, st, key_hi, key_lo);
        return;
    }
    if (smem) {
        allow_dynamic_smem((const void *)k_build_count<P>, table);
        allow_dynamic_smem((const void *)k_build_write<P>, table);
    }
    const uint64_t nchunks = (total + chunk - 1) / chunk;
    g_launches += 3;
    k_build_count<P><<<(unsigned)blocks, 256, sm, s>>>(D, ld, n, binom, smem, total, chunk,
                                                       cleared, st, order);
    k_chunk_offsets<<<1, 1024, 0, s>>>(order, nchunks, st);
    k_build_write<P><<<(unsigned)blocks, 256, sm, s>>>(D, ld, n, binom, smem, total, chunk,
                                                       cleared, st, order, key_hi, key_lo);
}

}  // namespace

size_t build_order_bytes(uint64_t total) {
    uint64_t chunk;
    build_grid(total, &chunk);
    return (size_t)((total + chunk - 1) / chunk + 1) * sizeof(unsigned long long);
}

void launch_build_columns(const float *D, int64_t ld, int64_t n, int p, const uint64_t *binom,
                          uint64_t total, const uint32_t *cleared, DevState *st, uint32_t *key_hi,
                          uint64_t *key_lo, cudaStream_t s, unsigned long long *order) {
    switch (p) {
        case 1: build_p<1>(D, ld, n, binom, total, cleared, st, key_hi, key_lo, order, s); break;
        case 2: build_p<2>(D, ld, n, binom, total, cleared, st, key_hi, key_lo, order, s); break;
        case 3: build_p<3>(D, ld, n, binom, total, cleared, st, key_hi, key_lo, order, s); break;
        case 4: build_p<4>(D, ld, n, binom, total, cleared, st, key_hi, key_lo, order, s); break;
        default: break;
    }
}

void launch_edge_pairs(const uint64_t *lo, uint64_t count, uint32_t *out, cudaStream_t s) {
    if (count == 0) return;
    uint64_t blocks = (count + 255) / 256;
    if (blocks > 152ull * 8) blocks = 152ull * 8;
    ++g_launches;
    k_edge_pairs<<<(unsigned)blocks, 256, 0, s>>>(lo, count, out);
}

void launch_lower_bound_u32(const uint32_t *a, uint64_t n, uint32_t key, unsigned long long *out,
                            cudaStream_t s) {
    ++g_launches;
    k_lower_bound_u32<<<1, 1, 0, s>>>(a, n, key, out);
}

void launch_invert_u32(const uint32_t *in, uint64_t count, uint32_t *out, cudaStream_t s) {
    if (count == 0) return;
    uint64_t blocks = (count + 255) / 256;
    if (blocks > 152ull * 8) blocks = 152ull * 8;
    ++g_launches;
    k_invert_u32<<<(unsigned)blocks, 256, 0, s>>>(in, count, out);
}

void launch_bitmap_set(const uint64_t *idx, uint64_t count, uint32_t *bitmap, cudaStream_t s) {
    if (count == 0) return;
    ++g_launches;
    k_bitmap_set<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(idx, count, bitmap);
}

}  // namespace rpp
