// radix_sort.cu -- least-significant-digit radix sort of (hi, lo) keys with an
// optional 64-bit payload (the "GPU-sort" of Alg. 7, whose implementation the
// paper leaves open).
//
// A key is the composite C = ((hi - hi_min) << lo_bits) | lo, where hi_min is
// the smallest hi among the keys (found on the device) and lo < 2^lo_bits;
// ascending C is ascending (hi, lo). Keys that arrive in increasing lo (the
// ordered filtration build) take C = hi - hi_min alone (lo_bits = 0): the
// passes are stable, so lo stays increasing within equal hi, and the sort
// needs no pass over the index bits. C is sorted 9 bits at a time, from the
// least significant digit up, every pass stable (diameter keys of a point
// cloud span about 27 significant bits: three passes of 9 bits, where 8-bit
// digits would take four). Nothing comes back to the
// host: the key count may itself live in device memory, and the passes whose
// digit is the same for every key are skipped by the kernels themselves.
//   prep    : the smallest hi (one atomic per block);
//   hist    : one sweep counts every digit position at once;
//   offsets : per digit position, the exclusive start of each digit value,
//             whether the pass is needed, and which buffer holds its input
//             (the parity of the needed passes before it);
//   onesweep: one kernel per pass. A block takes the next tile of keys (tile
//             order comes from an atomic ticket, so every tile it waits on
//             belongs to a block already running), counts its digits in
//             shared memory and publishes the counts at once, ranks its keys
//             stably (per-warp match and counts in key order), adds up the
//             counts of the tiles before it by decoupled look-back (a tile
//             that knows its inclusive prefix publishes it, so a look-back
//             stops there), and scatters its keys to their final positions
//             of this pass. Waits on another tile's entry are
//             bounded; a wait that runs out sets ERR_INTERNAL and continues.
//   finish  : copies the keys back into the caller's arrays when an odd
//             number of passes ran.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "internal.h"

namespace rpp {

namespace {

constexpr int DIGIT_BITS = RADIX_SORT_DIGIT_BITS;
constexpr int RADIX = RADIX_SORT_BINS;
constexpr int MAXP = 12;             // 96-bit composite keys at most (11 digits)
constexpr int OS_THREADS = RADIX;    // thread d owns digit value d in the look-back
constexpr int OS_WARPS = OS_THREADS / 32;
constexpr int OS_ITEMS = 4;          // keys per thread
constexpr int OS_WARP_KEYS = 32 * OS_ITEMS;
constexpr int OS_TILE = OS_THREADS * OS_ITEMS;
static_assert(OS_TILE == RADIX_SORT_TILE, "tile size shared with the scratch bound");
static_assert(RADIX <= (1 << 16), "digit and warp rank share one word");
constexpr uint64_t LB_AGG = 1ull << 62;     // tile count only
constexpr uint64_t LB_PREFIX = 2ull << 62;  // inclusive count of every tile up to this one
constexpr uint64_t LB_FLAGS = 3ull << 62;
constexpr int LB_EPOCH_SHIFT = 56;          // pass + 1 in bits 56..61
constexpr uint64_t LB_VALUE = (1ull << LB_EPOCH_SHIFT) - 1;
constexpr long long LB_SPIN_LIMIT = 1ll << 22;
constexpr int LB_WINDOW = 4;                // look-back entries loaded together

// Control block at the start of the scratch; zeroed before each sort.
struct SortCtl {
    unsigned long long hist[MAXP][RADIX];
    unsigned long long start[MAXP][RADIX];  // exclusive start of each digit value
    unsigned int tile_ticket[MAXP];
    unsigned int active[MAXP];               // pass needed (its digit is not constant)
    unsigned int src[MAXP];                  // 1: the pass reads the scratch buffers
    unsigned int final_src;
    unsigned int hi_min_inv;                 // ~(smallest hi), so that zero is the start
    unsigned int pad[3];
};

static_assert(sizeof(SortCtl) <= RADIX_SORT_CTL_BYTES, "control block bound");
constexpr size_t ctl_bytes() { return RADIX_SORT_CTL_BYTES; }

__device__ __forceinline__ uint64_t key_count(const unsigned long long *d_count, uint64_t n_cap) {
    if (!d_count) return n_cap;
    const uint64_t c = *d_count;
    return c < n_cap ? c : n_cap;
}

template <bool HAS_HI>
__device__ __forceinline__ unsigned digit_of(uint32_t h, uint64_t l, uint32_t hi_min, int lo_bits,
                                             int shift) {
    if constexpr (HAS_HI) {
        // lo_bits = 0: the keys are in increasing lo already; hi alone
        const unsigned __int128 c =
            ((unsigned __int128)(h - hi_min) << lo_bits) | (lo_bits ? l : 0ull);
        return (unsigned)(c >> shift) & (unsigned)(RADIX - 1);
    } else {
        return shift < 64 ? (unsigned)(l >> shift) & (unsigned)(RADIX - 1) : 0u;
    }
}

__global__ void __launch_bounds__(256) k_sort_prep(const uint32_t *__restrict__ hi, uint64_t n_cap,
                                                   const unsigned long long *d_count, SortCtl *ctl) {
    const uint64_t n = key_count(d_count, n_cap);
    uint32_t m = 0xffffffffu;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        m = min(m, hi[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(FULL_MASK, m, o));
    __shared__ uint32_t s_min[8];
    if ((threadIdx.x & 31) == 0) s_min[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = min(m, s_min[w]);
        atomicMax(&ctl->hi_min_inv, ~m);
    }
}

template <bool HAS_HI>
__global__ void __launch_bounds__(256) k_sort_hist(const uint32_t *__restrict__ hi,
                                                   const uint64_t *__restrict__ lo, uint64_t n_cap,
                                                   const unsigned long long *d_count, int lo_bits,
                                                   int passes, SortCtl *ctl) {
    __shared__ unsigned int sh[MAXP * RADIX];
    for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint64_t n = key_count(d_count, n_cap);
    const uint32_t hmin = HAS_HI ? ~ctl->hi_min_inv : 0u;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t l = lo[i];
        const uint32_t h = HAS_HI ? hi[i] : 0u;
        for (int p = 0; p < passes; ++p)
            atomicAdd(&sh[p * RADIX + digit_of<HAS_HI>(h, l, hmin, lo_bits, DIGIT_BITS * p)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x)
        if (sh[i]) atomicAdd(&ctl->hist[i / RADIX][i % RADIX], (unsigned long long)sh[i]);
}

// One block of RADIX threads: thread d owns digit value d.
__global__ void __launch_bounds__(RADIX) k_sort_offsets(uint64_t n_cap,
                                                        const unsigned long long *d_count,
                                                        int passes, SortCtl *ctl,
                                                        unsigned *passes_out) {
    __shared__ unsigned long long s_warp[RADIX / 32];
    __shared__ unsigned int s_const[MAXP];
    const uint64_t n = key_count(d_count, n_cap);
    const int d = threadIdx.x, lane = d & 31, w = d >> 5;
    for (int p = 0; p < passes; ++p) {
        const unsigned long long c = ctl->hist[p][d];
        if (d == 0) s_const[p] = 0;
        unsigned long long incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_warp[w] = incl;
        __syncthreads();
        unsigned long long before = 0;
        for (int k = 0; k < w; ++k) before += s_warp[k];
        ctl->start[p][d] = before + incl - c;
        if (c == n) s_const[p] = 1;  // one digit value holds every key
        __syncthreads();
    }
    if (d == 0) {
        unsigned int parity = 0, ran = 0;
        for (int p = 0; p < passes; ++p) {
            const unsigned int act = (n > 1 && !s_const[p]) ? 1u : 0u;
            ctl->active[p] = act;
            ctl->src[p] = parity;
            parity ^= act;
            ran += act;
        }
        ctl->final_src = parity;
        if (passes_out) atomicAdd(passes_out, ran);
    }
}

template <bool HAS_HI, bool HAS_VAL>
__global__ void __launch_bounds__(OS_THREADS, 2) k_onesweep(
    uint32_t *__restrict__ hi_a, uint64_t *__restrict__ lo_a, uint64_t *__restrict__ val_a,
    uint32_t *__restrict__ hi_b, uint64_t *__restrict__ lo_b, uint64_t *__restrict__ val_b,
    uint64_t n_cap, const unsigned long long *d_count, int lo_bits, int pass, SortCtl *ctl,
    unsigned long long *lookback, unsigned *err) {
    __shared__ unsigned int s_warp[OS_WARPS][RADIX];  // per-warp counts, then starts
    __shared__ unsigned int s_hist[RADIX];            // the tile's digit counts
    __shared__ unsigned long long s_base[RADIX];      // global start of each digit for this tile
    __shared__ unsigned int s_tile;
    if (!ctl->active[pass]) return;
    const uint64_t n = key_count(d_count, n_cap);
    const uint64_t ntiles = (n + OS_TILE - 1) / OS_TILE;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(&ctl->tile_ticket[pass], 1u);
#pragma unroll
    for (int k = 0; k < OS_WARPS; ++k) s_warp[k][tid] = 0;
    s_hist[tid] = 0;
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= ntiles) return;  // grids are sized for the largest count
    const bool from_b = ctl->src[pass] != 0;
    const uint32_t *hs = from_b ? hi_b : hi_a;
    const uint64_t *ls = from_b ? lo_b : lo_a;
    const uint64_t *vs = from_b ? val_b : val_a;
    uint32_t *hd = from_b ? hi_a : hi_b;
    uint64_t *ld = from_b ? lo_a : lo_b;
    uint64_t *vd = from_b ? val_a : val_b;
    const uint32_t hmin = HAS_HI ? ~ctl->hi_min_inv : 0u;
    const int shift = DIGIT_BITS * pass;

    // keys of this warp: item j of lane l is key base + j * 32 + l (key order
    // is (warp, item, lane), so per-warp ranks in item order are stable)
    const uint64_t base = tile * OS_TILE + (uint64_t)w * OS_WARP_KEYS;
    uint64_t kl[OS_ITEMS], kv[OS_ITEMS];
    uint32_t kh[OS_ITEMS];
    unsigned dg[OS_ITEMS];  // digit (RADIX: no key), then (rank in the warp << 16) | digit
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) {
        const uint64_t i = base + (uint64_t)j * 32 + lane;
        const bool ok = i < n;
        kl[j] = ok ? ls[i] : 0;
        kh[j] = (HAS_HI && ok) ? hs[i] : 0u;
        if constexpr (HAS_VAL) kv[j] = ok ? vs[i] : 0;
        dg[j] = ok ? digit_of<HAS_HI>(kh[j], kl[j], hmin, lo_bits, shift) : RADIX;
        if (ok) atomicAdd(&s_hist[dg[j]], 1u);
    }
    __syncthreads();
    // The tile's counts go out first, before its ranking, so that later tiles
    // looking back find them (and soon this tile's inclusive prefix) without
    // waiting on the ranking.
    const uint64_t epoch = (uint64_t)(pass + 1) << LB_EPOCH_SHIFT;
    unsigned long long *mine = lookback + tile * RADIX + tid;
    const unsigned int own = s_hist[tid];
    if (tile == 0) atomicExch(mine, (unsigned long long)(LB_PREFIX | epoch | own));
    else atomicExch(mine, (unsigned long long)(LB_AGG | epoch | own));
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) {
        const unsigned peers = __match_any_sync(FULL_MASK, dg[j]);
        const unsigned before = __popc(peers & lanemask_lt());
        const unsigned cnt = dg[j] < RADIX ? s_warp[w][dg[j]] : 0u;
        __syncwarp();
        if (dg[j] < RADIX && before == 0) s_warp[w][dg[j]] = cnt + __popc(peers);
        dg[j] |= (cnt + before) << 16;
        __syncwarp();
    }
    // thread tid owns digit value tid: look back for the tiles before this one
    if (tile == 0) {
        s_base[tid] = ctl->start[pass][tid];
    } else {
        // windows of LB_WINDOW entries loaded together
        uint64_t excl = 0;
        bool done = false;
        for (int64_t t0 = (int64_t)tile - 1; t0 >= 0 && !done; t0 -= LB_WINDOW) {
            unsigned long long e[LB_WINDOW];
#pragma unroll
            for (int i = 0; i < LB_WINDOW; ++i)
                e[i] = t0 - i >= 0 ? *(const volatile unsigned long long *)(lookback +
                                                                           (uint64_t)(t0 - i) *
                                                                               RADIX + tid)
                                   : 0ull;
#pragma unroll
            for (int i = 0; i < LB_WINDOW; ++i) {
                if (done || t0 - i < 0) {
                    done = true;
                    continue;
                }
                const volatile unsigned long long *src =
                    (const volatile unsigned long long *)(lookback + (uint64_t)(t0 - i) * RADIX +
                                                          tid);
                unsigned long long v = e[i];
                long long spins = 0;
                while (((v & LB_FLAGS) == 0 || (v & ~LB_FLAGS & ~LB_VALUE) != epoch) &&
                       spins < LB_SPIN_LIMIT) {
                    if (spins > 64) __nanosleep(64);
                    ++spins;
                    v = *src;
                }
                if (spins >= LB_SPIN_LIMIT) {  // never expected: report and go on
                    atomicOr(err, ERR_INTERNAL);
                    done = true;
                    continue;
                }
                excl += v & LB_VALUE;
                if ((v & LB_FLAGS) == LB_PREFIX) done = true;
            }
        }
        atomicExch(mine, (unsigned long long)(LB_PREFIX | epoch | (excl + own)));
        s_base[tid] = ctl->start[pass][tid] + excl;
    }
    __syncthreads();  // the ranks' per-warp counts are complete
    unsigned int run = 0;
#pragma unroll
    for (int k = 0; k < OS_WARPS; ++k) {
        const unsigned int c = s_warp[k][tid];
        s_warp[k][tid] = run;
        run += c;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) {
        const unsigned d = dg[j] & 0xffffu;
        if (d < RADIX) {
            const uint64_t pos = s_base[d] + s_warp[w][d] + (dg[j] >> 16);
            if (pos < n) {  // always: the counts partition the keys
                ld[pos] = kl[j];
                if constexpr (HAS_HI) hd[pos] = kh[j];
                if constexpr (HAS_VAL) vd[pos] = kv[j];
            }
        }
    }
}

// After the passes: keys that ended in the scratch buffers go back.
__global__ void __launch_bounds__(256) k_sort_finish(uint32_t *__restrict__ hi,
                                                     uint64_t *__restrict__ lo,
                                                     uint64_t *__restrict__ val,
                                                     const uint32_t *__restrict__ thi,
                                                     const uint64_t *__restrict__ tlo,
                                                     const uint64_t *__restrict__ tval,
                                                     uint64_t n_cap,
                                                     const unsigned long long *d_count,
                                                     const SortCtl *ctl) {
    if (!ctl->final_src) return;
    const uint64_t n = key_count(d_count, n_cap);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        lo[i] = tlo[i];
        if (hi) hi[i] = thi[i];
        if (val) val[i] = tval[i];
    }
}

template <bool HAS_HI, bool HAS_VAL>
void sort_passes(uint32_t *hi, uint64_t *lo, uint64_t *val, uint32_t *thi, uint64_t *tlo,
                 uint64_t *tval, SortCtl *ctl, unsigned long long *lookback, uint64_t n_cap,
                 const unsigned long long *d_count, int lo_bits, int passes, unsigned *err,
                 cudaStream_t s) {
    const uint64_t ntiles = (n_cap + OS_TILE - 1) / OS_TILE;
    for (int p = 0; p < passes; ++p) {
        ++g_launches;
        k_onesweep<HAS_HI, HAS_VAL><<<(unsigned)ntiles, OS_THREADS, 0, s>>>(
            hi, lo, val, thi, tlo, tval, n_cap, d_count, lo_bits, p, ctl, lookback, err);
    }
}

}  // namespace

size_t radix_scratch_bytes(uint64_t n_cap) { return radix_scratch_bound(n_cap); }

void radix_sort(uint32_t *hi, uint64_t *lo, uint64_t *val, uint32_t *tmp_hi, uint64_t *tmp_lo,
                uint64_t *tmp_val, void *scratch, uint64_t n_cap,
                const unsigned long long *d_count, int lo_bits, unsigned *err, cudaStream_t s,
                unsigned *passes_out) {
    if (n_cap <= 1) return;
    if (lo_bits < 1 && !hi) lo_bits = 1;
    if (lo_bits < 0) lo_bits = 0;
    const int bits = lo_bits + (hi ? 32 : 0);
    int passes = (bits + DIGIT_BITS - 1) / DIGIT_BITS;
    if (passes > MAXP) passes = MAXP;
    SortCtl *ctl = (SortCtl *)scratch;
    unsigned long long *lookback = (unsigned long long *)((char *)scratch + ctl_bytes());
    cudaMemsetAsync(scratch, 0, radix_scratch_bytes(n_cap), s);
    uint64_t hb = (n_cap + 255) / 256;
    if (hb > 152 * 4) hb = 152 * 4;
    if (hi) {
        ++g_launches;
        k_sort_prep<<<(unsigned)hb, 256, 0, s>>>(hi, n_cap, d_count, ctl);
        ++g_launches;
        k_sort_hist<true><<<(unsigned)hb, 256, 0, s>>>(hi, lo, n_cap, d_count, lo_bits, passes, ctl);
    } else {
        ++g_launches;
        k_sort_hist<false><<<(unsigned)hb, 256, 0, s>>>(hi, lo, n_cap, d_count, lo_bits, passes,
                                                        ctl);
    }
    ++g_launches;
    k_sort_offsets<<<1, RADIX, 0, s>>>(n_cap, d_count, passes, ctl, passes_out);
    if (hi && val)
        sort_passes<true, true>(hi, lo, val, tmp_hi, tmp_lo, tmp_val, ctl, lookback, n_cap, d_count,
                                lo_bits, passes, err, s);
    else if (hi)
        sort_passes<true, false>(hi, lo, nullptr, tmp_hi, tmp_lo, nullptr, ctl, lookback, n_cap,
                                 d_count, lo_bits, passes, err, s);
    else if (val)
        sort_passes<false, true>(nullptr, lo, val, nullptr, tmp_lo, tmp_val, ctl, lookback, n_cap,
                                 d_count, lo_bits, passes, err, s);
    else
        sort_passes<false, false>(nullptr, lo, nullptr, nullptr, tmp_lo, nullptr, ctl, lookback,
                                  n_cap, d_count, lo_bits, passes, err, s);
    ++g_launches;
    k_sort_finish<<<(unsigned)hb, 256, 0, s>>>(hi, lo, val, tmp_hi, tmp_lo, tmp_val, n_cap, d_count,
                                               ctl);
}

}  // namespace rpp
