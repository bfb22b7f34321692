// internal.h -- declarations shared by the library's CUDA kernels and its host
// code (pipeline, submatrix reduction, C ABI). Not installed; the public
// interface is include/rpp.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace rpp {

// Column status written by the apparent-pair pass (one byte per column).
enum : uint8_t { COL_LEFTOVER = 0, COL_APPARENT = 1, COL_CLEARED = 2 };

// "No pivot": the column's coboundary is empty inside the threshold.
constexpr uint64_t NO_PIVOT = ~0ull;

// Scalars the kernels share through device memory, so a pipeline needs no host
// round trip to pass them along.
struct DevState {
    float t;                   // threshold in use (min(user threshold, enclosing radius))
    float R;                   // enclosing radius
    unsigned int err;          // input validation flags (ERR_*)
    unsigned int pad0;
    unsigned long long ncols;  // columns written by the filtration kernel
    unsigned long long napp;   // apparent pairs written by the partition kernel
    unsigned long long nleft;  // leftover columns written by the partition kernel
    unsigned long long begin;  // first column inside a quantile threshold
    unsigned long long scanned;  // candidate vertices examined by the apparent pass
};

// Kernels launched by the calling thread (incremented by every launcher).
extern thread_local long long g_launches;

enum : unsigned int { ERR_NONFINITE = 1u, ERR_NEGATIVE = 2u, ERR_ASYMMETRIC = 4u, ERR_DIAGONAL = 8u };

// A leftover column handed to the host reduction, with its unreduced pivot
// (the oldest cofacet inside the threshold) found during the apparent pass.
struct Leftover {
    uint64_t sigma;   // combinatorial index of the column simplex
    uint64_t pivot;   // combinatorial index of its oldest cofacet, NO_PIVOT if none
    float diam;       // diameter of sigma
    float pdiam;      // diameter of the pivot
    uint64_t index;   // position of the column in coboundary order
};

// Binomial table C(v, k) for k = 0..kmax, v = 0..n, row-major by k; entries that
// overflow 63 bits saturate at UINT64_MAX (never used by valid inputs).
struct Binomial {
    int64_t n = 0;
    int kmax = 0;
    uint64_t *host = nullptr;  // (kmax + 1) * (n + 1)
    uint64_t at(int k, int64_t v) const { return host[(int64_t)k * (n + 1) + v]; }
};

// ---- kernel launchers (defined in the .cu files) --------------------------

// Distance matrix from points with the fixed operation order (no fused
// multiply-add, correctly rounded square root). D has row stride ld.
void launch_distance_matrix(const float *X, int64_t n, int32_t dim, float *D, int64_t ld,
                            cudaStream_t s);
// Copy a caller distance matrix (stride n) into D (stride ld), validating it.
void launch_copy_validate_distances(const float *src, int64_t n, float *D, int64_t ld,
                                    DevState *st, cudaStream_t s);
// Enclosing radius min_i max_j D[i][j] into st->R, and st->t = min(t_user, R).
void launch_enclosing_radius(const float *D, int64_t n, int64_t ld, DevState *st,
                             float t_user, cudaStream_t s);

// Filtration construction with clearing: every cidx in [0, total) of dimension p
// is decoded, its diameter taken, and kept when diam <= st->t and its bit in
// `cleared` (may be null) is clear. Kept columns are appended (in no particular
// order) as key_hi = ~bits(diam), key_lo = cidx; st->ncols counts them.
void launch_build_columns(const float *D, int64_t ld, int64_t n, int p, const uint64_t *binom,
                          uint64_t total, const uint32_t *cleared, DevState *st,
                          uint32_t *key_hi, uint64_t *key_lo, cudaStream_t s);

// LSD radix sort of (hi, lo) keys, ascending in (hi, lo), with an optional
// 64-bit payload. Sorts lo bits [0, lo_bits) then hi bits [0, hi_bits). The
// result is left in (hi, lo, val); tmp_* are scratch of the same sizes.
// `tile_counts` needs radix_tile_counts_size(n) entries.
size_t radix_tile_counts_size(uint64_t n);
void radix_sort(uint32_t *hi, uint64_t *lo, uint64_t *val, uint32_t *tmp_hi, uint64_t *tmp_lo,
                uint64_t *tmp_val, uint32_t *tile_counts, uint32_t *digit_hist, uint64_t n,
                int lo_bits, int hi_bits, cudaStream_t s);

// radix_sort without payload and without any allocation (host_hist: caller
// buffer of 12 * 256 entries).
void radix_sort_noalloc(uint32_t *hi, uint64_t *lo, uint32_t *tmp_hi, uint64_t *tmp_lo,
                        uint32_t *tile_counts, uint32_t *digit_hist, uint32_t *host_hist,
                        uint64_t n, int lo_bits, int hi_bits, cudaStream_t s);

// Mark columns at the given positions as cleared.
void launch_mark_cleared(const uint32_t *pos, int64_t count, uint8_t *status, cudaStream_t s);

// Apparent-pair pass (Alg. 3 with the Apparent Pairs Lemma) over the columns
// [0, ncols) in coboundary order. Writes status, pivot and pivot diameter.
void launch_apparent(const float *D, int64_t ld, int64_t n, int p, const uint64_t *binom,
                     const uint32_t *key_hi, const uint64_t *key_lo, uint64_t ncols,
                     DevState *st, uint8_t *status, uint64_t *pivot, float *pdiam,
                     int group, int sms, cudaStream_t s);

// Partition: apparent columns -> (tau, sigma) pairs; leftover columns -> Leftover.
void launch_partition(const uint8_t *status, const uint32_t *key_hi, const uint64_t *key_lo,
                      const uint64_t *pivot, const float *pdiam, uint64_t ncols,
                      uint64_t *app_tau, uint64_t *app_sigma, Leftover *left, DevState *st,
                      cudaStream_t s);

// First position i in [0, n) with a[i] >= key for ascending a, into *out.
void launch_lower_bound_u32(const uint32_t *a, uint64_t n, uint32_t key, unsigned long long *out,
                            cudaStream_t s);

// Per-vertex neighbour lists: row v of out (n x n) lists all vertices in
// increasing (D[v][w], w) order, packed as (bits(D[v][w]) << 32) | w. Returns false if n is too large for the
// shared-memory sort (the caller then sorts on the host).
bool launch_sort_rows(const float *D, int64_t ld, int64_t n, uint64_t *out, cudaStream_t s);

// Set bit `idx[i]` of a bitmap for every i.
void launch_bitmap_set(const uint64_t *idx, uint64_t count, uint32_t *bitmap, cudaStream_t s);

// ---- error helpers ---------------------------------------------------------
void set_last_error(const std::string &msg);

}  // namespace rpp
