// host.h -- host-side stages of the pipeline: the submatrix reduction of the
// leftover columns, and barcode assembly helpers.
#pragma once

#include <stdint.h>

#include <functional>
#include <unordered_map>
#include <vector>

#include "../../include/rpp.h"
#include "internal.h"

namespace rpp {

// Read-only view of one instance for the host stages.
struct HostInstance {
    int64_t n = 0;
    const float *D = nullptr;     // host copy, row stride ld
    int64_t ld = 0;
    const Binomial *B = nullptr;
    const uint64_t *nbr = nullptr;  // n x n neighbour lists: (bits(distance) << 32) | vertex, sorted
    // apparent pivots (tau) of the current dimension, sorted; null: apparent
    // pairs are recognised by testing them again
    const uint64_t *app_tau = nullptr;
    uint64_t napp = 0;
    // dimension 1, instead of app_tau (may be null): for every edge index, the
    // vertex its apparent pair adds to it, 0xFFFF if it has none
    const uint16_t *app_w = nullptr;
    // dimension 1 only (n <= 65535): every edge inside the threshold in
    // coboundary order (diameter descending, index ascending), as the GPU
    // sorted them: its vertices packed as (a << 16) | b, a > b, and
    // ~bits(diameter); null: the reduction sorts them itself if a walk sweeps
    const uint32_t *edge_ab = nullptr;
    const uint32_t *edge_hi = nullptr;
    int64_t nedges = 0;
    float t = 0.0f;                 // threshold in use
    float dist(int a, int b) const { return D[(int64_t)a * ld + b]; }
};

// Vertices v[0] > ... > v[p] of a p-simplex index.
void decode_host(const Binomial &B, uint64_t c, int p, int64_t n, int *v);
// Index of the p-simplex with vertices v[0] > ... > v[p].
uint64_t index_host(const Binomial &B, const int *v, int p);
// Youngest edge of a simplex (largest distance; ties: smallest edge index),
// returned as (u, w) with u > w.
void youngest_edge(const HostInstance &I, const int *v, int k, int32_t *u, int32_t *w);

// One persistence pair found on the host (or an essential class, tau = NO_PIVOT).
struct HostPair {
    uint64_t sigma, tau;
    float birth, death;
};

// ---- submatrix reduction ----------------------------------------------------
struct ReduceStats {
    int64_t free_pivot = 0, additions = 0, reads = 0, entries = 0, levels = 0;
    // sweeps of long dimension-1 walks: pivots found level by level, level
    // tests passed with no edge of V at either end, and the wall time of the
    // walks that swept (summed over walks, which may overlap in time)
    int64_t sweep_pivots = 0, sweep_idle = 0;
    double sweep_walk_ms = 0.0;
};

// Run fn(0) .. fn(count - 1) on the library's persistent host threads, the
// caller included (serially when threads <= 1). Calls may nest.
void parallel_for(int threads, int64_t count, const std::function<void(int64_t)> &fn);

// Reduce the leftover columns of dimension p (given in coboundary order) and
// append their pairs (zero-length included) and essential classes to out.
// The pair store has two layers (Sec. "Core System Optimizations"): pairs
// found here live in a hash map; apparent pairs are the array of their taus
// sorted on the GPU, searched through a small in-cache index. The owner of an
// apparent tau is its youngest facet (the definition of an apparent pair), so
// only the taus are needed.
void reduce_leftovers(const HostInstance &I, int p, const Leftover *left, int64_t nleft,
                      int threads, std::vector<HostPair> &out, ReduceStats &stats);

}  // namespace rpp
