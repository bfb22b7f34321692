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
    unsigned int sort_passes[8];  // radix passes that ran in the column sort of dimension p
};

// Kernels launched by the calling thread (incremented by every launcher).
extern thread_local long long g_launches;

enum : unsigned int {
    ERR_NONFINITE = 1u,
    ERR_NEGATIVE = 2u,
    ERR_ASYMMETRIC = 4u,
    ERR_DIAGONAL = 8u,
    ERR_INTERNAL = 16u  // a kernel's bounded loop ran out (reported, never expected)
};

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
// `cleared` (may be null) is clear. Kept columns are appended as key_hi =
// ~bits(diam), key_lo = cidx; st->ncols counts them. With `order` (device
// scratch of build_order_bytes(total) bytes: per-chunk counts and offsets)
// they are written in increasing cidx and st->ncols is set to their count, so that radix_sort with lo_bits = 0 (the
// diameter digits alone) puts them in coboundary order; without it, in no
// particular order.
void launch_build_columns(const float *D, int64_t ld, int64_t n, int p, const uint64_t *binom,
                          uint64_t total, const uint32_t *cleared, DevState *st,
                          uint32_t *key_hi, uint64_t *key_lo, cudaStream_t s,
                          unsigned long long *order = nullptr);
size_t build_order_bytes(uint64_t total);

// LSD radix sort of (hi, lo) keys, ascending in (hi, lo) (hi may be null: lo
// alone), with an optional 64-bit payload; lo < 2^lo_bits. lo_bits = 0 (with
// hi): the keys arrive in increasing lo, and only hi's digits are sorted
// (every pass is stable, so lo stays increasing within equal hi). The key count is
// min(*d_count, n_cap) when d_count (device memory) is given, else n_cap, so
// the sort needs nothing from the host. The result is left in (hi, lo, val);
// tmp_* are buffers of the same sizes, scratch holds radix_scratch_bytes(n_cap)
// bytes. A bounded wait that runs out ORs ERR_INTERNAL into *err (device).
// Passes whose digit is the same for every key do no work; when passes_out
// (device memory) is given, the number of passes that did is added to it.
constexpr int RADIX_SORT_DIGIT_BITS = 9;                     // key bits sorted per pass
constexpr int RADIX_SORT_BINS = 1 << RADIX_SORT_DIGIT_BITS;  // digit values of one pass
constexpr uint64_t RADIX_SORT_TILE = 2048;                   // keys per tile of one pass
constexpr size_t RADIX_SORT_CTL_BYTES = 128 * 1024;          // the sort's control block
constexpr size_t radix_scratch_bound(uint64_t n_cap) {
    return RADIX_SORT_CTL_BYTES +
           (size_t)((n_cap + RADIX_SORT_TILE - 1) / RADIX_SORT_TILE + 1) * RADIX_SORT_BINS * 8;
}
size_t radix_scratch_bytes(uint64_t n_cap);  // = radix_scratch_bound(n_cap)
void radix_sort(uint32_t *hi, uint64_t *lo, uint64_t *val, uint32_t *tmp_hi, uint64_t *tmp_lo,
                uint64_t *tmp_val, void *scratch, uint64_t n_cap,
                const unsigned long long *d_count, int lo_bits, unsigned *err, cudaStream_t s,
                unsigned *passes_out = nullptr);

// H0 of one instance on the device: the minimum spanning forest of the edges
// inside st->t under the filtration's order of edges (Boruvka, a fixed number
// of rounds, no host round trip). mst receives the forest's keys
// (bits(d) << 32) | ~index, *nmst their count; comp, parent, next: n ints,
// best: n keys, flags: 64 words of scratch. A root search beyond its bound
// sets ERR_INTERNAL.
void launch_h0_forest(const float *D, int64_t ld, int64_t n, DevState *st, int32_t *comp,
                      int32_t *parent, int32_t *next, unsigned long long *best,
                      unsigned long long *mst, unsigned *nmst, unsigned *flags, cudaStream_t s);
// Mark the forest's columns cleared in the sorted dimension-1 array (ncols
// columns, ascending (key_hi, key_lo)); pos[i] receives the position of edge i.
// The column count is min(*d_ncols, ncols) when d_ncols (device) is given.
void launch_h0_clear(const unsigned long long *mst, const unsigned *nmst, int64_t n,
                     const uint32_t *key_hi, const uint64_t *key_lo, uint64_t ncols,
                     const unsigned long long *d_ncols, uint8_t *status, uint32_t *pos,
                     cudaStream_t s);

// out[i] = ~in[i] (sort keys ~bits(diameter) back to diameter bits).
void launch_invert_u32(const uint32_t *in, uint64_t count, uint32_t *out, cudaStream_t s);

// The vertices of edge indices, packed (a << 16) | b with a > b (n <= 65535).
void launch_edge_pairs(const uint64_t *lo, uint64_t count, uint32_t *out, cudaStream_t s);


// Apparent-pair pass (Alg. 3 with the Apparent Pairs Lemma) over the columns
// [0, ncols) in coboundary order. Writes each column's status, and its pivot
// and pivot diameter (for apparent columns only when app_piv, below).
// (ncols, d_ncols: the column count is min(*d_ncols, ncols) when d_ncols,
// device memory, is given; grids are sized for ncols.)
// aw (dimension 1, may be null): aw[edge index] = the vertex the edge's
// apparent pair adds, written for apparent columns (the caller fills 0xFFFF).
// app_piv = false: apparent columns get no pivot and pivot diameter (only
// their status and aw), for a caller that never reads their tau; leftover
// columns always get both.
void launch_apparent(const float *D, int64_t ld, int64_t n, int p, const uint64_t *binom,
                     const uint32_t *key_hi, const uint64_t *key_lo, uint64_t ncols,
                     const unsigned long long *d_ncols, DevState *st, uint8_t *status,
                     uint64_t *pivot, float *pdiam, uint16_t *aw, int group, int sms,
                     cudaStream_t s, bool app_piv = true);

// Partition: apparent columns -> (tau, sigma) pairs (app_tau and app_sigma
// both null: counted in st->napp only); leftover columns -> Leftover.
void launch_partition(const uint8_t *status, const uint32_t *key_hi, const uint64_t *key_lo,
                      const uint64_t *pivot, const float *pdiam, uint64_t ncols,
                      const unsigned long long *d_ncols, uint64_t *app_tau,
                      uint64_t *app_sigma, Leftover *left, DevState *st, cudaStream_t s);

// First position i in [0, n) with a[i] >= key for ascending a, into *out.
void launch_lower_bound_u32(const uint32_t *a, uint64_t n, uint32_t key, unsigned long long *out,
                            cudaStream_t s);

// Per-vertex neighbour lists: row v of out (n x n) lists all vertices in
// increasing (D[v][w], w) order, packed as (bits(D[v][w]) << 32) | w. Returns false if n is too large for the
// shared-memory sort (the caller then sorts on the host).
bool launch_sort_rows(const float *D, int64_t ld, int64_t n, uint64_t *out, cudaStream_t s);

// Set bit `idx[i]` of a bitmap for every i.
void launch_bitmap_set(const uint64_t *idx, uint64_t count, uint32_t *bitmap, cudaStream_t s);

// ---- thresholded (sparse 1-skeleton) construction, dimensions p >= 2 --------

// Neighbour lists of the threshold graph (D[a][w] <= st->t, w != a), ascending.
// fill = false: off[0..n] = offsets (off holds n + 1 entries); fill = true:
// nbr[off[a] .. off[a+1]) = the neighbours of a (nbr holds off[n] entries).
void launch_csr_build(const float *D, int64_t ld, int64_t n, const DevState *st,
                      unsigned long long *off, uint32_t *nbr, bool fill, cudaStream_t s);
// The p-simplices inside st->t, each found from its facet without its lowest
// vertex among the (p-1)-simplices `prev` (indices; every (p-1)-simplex inside
// t must be listed). Clearing: indices in dead_a or dead_b (sorted) are not
// columns. write = false counts into cnt[0] (simplices) and cnt[1] (columns);
// write = true appends columns (key_hi = ~bits(diam), key_lo = index; at most
// col_cap) and, if all_out is given, every simplex's index (at most all_cap),
// advancing cnt[1] and cnt[0] (zero them first).
void launch_sparse_build(const float *D, int64_t ld, int64_t n, int p, const uint64_t *binom,
                         const uint64_t *prev, uint64_t nprev, const unsigned long long *off,
                         const uint32_t *nbr, const DevState *st, const uint64_t *dead_a,
                         uint64_t ndead_a, const uint64_t *dead_b, uint64_t ndead_b, bool write,
                         unsigned long long *cnt, uint32_t *key_hi, uint64_t *key_lo,
                         uint64_t col_cap, uint64_t *all_out, uint64_t all_cap, cudaStream_t s);
// The apparent-pair pass over sorted columns of dimension p with candidates
// from the neighbour lists (same outputs as launch_apparent).
void launch_apparent_sparse(const float *D, int64_t ld, int64_t n, int p, const uint64_t *binom,
                            const unsigned long long *off, const uint32_t *nbr,
                            const uint32_t *key_hi, const uint64_t *key_lo, uint64_t ncols,
                            const unsigned long long *d_ncols, DevState *st, uint8_t *status,
                            uint64_t *pivot, float *pdiam, int sms, cudaStream_t s);

// ---- fused batch of small clouds, dimensions 0 and 1 ------------------------

constexpr int BATCH_NMAX = 1024;  // largest cloud of the fused pass

// One cloud of a fused batch.
struct BatchCloud {
    int64_t pt_off;   // offset (floats) of its points in the packed point buffer
    int64_t d_off;    // offset (floats) of its n x ld distance matrix in the scratch
    int32_t n, dim, ld;
    int32_t mst_off;  // first of its n - 1 MST slots
    float t_user;     // threshold (INFINITY: none)
    int32_t max_dim;  // 0: H0 only (no apparent-pair test)
    uint64_t qrank;   // > 0: threshold = the qrank-th smallest of the C(n,2) distances
    int64_t aw_off;   // offset of its C(n,2) entries in the apparent-vertex buffer
};

// What the fused pass reports per cloud.
struct BatchOut {
    float R, t;                 // enclosing radius, threshold in use
    uint32_t nmst, err;         // MST edges written (H0 deaths), ERR_* flags
    unsigned long long ncols;   // edges inside the threshold (MST edges included)
    unsigned long long napp, nleft, scanned;
};

// The fused pass: per cloud (one block at a time, clouds taken in `order`)
// distances, enclosing radius and threshold, the minimum spanning forest
// inside the threshold (H0, and the clearing set of dimension 1), then, when
// the cloud asks for dimension 1, the apparent-pair test of every other edge
// inside the threshold. Leftover columns are appended to `left` (cloud in
// `left_cloud`) while fewer than left_cap; ctl->left_count counts them all.
// `group` is the lane-group width of the test.
struct BatchConfig {
    int threads = 256, group = 8;  // group: G lanes per column, or 10 G + U for U blocks a step
    // blocks per SM at most (0: as many as fit): fewer clouds in flight keep
    // their distance matrices in L2 between the kernel's passes over them
    int per_sm = 0;
};
// Control block of one fused launch (device memory).
struct BatchCtl {
    unsigned int queue;               // next position in `order` (0 on entry)
    int nclouds;                      // clouds in this launch
    unsigned long long left_count;    // leftover columns found (0 on entry)
};
// Launch shape of the fused kernel for clouds of up to nmax points in up to
// dimcap dimensions; sets the kernel's shared-memory attribute. Call outside
// stream capture.
struct BatchPlan {
    int nmax = 0, dimcap = 0, blocks = 0;
    size_t smem = 0;
    BatchConfig cfg;
};
BatchPlan plan_batch_h1(int nmax, int dimcap, BatchConfig cfg, int sms);
// app_w: per cloud (from aw_off), for every edge index e < C(n,2), the vertex
// that the edge's apparent pair adds to it, or 0xFFFF if the edge is not the
// first simplex of an apparent pair (outside the threshold, cleared, leftover).
void launch_batch_h1(const BatchPlan &plan, const float *pts, const BatchCloud *clouds,
                     const int32_t *order, BatchCtl *ctl, float *Dbuf, uint64_t *mst_out,
                     BatchOut *outs, Leftover *left, int32_t *left_cloud, uint64_t left_cap,
                     uint16_t *app_w, cudaStream_t s);

// Rows of selected clouds for the host reduction: for job j (cloud c =
// jobs[j]) copy its distance matrix to Dout + out_off[j] (stride n), its
// sorted neighbour lists (as launch_sort_rows) to nbr + out_off[j], and its
// apparent vertices (app_w from the cloud's aw_off) to aw_out +
// out_off[njobs + j].
void launch_batch_rows(const float *Dbuf, const BatchCloud *clouds, const int32_t *jobs, int njobs,
                       const int64_t *out_off, int nmax, float *Dout, uint64_t *nbr,
                       const uint16_t *app_w, uint16_t *aw_out, cudaStream_t s);

// The dimension-1 reduction of small clouds' leftover columns on the device
// (reduce_small.cu), one warp per job: job i reduces the nleft leftover
// columns left[left_off .. left_off + nleft) (sorted by index) of a cloud of
// n points whose distance rows are D + d_off (stride n) and whose apparent
// vertices are aw + aw_off, inside threshold t. Per column it writes the
// death (triangle index, NO_PIVOT if essential), its diameter, and the
// column's final edge set (vcnt edges at vpool + v_off + vstart; the job's
// pool holds v_cap = reduce_small_vpool_words(nleft, n) words). status[i] is
// 0 when the job finished on the device, 1 when the host must reduce the
// cloud; adds[i] counts additions.
struct ReduceJob {
    int64_t d_off, aw_off, left_off, nleft, v_off, v_cap;
    int32_t n;
    float t;
};
constexpr int REDUCE_SMALL_NMAX = 512;  // largest cloud the device reduces
size_t reduce_small_vpool_words(uint64_t nleft, uint64_t n);
struct ReduceSmallArgs {
    const float *D = nullptr;
    const uint16_t *aw = nullptr;
    const ReduceJob *jobs = nullptr;
    int njobs = 0, nmax = 0;
    const Leftover *left = nullptr;
    uint32_t *vpool = nullptr, *vstart = nullptr, *vcnt = nullptr;
    uint64_t *death = nullptr;
    float *ddiam = nullptr;
    int32_t *status = nullptr, *adds = nullptr;
    // The second phase (clouds whose walks outgrow the cursors sweep by
    // diameter level; launch_reduce_small_sweep): its status and additions
    // per job (0 for jobs the first phase finished), room for ecap edge keys
    // in ekeys and etmp, the radix sort's scratch (radix_scratch_bytes(ecap)),
    // a key counter and an error word.
    int32_t *status_b = nullptr, *adds_b = nullptr;
    const int32_t *order_b = nullptr;  // the order the second phase takes jobs in
    unsigned *next_b = nullptr;        // its job counter
    int blocks_b = 0;                  // its blocks (0: one per SM)
    // First phase: a flag in mapped host memory (nullptr: none); once the
    // host sets it the jobs stop at their next check (status 1).
    const unsigned *cancel = nullptr;
    uint64_t *ekeys = nullptr, *etmp = nullptr;
    uint16_t *ekaw = nullptr;  // ecap entries: each sorted edge's apparent vertex
    void *escratch = nullptr;
    unsigned long long *ecount = nullptr;
    unsigned *eerr = nullptr;
    uint64_t ecap = 0;
};
// The first phase (cursors only; status 1 hands a job on).
void launch_reduce_small(const ReduceSmallArgs &a, cudaStream_t s);
// The second phase, over the jobs the first handed on (after it, in stream
// order): death, ddiam and the pool are written for those jobs only.
void launch_reduce_small_sweep(const ReduceSmallArgs &a, cudaStream_t s);

// Gather clouds given by device pointers into the packed point buffer.
void launch_gather_points(const float *const *src, const BatchCloud *clouds, int nclouds,
                          float *pts, cudaStream_t s);

// Allow kernel fn at least `bytes` of dynamic shared memory on the current
// device. The attribute belongs to the kernel, not to a launch, so callers on
// several threads must only ever raise it: a per-(device, kernel) maximum
// under a lock. Returns the error of cudaFuncSetAttribute, if any.
cudaError_t allow_dynamic_smem(const void *fn, size_t bytes);

// ---- error helpers ---------------------------------------------------------
void set_last_error(const std::string &msg);

}  // namespace rpp
