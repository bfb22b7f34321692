/*
 * rpp.h -- C ABI of the GB300 Vietoris-Rips barcode library (librpp.so).
 *
 * Computes persistence barcodes over Z/2 of the Vietoris-Rips filtration
 * Rips_s(X) = { sigma : diam(sigma) <= s }, s <= t (Sec. 2, definition of the
 * Rips filtration and of persistence pairs), following the method of
 * Zhang, Xiao, Wang, "GPU-Accelerated Computation of Vietoris-Rips Persistence
 * Barcodes" (arXiv 2003.07989):
 *   - filtration construction with clearing on the GPU (Alg. 6 and Alg. 7):
 *     every p-simplex is indexed in the combinatorial number system
 *     (Sec. "The Combinatorial Number System"), its diameter is the largest
 *     distance among its vertices, simplices above the threshold and cleared
 *     simplices are dropped, the rest are sorted by decreasing diameter then
 *     increasing index (coboundary order, Sec. "The Coboundary Matrix");
 *   - apparent pairs found with one independent test per column (Alg. 3 and
 *     the Apparent Pairs Lemma) and partitioned into a sorted pair array and
 *     the leftover columns (Fig. "post-apparent", Sec. "Core System
 *     Optimizations");
 *   - submatrix reduction of the leftover columns on the host with the
 *     two-layer pair store (hash map over the sorted apparent array) and the
 *     reduction-matrix technique (Sec. "Reduction Matrix vs. Oblivious Matrix
 *     Reduction"); H0 from the minimum spanning forest (Sec. "Zero-Dimensional
 *     Persistence Computation"; Kruskal's forest, built here by Boruvka's
 *     rounds on the GPU).
 *
 * Conventions common to every entry point:
 *   - Every call returns an rpp_status and never aborts the process. Invalid
 *     arguments are reported before any GPU work is queued. rpp_last_error()
 *     returns a thread-local message describing the last failure.
 *   - Input buffers are owned by the caller; the library never frees them.
 *     A data pointer may be device memory or host memory (pageable or pinned);
 *     the library asks the CUDA runtime which one it is. A buffer must hold
 *     the floats its sizes declare (n * dim points or n * n distances): the
 *     library cannot check its extent, and a shorter buffer is read past its
 *     end (on systems where the GPU reads host memory directly, a device
 *     memory fault).
 *   - Results are owned by the library and freed with rpp_result_free.
 *   - All GPU work of a call runs on the given CUDA stream (cudaStream_t passed
 *     as void*; NULL means the legacy default stream). A call returns after its
 *     results are complete on the host.
 *   - Distances are float32. Diameters and interval endpoints are exact
 *     distance-matrix entries; there is no rounding of the filtration order.
 *   - Ordering of simplices (the simplex-wise refinement, Sec. "The Simplex-wise
 *     Refinement"): increasing diameter, then increasing dimension, then
 *     decreasing combinatorial index.
 *   - A context may be used from several threads; calls on one context are
 *     serialised internally per workspace.
 */
#ifndef RPP_H
#define RPP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RPP_OK = 0,
    RPP_E_INVALID = 1,   /* bad argument or input (non-finite, negative, asymmetric ...) */
    RPP_E_NOMEM = 2,     /* device or host allocation failed, or the budget is exceeded */
    RPP_E_OVERFLOW = 3,  /* an index does not fit: C(n, max_dim + 2) the 63-bit simplex
                            index, or C(n, 2) the 32-bit edge index (n > 92682) */
    RPP_E_CUDA = 4,      /* a CUDA runtime call failed (message in rpp_last_error) */
    RPP_E_TIMEOUT = 5,   /* a bounded wait ran out (poll deadline, device wait limit) */
    RPP_E_BUSY = 6       /* admission refused: no slot or memory free right now */
} rpp_status;

typedef enum {
    RPP_INPUT_POINTS = 0,    /* data is n x dim float32, row-major */
    RPP_INPUT_DISTANCES = 1  /* data is n x n float32, row-major, symmetric, zero
                                diagonal, non-negative, finite */
} rpp_input_kind;

/* One persistence interval [birth, death); death = +INFINITY for an essential
 * class. Zero-length intervals are never reported. */
typedef struct {
    float birth, death;
} rpp_interval;

/* The edges that realise an interval's endpoints: (bu, bv) is the youngest
 * edge of the birth simplex (its longest edge; ties broken by the filtration
 * order), (du, dv) the youngest edge of the death simplex. -1 where there is
 * none (H0 births, essential deaths). */
typedef struct {
    int32_t bu, bv, du, dv;
} rpp_critical;

#define RPP_MAX_DIM 4

/* Per-call counters and stage times. Index p of the arrays is the column
 * dimension p (p = 1 .. max_dim). */
typedef struct {
    int64_t n;
    int32_t max_dim;
    float threshold;                     /* the threshold actually used */
    float enclosing_radius;
    int64_t candidates[RPP_MAX_DIM + 1];  /* C(n, p+1) */
    int64_t columns[RPP_MAX_DIM + 1];     /* columns after threshold and clearing */
    int64_t cleared[RPP_MAX_DIM + 1];     /* columns removed by clearing */
    int64_t apparent[RPP_MAX_DIM + 1];    /* apparent pairs (sigma of dim p) */
    int64_t leftover[RPP_MAX_DIM + 1];    /* columns handed to the submatrix reduction */
    int64_t free_pivot[RPP_MAX_DIM + 1];  /* leftover columns whose first pivot was free */
    int64_t additions[RPP_MAX_DIM + 1];   /* column additions in the submatrix reduction */
    int64_t store_reads[RPP_MAX_DIM + 1]; /* pair-store lookups in the reduction */
    int64_t entries[RPP_MAX_DIM + 1];     /* coboundary entries the reduction examined */
    int64_t intervals[RPP_MAX_DIM + 1];   /* nonzero intervals reported (index 0 = H0) */
    int64_t scanned[RPP_MAX_DIM + 1];     /* candidate vertices a sequential apparent test
                                             examines up to its exit, summed over columns */
    int64_t sweep_levels[RPP_MAX_DIM + 1]; /* diameter levels swept by long dimension-1 walks */
    int64_t kernel_launches;              /* CUDA kernels this call launched */
    /* Per-stage device time from CUDA events on the call's stream, filled when
     * the context records RPP_RECORD_TIMING: 0 distances, 1 enclosing radius,
     * 2 filtration (build), 3 column sort, 4 apparent-pair pass, 5 partition,
     * 6 pair sort, 7 other small kernels. */
    double stage_ms[8];
    int64_t stage_launches[8];
    double ms_device;                     /* wall time spent waiting on the GPU */
    double ms_host_reduce;                /* wall time of the submatrix reductions */
    double ms_host_h0;                    /* wall time of the H0 stage (forest, intervals) */
    double ms_total;
    int64_t sparse[RPP_MAX_DIM + 1];      /* 1 where dimension p's columns were built as cliques
                                             of the threshold graph (rpp_context_set_sparse) */
    int64_t sweep_pivots[RPP_MAX_DIM + 1]; /* nonzero entries the level sweeps found (each
                                             then added an owner or ended its walk) */
    int64_t sweep_idle[RPP_MAX_DIM + 1];  /* level tests passed at once: no edge of the walk's
                                             set at either end of the level's edge */
    double ms_sweep_walks;                /* wall time of the walks that swept, summed over
                                             walks (they may overlap in time) */
    int64_t device_columns[RPP_MAX_DIM + 1]; /* leftover columns reduced on the device
                                             (batched clouds of <= 512 points) */
    int64_t sort_passes[RPP_MAX_DIM + 1]; /* radix passes the column sort of dimension p ran:
                                             9-bit digit positions of the key that were not
                                             the same for every column (others are skipped) */
} rpp_stats;

typedef struct rpp_context rpp_context;
typedef struct rpp_result rpp_result;

/* Create a context on CUDA device `device`. mem_budget_bytes bounds the device
 * workspace the context may hold (0 = no bound). Allocation is lazy. */
rpp_status rpp_context_create(int device, size_t mem_budget_bytes, rpp_context **out);
void rpp_context_destroy(rpp_context *ctx);

/* Barcodes of dimensions 0..max_dim of Rips_t.
 *   data       points (n x dim) or distances (n x n), float32, device or host.
 *   kind       RPP_INPUT_POINTS or RPP_INPUT_DISTANCES (dim ignored).
 *   n          number of points, 1 <= n <= 92682 (C(n, 2) < 2^32).
 *   max_dim    0 <= max_dim <= RPP_MAX_DIM.
 *   threshold  closed threshold t >= 0; +INFINITY means the full filtration.
 *              The enclosing radius R bounds the work: min(t, R) is used,
 *              which leaves every nonzero interval unchanged (Proposition in
 *              Sec. "Filtering Out Simplices by Diameter Equal to the
 *              Enclosing Radius").
 *   stream     cudaStream_t or NULL.
 *   out        receives a result handle on success.
 * Errors: RPP_E_INVALID, RPP_E_OVERFLOW, RPP_E_NOMEM, RPP_E_CUDA. */
rpp_status rpp_barcodes(rpp_context *ctx, const float *data, rpp_input_kind kind, int64_t n,
                        int32_t dim, int32_t max_dim, float threshold, void *stream,
                        rpp_result **out);

/* As rpp_barcodes, with the threshold given as the nearest-rank quantile q in
 * (0, 1] of the C(n,2) pairwise distances (the ceil(q * C(n,2))-th smallest
 * distance). */
rpp_status rpp_barcodes_quantile(rpp_context *ctx, const float *data, rpp_input_kind kind,
                                 int64_t n, int32_t dim, int32_t max_dim, double quantile,
                                 void *stream, rpp_result **out);

/* Apparent-pair census of dimension 1 (Sec. "Experiments on the Apparent
 * Pairs Rate" and its figure of the apparent fraction): on the full
 * filtration (every edge: neither a threshold nor the enclosing radius cuts
 * it) the edges are built and sorted, Kruskal's merging edges are cleared,
 * and the apparent-pair pass (Alg. 3) tests every other edge; the submatrix
 * reduction does not run. On success *out (caller-owned) holds
 * candidates[1] = C(n,2) edges, cleared[1] (merging edges), apparent[1] and
 * leftover[1] (cleared + apparent + leftover = C(n,2)) and the stage times;
 * the apparent fraction of the paper's figure is apparent[1] / C(n,2).
 * data, kind, n, dim and stream as in rpp_barcodes.
 * Errors: RPP_E_INVALID, RPP_E_OVERFLOW, RPP_E_NOMEM, RPP_E_CUDA. */
rpp_status rpp_apparent_census(rpp_context *ctx, const float *data, rpp_input_kind kind,
                               int64_t n, int32_t dim, void *stream, rpp_stats *out);

/* The filtration construction of one dimension on its own (Alg. 6 and Alg.
 * 7 without clearing, Sec. "Filtration Construction with Clearing"): every
 * p-simplex with diameter <= min(threshold, R), R the enclosing radius, in
 * coboundary order (decreasing diameter, then increasing combinatorial index,
 * Sec. "The Coboundary Matrix"). Columns are built on the device and sorted
 * there by the library's radix sort.
 *   data, kind, n, dim, threshold, stream  as in rpp_barcodes; n >= p + 1.
 *   p          1 <= p <= RPP_MAX_DIM; C(n, p+1) candidates must not exceed
 *              2^32 (RPP_E_NOMEM otherwise).
 *   diam_out, cidx_out  caller-owned arrays (device or host memory) of
 *              `capacity` entries receiving the diameters and indices, or
 *              both NULL to leave the columns in the context's workspace
 *              (for timing: only the count and the counters come back).
 *   count_out  receives the number of columns (also when capacity is short).
 *   stats_out  optional: candidates[p], columns[p], threshold,
 *              enclosing_radius, stage_ms (with RPP_RECORD_TIMING),
 *              kernel_launches, ms_total.
 * Errors: RPP_E_INVALID (arguments, invalid distances, capacity below the
 * count), RPP_E_OVERFLOW, RPP_E_NOMEM, RPP_E_CUDA. */
rpp_status rpp_filtration(rpp_context *ctx, const float *data, rpp_input_kind kind, int64_t n,
                          int32_t dim, int32_t p, float threshold, void *stream, float *diam_out,
                          uint64_t *cidx_out, int64_t capacity, int64_t *count_out,
                          rpp_stats *stats_out);

/* Number of intervals of dimension p (0 <= p <= max_dim) in a result. */
int64_t rpp_result_count(const rpp_result *res, int32_t p);
/* Intervals of dimension p, host memory owned by the result, sorted by
 * (birth, death). */
const rpp_interval *rpp_result_intervals(const rpp_result *res, int32_t p);
/* Realising edges, parallel to rpp_result_intervals. */
const rpp_critical *rpp_result_critical(const rpp_result *res, int32_t p);
rpp_status rpp_result_stats(const rpp_result *res, rpp_stats *out);
void rpp_result_free(rpp_result *res);

/* The same accessors over many results at once (e.g. the out[] of
 * rpp_barcodes_batched), so that a caller pays one call per array rather
 * than one per result.
 *   rpp_results_gather: the dimension-p intervals and realising edges of
 *     results[0..count-1], result after result, into caller-owned host
 *     arrays. offsets[0..count] (caller-owned) receives where each result's
 *     entries start (offsets[count] = total); a result without dimension p
 *     contributes none. With intervals and critical both NULL only offsets
 *     are written, to size the arrays; otherwise each non-NULL array must
 *     hold offsets[count] entries.
 *   rpp_results_stats: out[i] = the counters of results[i].
 *   rpp_results_free: rpp_result_free of every non-NULL entry.
 * Errors: RPP_E_INVALID for a NULL array, a NULL result, count < 0 or p
 * outside [0, RPP_MAX_DIM]; nothing is written then. */
rpp_status rpp_results_gather(const rpp_result *const *results, int32_t count, int32_t p,
                              int64_t *offsets, rpp_interval *intervals, rpp_critical *critical);
rpp_status rpp_results_stats(const rpp_result *const *results, int32_t count, rpp_stats *out);
void rpp_results_free(rpp_result *const *results, int32_t count);

/* Many independent clouds in one call (the batched form of the paper's
 * computation; the paper itself runs one distance matrix at a time).
 * Clouds of at most 1024 points with max_dim <= 1 run together in one fused
 * launch per size bucket (64, 128, 256, 512, 1024 points): each block of the
 * launch takes a whole cloud through its distance matrix, enclosing radius and
 * threshold, H0 by a minimum spanning forest, and the apparent-pair test of its
 * edges; the launch is a captured CUDA graph and its shape is chosen per
 * bucket by the context's autotuner. Host reductions of the clouds with
 * leftover columns run on the library's host threads. Other clouds (larger,
 * max_dim >= 2, or a context recording columns or pairs) run one at a time.
 * Results are identical to rpp_barcodes on each cloud alone.
 *   data[i]       points of cloud i (n[i] x dim[i] float32, row-major), device
 *                 or host memory, owned by the caller.
 *   thresholds    per cloud threshold (+INFINITY = full), or NULL for all full.
 *   quantiles     per cloud quantile in (0,1] overriding the threshold, or NULL.
 *   stream        CUDA stream for every copy and launch (NULL: legacy stream).
 *   out[i]        result of cloud i (free each with rpp_result_free, or all of
 *                 them with rpp_results_free; rpp_results_gather copies them).
 * Errors: RPP_E_INVALID (a cloud's arguments, or non-finite coordinates),
 * RPP_E_NOMEM, RPP_E_CUDA. On error no result is returned. */
rpp_status rpp_barcodes_batched(rpp_context *ctx, int32_t batch, const float *const *data,
                                const int64_t *n, const int32_t *dim, int32_t max_dim,
                                const float *thresholds, const double *quantiles, void *stream,
                                rpp_result **out);

/* Batch behaviour of a context. fused = 0 runs every cloud of a batch through
 * the one-at-a-time pipeline (for comparisons); autotune = 0 keeps the default
 * launch shapes for size buckets not yet tuned: 256 threads and 8 lanes per
 * column in the fused pass, and in the single-instance apparent pass 4 lanes
 * with 2 (n <= 256) or 4 candidate blocks a step. With autotune = 1 the first
 * instance of a bucket times the candidate shapes on its own columns (every
 * shape gives the same results). Both default to 1. Errors: RPP_E_INVALID for
 * a NULL context. */
rpp_status rpp_context_set_batch(rpp_context *ctx, int32_t fused, int32_t autotune);

/* How dimensions p >= 2 are built (Sec. "Computation Induced by Sparse
 * 1-Skeletons"). With a threshold t far below the enclosing radius most of the
 * C(n, p+1) indices name simplices with an edge longer than t; the thresholded
 * construction instead lists the cliques of the graph of edges inside t
 * (every p-simplex from its facet without its lowest vertex and a common
 * neighbour below it), clears by binary search in the previous dimension's
 * sorted deaths, and tests apparent pairs over neighbour lists only. Both
 * constructions give the same columns and barcodes.
 *   mode 0 (default): thresholded when fewer than a quarter of the C(n, 2)
 *          edges lie inside t, or when C(n, p+1) >= 2^32;
 *   mode 1: always thresholded; mode 2: never (C(n, p+1) >= 2^32 then fails
 *          with RPP_E_NOMEM).
 * Errors: RPP_E_INVALID for a NULL context or another mode. */
rpp_status rpp_context_set_sparse(rpp_context *ctx, int32_t mode);

/* Where the batched clouds' leftover columns of dimension 1 are reduced
 * (Alg. 1, the submatrix reduction of Sec. "Core System Optimizations").
 * Clouds of up to 512 points in a fused launch can be reduced on the device,
 * one warp per cloud in column order, on a stream of the library's own that
 * starts after the fused pass and runs beside the host reductions and the
 * next launch's pass. A first phase walks each column with lazy cursors over
 * its edges' cofacets and hands on a cloud whose column needs more than 64
 * additions or sums more than 64 edges; a second phase (mode 2) redoes those
 * clouds, letting such a column go on as a sweep over the diameter levels of
 * the cloud's sorted edges.
 * mode = 1: the first phase only. The host threads take the clouds
 * the device does not reduce first, then the others heaviest first; a thread
 * reaching a cloud whose device result is on the host uses it, and otherwise
 * reduces the cloud itself; once every cloud has its pairs the host raises
 * a flag that stops the device's jobs, and the workspace's next launch waits
 * for them.
 * mode = 2: both phases, and the host waits for the device's result of every
 * cloud it sent there (a cloud whose sweep meets a level of more than 32
 * equal edges, or whose final edge sets outgrow its pool, is still reduced on
 * the host).
 * mode = 0 (default): every cloud is reduced on the host only.
 * All modes give the same barcodes and realising edges; rpp_stats.
 * device_columns counts the columns whose pairs came from the device.
 * Errors: RPP_E_INVALID for a NULL context or another mode. */
rpp_status rpp_context_set_device_reduce(rpp_context *ctx, int32_t mode);

/* The launch shape the autotuner chose for the bucket of clouds with up to
 * nmax points (64, 128, 256, 512 or 1024): threads per block and the
 * apparent-pair test's shape, G lanes per column testing one block of G
 * candidates a step (group = G) or U blocks (group = 10 G + U); both 0 if the
 * bucket has not run yet.
 * Errors: RPP_E_INVALID for a NULL argument. */
rpp_status rpp_context_batch_tuning(rpp_context *ctx, int32_t nmax, int32_t *threads,
                                    int32_t *group);

/* Backward of the interval endpoints to the point coordinates.
 * For every finite interval of dimension p >= 0 of result i, with birth edge
 * (u, v) and death edge (u', v'):
 *   grad_points[u]  += g_birth * (x_u - x_v) / |x_u - x_v|, grad_points[v] -= same,
 *   grad_points[u'] += g_death * (x_u' - x_v') / |x_u' - x_v'|, grad_points[v'] -= same.
 * (An endpoint is a distance |x_u - x_v|; this is its gradient.)
 *   points       device, batch clouds stored back to back (cloud i at offset
 *                sum_{j<i} n[j] * dim), float32.
 *   results      the forward results, one per cloud (points input, same dim).
 *   grad_birth, grad_death  device float32, one entry per interval of every
 *                cloud, concatenated in (cloud, dimension, interval) order;
 *                entries of essential deaths are ignored.
 *   grad_points  device float32, same layout as points, overwritten.
 * Zero-length intervals are not in the result, so they receive no gradient. */
rpp_status rpp_barcodes_backward(rpp_context *ctx, int32_t batch, const float *points,
                                 const int64_t *n, int32_t dim,
                                 const rpp_result *const *results, const float *grad_birth,
                                 const float *grad_death, float *grad_points, void *stream);

/* Total interval count of a result over dimensions 0..max_dim. */
int64_t rpp_result_total(const rpp_result *res);

/* The distance matrix of points with the library's fixed float32 formula
 * (Sec. 2: D[i,j] = d(point i, point j), D[i,i] = 0; per pair, s = 0,
 * s = s + (x_k - y_k)^2 for k = 0..dim-1 rounded to nearest without fused
 * multiply-add, then a correctly rounded square root).
 *   points  n x dim float32, device or host.
 *   out     n x n float32 row-major, device or host, caller-owned, overwritten. */
rpp_status rpp_distance_matrix(rpp_context *ctx, const float *points, int64_t n, int32_t dim,
                               float *out, void *stream);

/* ---- the edge filtration without any device allocation ----
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc: code running inside another runtime's device
 * memory pool, where all allocations must go through that owner, and
 * latency-critical loops, where cudaMalloc or cudaFree would synchronise the
 * device. It computes the dimension-1 columns of the library's filtration
 * construction without clearing: every edge with diameter <= threshold,
 * sorted by decreasing diameter, then increasing combinatorial index.
 *   D          device, n x n float32 row-major distance matrix (symmetric,
 *              finite, non-negative, zero diagonal, no -0.0; not checked).
 *   n          1 <= n <= 724.
 *   threshold  closed threshold t >= 0 (+INFINITY: every edge).
 *   diam_out, cidx_out  device arrays of `capacity` entries, caller-owned;
 *              the first *count_out entries are overwritten with the result.
 *   capacity   must be >= C(n, 2).
 *   count_out  host, receives the number of edges written.
 * It allocates nothing: its scratch is one static device array of about
 * 3.8 MB (up to 262,144 edges) that every GPU loading the library holds until
 * the process exits. The first call on a device may be the one that loads the
 * library's device code there, and so the one that places that array on the
 * device; make that first call before any stream capture. Every call looks up
 * the array's device address for the current device. All calls share the
 * array, so calls that overlap on the GPU (other streams, other threads) race
 * and must be serialised by the caller. Returns RPP_E_INVALID for n above the
 * bound, a short capacity, D or an output not in memory of the current
 * device, or a stream of another device; RPP_E_CUDA if a CUDA call fails.
 * Waits for its stream before returning. */
rpp_status rpp_filtration_edges_noalloc(const float *D, int64_t n, float threshold,
                                        float *diam_out, uint64_t *cidx_out, int64_t capacity,
                                        int64_t *count_out, void *stream);

/* ---- measurement: the L2 read-bandwidth ceiling ----
 *
 * Not a step of the method. The apparent-pair pass (Alg. 3) reads distance
 * rows that stay in L2 (a 2000-point matrix is 16 MB), so the roofline that
 * bounds its loads is the L2's read bandwidth, not HBM's. This call queues
 * one kernel that reads the `bytes` bytes at buf `reps` times with loads
 * cached in L2 only (never served by L1), over `blocks` blocks of 512
 * threads, and adds the sum of every 32-bit word it read (mod 2^32, i.e.
 * reps times the buffer's word sum) to *sink. The caller times the launch on
 * its stream; with a buffer that fits in L2 and one launch before to bring
 * it there, bytes * reps / time is the L2 read bandwidth.
 *   buf     device memory of the current device, 16-byte aligned; read only.
 *   bytes   a positive multiple of 16.
 *   reps    1 <= reps <= 2^20.
 *   blocks  1 <= blocks <= 65535.
 *   sink    device memory of the current device, one uint32_t, 4-byte
 *           aligned; the caller zeroes it.
 *   stream  cudaStream_t of the current device, or NULL.
 * Does not wait for the stream. Errors: RPP_E_INVALID (a NULL, misaligned or
 * non-device pointer, a size, reps or blocks out of range, a stream of
 * another device), RPP_E_CUDA (the launch failed). */
rpp_status rpp_l2_read_probe(const void *buf, size_t bytes, int32_t reps, int32_t blocks,
                             uint32_t *sink, void *stream);

/* ---- recording of intermediate arrays (inspection and parity checks) ---- */

#define RPP_RECORD_COLUMNS 1  /* keep each dimension's column array */
#define RPP_RECORD_APPARENT 2 /* keep each dimension's apparent pairs */
#define RPP_RECORD_TIMING 4   /* time each stage with CUDA events (rpp_stats.stage_ms) */

/* Make later calls on ctx copy the selected intermediate arrays into their
 * results (0 turns recording off). Costs host memory and copy time. */
rpp_status rpp_context_set_record(rpp_context *ctx, int32_t flags);

/* The columns of dimension p (p >= 1) after the threshold and clearing, in
 * coboundary order: decreasing diameter, then increasing combinatorial index
 * (the output of Alg. 7). Sets *diam and *cidx to arrays owned by the result
 * and returns their length, or -1 if the result did not record them. */
int64_t rpp_result_columns(const rpp_result *res, int32_t p, const float **diam,
                           const uint64_t **cidx);

/* The apparent pairs (sigma of dimension p, tau of dimension p+1) found by the
 * apparent-pair pass (Alg. 3), sorted by tau (the second layer of the pair
 * store). Returns their number, or -1 if the result did not record them. */
int64_t rpp_result_apparent(const rpp_result *res, int32_t p, const uint64_t **sigma,
                            const uint64_t **tau);

/* ---- serving: continuous batching of requests that arrive over time ---- */

typedef struct rpp_server rpp_server;

typedef struct {
    int32_t max_slots;          /* requests in flight on the device at once */
    size_t device_bytes;        /* device memory the admitted requests may hold */
    int32_t host_threads;       /* threads for the host reductions (0 = auto) */
    int32_t max_batch;          /* most requests one slot takes into one fused batch
                                   (rpp_barcodes_batched); <= 1: one request per slot */
} rpp_server_config;

rpp_status rpp_server_create(rpp_context *ctx, const rpp_server_config *cfg, rpp_server **out);
/* Submit one request (points copied at submission, host or device memory).
 * Returns RPP_E_BUSY if the request alone can never fit the memory bound. */
rpp_status rpp_server_submit(rpp_server *srv, const float *points, int64_t n, int32_t dim,
                             int32_t max_dim, float threshold, double quantile,
                             uint64_t *ticket);
/* Wait up to timeout_ms (< 0: forever) for a request; RPP_E_TIMEOUT if not done. */
rpp_status rpp_server_poll(rpp_server *srv, uint64_t ticket, int32_t timeout_ms,
                           rpp_result **out);
/* The next finished request in completion order (a completion queue): its
 * ticket into *ticket and its result into *out, as rpp_server_poll would give
 * for that ticket (a request already taken by rpp_server_poll is skipped).
 * Waits up to timeout_ms (< 0: with no bound) for one to finish; returns
 * RPP_E_TIMEOUT if none did. With every submitted request already taken and
 * timeout_ms < 0 it waits for the next submission's completion. */
rpp_status rpp_server_next(rpp_server *srv, int32_t timeout_ms, uint64_t *ticket,
                           rpp_result **out);
/* Drain every outstanding request and stop the worker threads. */
void rpp_server_destroy(rpp_server *srv);

const char *rpp_status_string(rpp_status s);
const char *rpp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RPP_H */
