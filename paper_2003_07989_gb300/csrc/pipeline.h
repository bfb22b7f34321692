// pipeline.h -- device workspaces and the per-instance barcode pipeline.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/rpp.h"
#include "host.h"
#include "internal.h"

namespace rpp {

// A grow-only device buffer.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// A grow-only pinned host buffer.
struct HostBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct Status {
    rpp_status code = RPP_OK;
    std::string msg;
    bool ok() const { return code == RPP_OK; }
};

#define RPP_CK(call)                                                                  \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            ::rpp::Status st_;                                                        \
            st_.code = RPP_E_CUDA;                                                    \
            st_.msg = std::string(#call) + ": " + cudaGetErrorString(e_) + " (" +     \
                      ::rpp::source_name(__FILE__) + ":" + std::to_string(__LINE__) + ")"; \
            return st_;                                                               \
        }                                                                             \
    } while (0)

#define RPP_TRY(expr)                 \
    do {                              \
        ::rpp::Status s_ = (expr);    \
        if (!s_.ok()) return s_;      \
    } while (0)

double now_ms();
// The file name of a source path (for error messages).
inline const char *source_name(const char *path) {
    const char *b = path;
    for (const char *p = path; *p; ++p)
        if (*p == '/') b = p + 1;
    return b;
}
int bits_for(uint64_t x);  // bits needed to write x (0 for x = 0)
// Nearest rank of the q-quantile among the C(n, 2) distances: ceil(q C(n, 2)),
// clamped to [1, C(n, 2)].
uint64_t quantile_rank(double q, uint64_t n);
Status fail(rpp_status code, const std::string &msg);
float bits_to_float(uint32_t b);

// Everything one in-flight instance needs. A context keeps a pool of these.
struct Workspace {
    int device = 0;
    size_t budget = 0;        // 0 = unbounded
    size_t device_bytes = 0;  // currently held
    DevBuf X, Dsrc, D, state, state_tune, binom, key_hi, key_lo, tmp_hi, tmp_lo, tmp_val, tiles, hist,
        status, pivot, pdiam, app_tau, app_sigma, left, bitmap, mst, up, nbr, h0;
    DevBuf csr_off, csr_nbr, sp_a, sp_b, sp_c, sp_cnt;  // the thresholded construction
    DevBuf aw;    // dimension 1: the vertex each edge's apparent pair adds
    DevBuf order; // the ordered filtration build's ticket and look-back counts
    HostBuf h_aw;
    HostBuf h_hi, h_lo, h_tau, h_sigma, h_left, h_D, h_state, h_mst, h_up, h_nbr, h_ehi, h_eab;
    Binomial binom_host;      // cached table
    int64_t binom_n = -1;
    int binom_k = -1;
    bool binom_on_device = false;
    std::vector<uint64_t> binom_store;
    std::vector<cudaEvent_t> events;  // pool for stage timing
    // the fused batch pass (batch.cpp)
    DevBuf b_aw, b_awout;
    DevBuf b_pts, b_clouds, b_order, b_ctl, b_D, b_mst, b_outs, b_left, b_lcloud, b_jobs, b_off,
        b_Dout, b_nbr, b_src;
    HostBuf hb_awout;
    HostBuf hb_pts, hb_clouds, hb_order, hb_ctl, hb_outs, hb_mst, hb_left, hb_lcloud, hb_jobs,
        hb_off, hb_Dout, hb_nbr, hb_src;
    // the device reduction of small clouds' leftover columns
    DevBuf r_jobs, r_left, r_vpool, r_vstart, r_vcnt, r_death, r_ddiam, r_stat;
    DevBuf r_ekeys, r_etmp, r_esort, r_ekaw;  // its second phase: sorted edges, sort scratch
    HostBuf hr_in, hr_out, hr_out_b;
    HostBuf hr_cancel;  // the first phase's cancel flag (mapped: the device reads it)
    cudaStream_t reduce_stream = nullptr;  // the device reduction runs beside the next pass
    cudaEvent_t ev_rows = nullptr;         // rows of the fused launch ready
    cudaEvent_t ev_reduce = nullptr;       // the first phase's results on the host
    cudaEvent_t ev_reduce_b = nullptr;     // the second phase's
    // A cancelled first phase may still be finishing on reduce_stream: the
    // workspace's fused-launch buffers wait for ev_reduce before their next use.
    bool reduce_pending = false;
    // captured fused launches by (shape, buffer addresses), most recent last
    std::vector<std::pair<std::vector<uintptr_t>, cudaGraphExec_t>> graphs;
    cudaStream_t capture_stream = nullptr;
    ~Workspace();
    Status dev(DevBuf &b, size_t bytes, void **out);
    Status host(HostBuf &b, size_t bytes, void **out);
};

// Tunables chosen per size bucket by the autotuner (autotune.cpp).
struct Tuning {
    int group = 44;  // apparent-pair pass shape: G lanes per column, or 10 G + U for U blocks a step
};

struct Context;

// One instance request.
struct Instance {
    const float *data = nullptr;
    rpp_input_kind kind = RPP_INPUT_POINTS;
    int64_t n = 0;
    int32_t dim = 0;
    int32_t max_dim = 1;
    float threshold = INFINITY;
    double quantile = 0.0;  // > 0: threshold by quantile
    // apparent-pair census: dimension 1 of the full filtration (no threshold,
    // no enclosing-radius cut), stopping after the apparent-pair pass
    bool census = false;
};

}  // namespace rpp

// The opaque result handle.
struct rpp_result {
    int32_t max_dim = 0;
    std::vector<rpp_interval> iv[RPP_MAX_DIM + 1];
    std::vector<rpp_critical> cr[RPP_MAX_DIM + 1];
    rpp_stats stats{};
    // recorded intermediate arrays (rpp_context_set_record)
    bool has_cols[RPP_MAX_DIM + 1] = {};
    bool has_app[RPP_MAX_DIM + 1] = {};
    std::vector<float> col_diam[RPP_MAX_DIM + 1];
    std::vector<uint64_t> col_idx[RPP_MAX_DIM + 1];
    std::vector<uint64_t> app_sigma[RPP_MAX_DIM + 1];
    std::vector<uint64_t> app_tau[RPP_MAX_DIM + 1];
};

struct rpp_context {
    int device = 0;
    size_t budget = 0;
    int sms = 0;
    int record = 0;  // RPP_RECORD_* flags
    int host_threads = 1;  // threads for the host reductions
    // dimensions p >= 2: 0 chooses the thresholded (clique) construction by the
    // share of edges inside t, 1 always takes it, 2 never
    int sparse_mode = 0;
    std::mutex mu;
    std::vector<rpp::Workspace *> free_ws;
    std::vector<rpp::Workspace *> all_ws;
    rpp::Tuning tuning_for(int64_t n, int p);
    rpp::Workspace *acquire();
    void release(rpp::Workspace *ws);
    // the fused batch pass: launch shape per size bucket, filled by the autotuner
    bool batch_fused = true;  // false: every cloud of a batch takes run_instance
    // fused clouds of <= 512 points reduce on the device: 0 never; 1 beside
    // the host reductions, short walks only (the host takes what the device
    // has finished when it reaches a cloud); 2 every walk, long ones as level
    // sweeps (the host waits for the device's results)
    int device_reduce = 0;
    bool autotune = true;
    std::mutex tune_mu;
    std::map<int, rpp::BatchConfig> batch_tuning;  // bucket nmax -> chosen shape
    // the single-instance apparent pass: (p, size bucket) -> launch shape
    std::map<std::pair<int, int64_t>, int> apparent_tuning;
};

namespace rpp {

// Below this share of the C(n, 2) edges inside the threshold, dimensions
// p >= 2 are built as cliques of the threshold graph (sparse.cu).
constexpr double SPARSE_DENSITY = 0.25;

// Run one instance end to end on `stream` with workspace `ws`.
Status run_instance(rpp_context *ctx, Workspace &ws, const Instance &in, cudaStream_t stream,
                    rpp_result *res);
// Run validated instances as one batch (fused pass where eligible, batch.cpp);
// out[i] receives instance i's result. On error no result is left in out.
// ws2 (optional, another workspace of the context): fused launches overlap,
// the device work of one with the host reductions of the one before.
Status run_batch(rpp_context *ctx, Workspace &ws, const std::vector<Instance> &ins,
                 cudaStream_t stream, rpp_result **out, Workspace *ws2 = nullptr);
// Whether run_batch takes this instance through the fused pass.
bool batch_fused_eligible(const rpp_context *ctx, const Instance &in);
// The fused launch an eligible instance joins (size bucket and dimension
// capacity): instances of one bucket share a launch.
int64_t batch_bucket(const Instance &in);
// Device bytes a workspace holds after run_batch over these fused-eligible
// instances (an upper bound).
size_t batch_device_bytes(const std::vector<Instance> &ins);
// Device bytes a workspace holds after running this instance.
// rpp_filtration: dimension p's columns without clearing, built and sorted.
Status run_filtration(rpp_context *ctx, Workspace &ws, const Instance &in, int p, cudaStream_t s,
                      float *diam_out, uint64_t *cidx_out, int64_t capacity, int64_t *count,
                      rpp_stats &S);
size_t instance_device_bytes(const Instance &in);
// Validate an instance before any GPU work.
Status validate_instance(const Instance &in);
// Fill a binomial table C(v, k), k <= kmax, v <= n (saturating).
void fill_binomial(int64_t n, int kmax, std::vector<uint64_t> &store, Binomial &B);
bool is_device_pointer(const void *p);
// Record a failed status as the thread's last error and return its code.
rpp_status report(const Status &s);
// Append an interval of dimension q with its realising edges.
void add_interval(rpp_result *res, int q, float b, float d, const rpp_critical &c);
// Sort the intervals of dimension q by (birth, death, realising edges).
void sort_result(rpp_result *res, int q);

}  // namespace rpp
