// api.cpp -- the C ABI declared in include/rpp.h: contexts, single-instance
// barcodes, result accessors, status strings.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>

#include "pipeline.h"

namespace rpp {

namespace {
thread_local std::string g_last_error;
}

thread_local long long g_launches = 0;

void set_last_error(const std::string &msg) { g_last_error = msg; }

rpp_status report(const Status &s) {
    if (!s.ok()) set_last_error(s.msg);
    return s.code;
}

}  // namespace rpp

using namespace rpp;

rpp::Workspace *rpp_context::acquire() {
    std::lock_guard<std::mutex> g(mu);
    if (!free_ws.empty()) {
        Workspace *w = free_ws.back();
        free_ws.pop_back();
        return w;
    }
    Workspace *w = new Workspace();
    w->device = device;
    w->budget = budget;
    all_ws.push_back(w);
    return w;
}

void rpp_context::release(rpp::Workspace *ws) {
    std::lock_guard<std::mutex> g(mu);
    free_ws.push_back(ws);
}

extern "C" {

rpp_status rpp_context_create(int device, size_t mem_budget_bytes, rpp_context **out) {
    if (!out) {
        set_last_error("out is NULL");
        return RPP_E_INVALID;
    }
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        set_last_error(std::string("no such CUDA device: ") +
                       (e != cudaSuccess ? cudaGetErrorString(e) : std::to_string(device)));
        return RPP_E_CUDA;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        set_last_error("cudaGetDeviceProperties failed");
        return RPP_E_CUDA;
    }
    rpp_context *c = new rpp_context();
    c->device = device;
    c->budget = mem_budget_bytes;
    c->sms = prop.multiProcessorCount;
    const unsigned hw = std::thread::hardware_concurrency();
    c->host_threads = hw == 0 ? 4 : (int)std::min(hw, 32u);
    *out = c;
    return RPP_OK;
}

void rpp_context_destroy(rpp_context *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    for (Workspace *w : ctx->all_ws) delete w;
    delete ctx;
}

static rpp_status run_one(rpp_context *ctx, const Instance &in, void *stream, rpp_result **out) {
    if (!out) {
        set_last_error("out is NULL");
        return RPP_E_INVALID;
    }
    *out = nullptr;
    Status v = validate_instance(in);  // before the context: argument checks need no device
    if (!v.ok()) return report(v);
    if (!ctx) {
        set_last_error("ctx is NULL");
        return RPP_E_INVALID;
    }
    Workspace *ws = ctx->acquire();
    rpp_result *res = new rpp_result();
    Status s = run_instance(ctx, *ws, in, (cudaStream_t)stream, res);
    ctx->release(ws);
    if (!s.ok()) {
        delete res;
        return report(s);
    }
    *out = res;
    return RPP_OK;
}

rpp_status rpp_barcodes(rpp_context *ctx, const float *data, rpp_input_kind kind, int64_t n,
                        int32_t dim, int32_t max_dim, float threshold, void *stream,
                        rpp_result **out) {
    Instance in;
    in.data = data;
    in.kind = kind;
    in.n = n;
    in.dim = dim;
    in.max_dim = max_dim;
    in.threshold = threshold;
    return run_one(ctx, in, stream, out);
}

rpp_status rpp_barcodes_quantile(rpp_context *ctx, const float *data, rpp_input_kind kind,
                                 int64_t n, int32_t dim, int32_t max_dim, double quantile,
                                 void *stream, rpp_result **out) {
    Instance in;
    in.data = data;
    in.kind = kind;
    in.n = n;
    in.dim = dim;
    in.max_dim = max_dim;
    in.threshold = INFINITY;
    in.quantile = quantile;
    if (!(quantile > 0.0 && quantile <= 1.0)) {
        set_last_error("quantile must be in (0, 1]");
        return RPP_E_INVALID;
    }
    return run_one(ctx, in, stream, out);
}

rpp_status rpp_apparent_census(rpp_context *ctx, const float *data, rpp_input_kind kind,
                               int64_t n, int32_t dim, void *stream, rpp_stats *out) {
    if (!out) {
        set_last_error("out is NULL");
        return RPP_E_INVALID;
    }
    Instance in;
    in.data = data;
    in.kind = kind;
    in.n = n;
    in.dim = dim;
    in.max_dim = 1;
    in.threshold = INFINITY;
    in.census = true;
    rpp_result *res = nullptr;
    const rpp_status st = run_one(ctx, in, stream, &res);
    if (st != RPP_OK) return st;
    *out = res->stats;
    delete res;
    return RPP_OK;
}

rpp_status rpp_filtration(rpp_context *ctx, const float *data, rpp_input_kind kind, int64_t n,
                          int32_t dim, int32_t p, float threshold, void *stream, float *diam_out,
                          uint64_t *cidx_out, int64_t capacity, int64_t *count_out,
                          rpp_stats *stats_out) {
    if (!count_out) {
        set_last_error("count_out is NULL");
        return RPP_E_INVALID;
    }
    if (p < 1 || p > RPP_MAX_DIM) {
        set_last_error("p must be in [1, RPP_MAX_DIM]");
        return RPP_E_INVALID;
    }
    if ((diam_out || cidx_out) && capacity < 0) {
        set_last_error("capacity must be >= 0");
        return RPP_E_INVALID;
    }
    Instance in;
    in.data = data;
    in.kind = kind;
    in.n = n;
    in.dim = dim;
    in.max_dim = p;
    in.threshold = threshold;
    Status v = validate_instance(in);
    if (!v.ok()) return report(v);
    if (!ctx) {
        set_last_error("ctx is NULL");
        return RPP_E_INVALID;
    }
    Workspace *ws = ctx->acquire();
    rpp_stats S;
    Status st = run_filtration(ctx, *ws, in, p, (cudaStream_t)stream, diam_out, cidx_out,
                               capacity, count_out, S);
    ctx->release(ws);
    if (stats_out) *stats_out = S;
    return report(st);
}

rpp_status rpp_context_set_sparse(rpp_context *ctx, int32_t mode) {
    if (!ctx || mode < 0 || mode > 2) {
        set_last_error("rpp_context_set_sparse: NULL context or mode not in 0..2");
        return RPP_E_INVALID;
    }
    ctx->sparse_mode = mode;
    return RPP_OK;
}

int64_t rpp_result_count(const rpp_result *res, int32_t p) {
    if (!res || p < 0 || p > res->max_dim) return -1;
    return (int64_t)res->iv[p].size();
}

const rpp_interval *rpp_result_intervals(const rpp_result *res, int32_t p) {
    if (!res || p < 0 || p > res->max_dim) return nullptr;
    return res->iv[p].data();
}

const rpp_critical *rpp_result_critical(const rpp_result *res, int32_t p) {
    if (!res || p < 0 || p > res->max_dim) return nullptr;
    return res->cr[p].data();
}

int64_t rpp_result_total(const rpp_result *res) {
    if (!res) return -1;
    int64_t t = 0;
    for (int q = 0; q <= res->max_dim; ++q) t += (int64_t)res->iv[q].size();
    return t;
}

rpp_status rpp_result_stats(const rpp_result *res, rpp_stats *out) {
    if (!res || !out) {
        set_last_error("res or out is NULL");
        return RPP_E_INVALID;
    }
    *out = res->stats;
    return RPP_OK;
}

void rpp_result_free(rpp_result *res) { delete res; }

rpp_status rpp_results_gather(const rpp_result *const *results, int32_t count, int32_t p,
                              int64_t *offsets, rpp_interval *intervals, rpp_critical *critical) {
    if (count < 0 || (count > 0 && !results) || !offsets || p < 0 || p > RPP_MAX_DIM) {
        set_last_error("rpp_results_gather: invalid arguments");
        return RPP_E_INVALID;
    }
    for (int32_t i = 0; i < count; ++i)
        if (!results[i]) {
            set_last_error("rpp_results_gather: result " + std::to_string(i) + " is NULL");
            return RPP_E_INVALID;
        }
    int64_t at = 0;
    for (int32_t i = 0; i < count; ++i) {
        offsets[i] = at;
        const rpp_result *r = results[i];
        if (p > r->max_dim) continue;
        const size_t m = r->iv[p].size();
        if (intervals && m) std::memcpy(intervals + at, r->iv[p].data(), m * sizeof(rpp_interval));
        if (critical && m) std::memcpy(critical + at, r->cr[p].data(), m * sizeof(rpp_critical));
        at += (int64_t)m;
    }
    offsets[count] = at;
    return RPP_OK;
}

rpp_status rpp_results_stats(const rpp_result *const *results, int32_t count, rpp_stats *out) {
    if (count < 0 || (count > 0 && (!results || !out))) {
        set_last_error("rpp_results_stats: invalid arguments");
        return RPP_E_INVALID;
    }
    for (int32_t i = 0; i < count; ++i)
        if (!results[i]) {
            set_last_error("rpp_results_stats: result " + std::to_string(i) + " is NULL");
            return RPP_E_INVALID;
        }
    for (int32_t i = 0; i < count; ++i) out[i] = results[i]->stats;
    return RPP_OK;
}

void rpp_results_free(rpp_result *const *results, int32_t count) {
    if (!results) return;
    for (int32_t i = 0; i < count; ++i) delete results[i];
}

rpp_status rpp_context_set_record(rpp_context *ctx, int32_t flags) {
    if (!ctx || flags < 0 || flags > (RPP_RECORD_COLUMNS | RPP_RECORD_APPARENT | RPP_RECORD_TIMING)) {
        set_last_error("rpp_context_set_record: invalid arguments");
        return RPP_E_INVALID;
    }
    ctx->record = flags;
    return RPP_OK;
}

int64_t rpp_result_columns(const rpp_result *res, int32_t p, const float **diam,
                           const uint64_t **cidx) {
    if (!res || p < 1 || p > res->max_dim || !res->has_cols[p]) return -1;
    if (diam) *diam = res->col_diam[p].data();
    if (cidx) *cidx = res->col_idx[p].data();
    return (int64_t)res->col_idx[p].size();
}

int64_t rpp_result_apparent(const rpp_result *res, int32_t p, const uint64_t **sigma,
                            const uint64_t **tau) {
    if (!res || p < 1 || p > res->max_dim || !res->has_app[p]) return -1;
    if (sigma) *sigma = res->app_sigma[p].data();
    if (tau) *tau = res->app_tau[p].data();
    return (int64_t)res->app_tau[p].size();
}

rpp_status rpp_distance_matrix(rpp_context *ctx, const float *points, int64_t n, int32_t dim,
                               float *out, void *stream) {
    if (!ctx || !points || !out || n < 1 || dim < 1) {
        set_last_error("rpp_distance_matrix: invalid arguments");
        return RPP_E_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        set_last_error("rpp_distance_matrix: cudaSetDevice failed");
        return RPP_E_CUDA;
    }
    Workspace *ws = ctx->acquire();
    Status st;
    void *X = (void *)points, *D = nullptr;
    if (!is_device_pointer(points)) {
        st = ws->dev(ws->X, (size_t)n * dim * 4, &X);
        if (st.ok() && cudaMemcpyAsync(X, points, (size_t)n * dim * 4, cudaMemcpyHostToDevice, s) !=
                           cudaSuccess)
            st = Status{RPP_E_CUDA, "rpp_distance_matrix: upload failed"};
    }
    const int64_t ld = (n + 31) / 32 * 32;
    if (st.ok()) st = ws->dev(ws->D, (size_t)n * ld * 4, &D);
    if (st.ok()) {
        launch_distance_matrix((const float *)X, n, dim, (float *)D, ld, s);
        // strided copy into the caller's n x n buffer (device or host)
        cudaError_t e = cudaMemcpy2DAsync(out, (size_t)n * 4, D, (size_t)ld * 4, (size_t)n * 4,
                                          (size_t)n, cudaMemcpyDefault, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess)
            st = Status{RPP_E_CUDA, std::string("rpp_distance_matrix: ") + cudaGetErrorString(e)};
    }
    ctx->release(ws);
    return st.ok() ? RPP_OK : report(st);
}

const char *rpp_status_string(rpp_status s) {
    switch (s) {
        case RPP_OK: return "ok";
        case RPP_E_INVALID: return "invalid argument";
        case RPP_E_NOMEM: return "out of memory";
        case RPP_E_OVERFLOW: return "index overflow";
        case RPP_E_CUDA: return "CUDA error";
        case RPP_E_TIMEOUT: return "timeout";
        case RPP_E_BUSY: return "busy";
    }
    return "unknown status";
}

const char *rpp_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
