// batch.cpp -- many independent clouds per call, and the size-bucket tuning
// table used by the apparent-pair pass.
#include <cmath>

#include "pipeline.h"

using namespace rpp;

rpp::Tuning rpp_context::tuning_for(int64_t n, int p) {
    rpp::Tuning t;
    (void)p;
    t.group = n <= 256 ? 4 : 8;
    return t;
}

extern "C" rpp_status rpp_barcodes_batched(rpp_context *ctx, int32_t batch,
                                           const float *const *data, const int64_t *n,
                                           const int32_t *dim, int32_t max_dim,
                                           const float *thresholds, const float *quantiles,
                                           void *stream, rpp_result **out) {
    if (!ctx || batch < 0 || (batch > 0 && (!data || !n || !dim || !out))) {
        set_last_error("rpp_barcodes_batched: invalid arguments");
        return RPP_E_INVALID;
    }
    std::vector<Instance> ins(batch);
    for (int32_t i = 0; i < batch; ++i) {
        Instance &in = ins[i];
        in.data = data[i];
        in.kind = RPP_INPUT_POINTS;
        in.n = n[i];
        in.dim = dim[i];
        in.max_dim = max_dim;
        in.threshold = thresholds ? thresholds[i] : INFINITY;
        in.quantile = quantiles ? quantiles[i] : 0.0f;
        Status v = validate_instance(in);
        if (!v.ok()) {
            v.msg = "cloud " + std::to_string(i) + ": " + v.msg;
            return report(v);
        }
    }
    Workspace *ws = ctx->acquire();
    for (int32_t i = 0; i < batch; ++i) {
        rpp_result *res = new rpp_result();
        Status s = run_instance(ctx, *ws, ins[i], (cudaStream_t)stream, res);
        if (!s.ok()) {
            delete res;
            for (int32_t j = 0; j < i; ++j) {
                rpp_result_free(out[j]);
                out[j] = nullptr;
            }
            ctx->release(ws);
            s.msg = "cloud " + std::to_string(i) + ": " + s.msg;
            return report(s);
        }
        out[i] = res;
    }
    ctx->release(ws);
    return RPP_OK;
}
