// backward.cu -- gradients of the interval endpoints with respect to the point
// coordinates (a differentiation layer on top of the paper's method).
//
// Every endpoint of a finite interval is a distance-matrix entry: the length
// |x_u - x_v| of the youngest edge of the birth or death simplex. Its gradient
// with respect to x_u is (x_u - x_v) / |x_u - x_v|. The host groups the
// contributions by target point (a CSR list), so one thread per point sums
// its contributions in a fixed order: the result is deterministic, with no
// atomics.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "pipeline.h"

namespace rpp {

namespace {

// entry: other endpoint (global point index) and the gradient slot; slot bit
// 31 set selects grad_death, otherwise grad_birth.
struct Contribution {
    int32_t other;
    uint32_t slot;
};

__global__ void k_backward(const float *__restrict__ X, int dim, int64_t npoints,
                           const int64_t *__restrict__ offsets,
                           const Contribution *__restrict__ contrib,
                           const float *__restrict__ grad_birth,
                           const float *__restrict__ grad_death, float *__restrict__ grad) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= npoints) return;
    const int64_t b = offsets[u], e = offsets[u + 1];
    for (int k0 = 0; k0 < dim; k0 += 16) {
        float acc[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[k] = 0.0f;
        for (int64_t j = b; j < e; ++j) {
            const Contribution c = contrib[j];
            const float g = (c.slot & 0x80000000u) ? grad_death[c.slot & 0x7fffffffu]
                                                   : grad_birth[c.slot];
            // edge length with the library's distance formula
            float s = 0.0f;
            for (int k = 0; k < dim; ++k) {
                const float d = __fsub_rn(X[u * dim + k], X[(int64_t)c.other * dim + k]);
                s = __fadd_rn(s, __fmul_rn(d, d));
            }
            const float len = __fsqrt_rn(s);
            if (!(len > 0.0f)) continue;  // coincident points: no direction
            const float scale = g / len;
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (k0 + k < dim)
                    acc[k] += scale * (X[u * dim + k0 + k] - X[(int64_t)c.other * dim + k0 + k]);
        }
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (k0 + k < dim) grad[u * dim + k0 + k] = acc[k];
    }
}

}  // namespace

}  // namespace rpp

using namespace rpp;

extern "C" rpp_status rpp_barcodes_backward(rpp_context *ctx, int32_t batch, const float *points,
                                            const int64_t *n, int32_t dim,
                                            const rpp_result *const *results,
                                            const float *grad_birth, const float *grad_death,
                                            float *grad_points, void *stream) {
    if (!ctx || batch < 0 || (batch > 0 && (!points || !n || !results || !grad_points)) ||
        dim < 1) {
        set_last_error("rpp_barcodes_backward: invalid arguments");
        return RPP_E_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaSetDevice(ctx->device);
    int64_t npoints = 0, nint = 0;
    std::vector<int64_t> base(batch);
    for (int32_t i = 0; i < batch; ++i) {
        if (!results[i] || n[i] < 1) {
            set_last_error("rpp_barcodes_backward: missing result or bad n");
            return RPP_E_INVALID;
        }
        base[i] = npoints;
        npoints += n[i];
        nint += rpp_result_total(results[i]);
    }
    if (nint > 0 && (!grad_birth || !grad_death)) {
        set_last_error("rpp_barcodes_backward: gradient arrays are NULL");
        return RPP_E_INVALID;
    }
    if (nint >= (int64_t)0x7fffffff) {
        set_last_error("rpp_barcodes_backward: too many intervals");
        return RPP_E_INVALID;
    }
    // CSR of contributions by target point
    std::vector<int64_t> count(npoints + 1, 0);
    struct Raw {
        int32_t u, other;
        uint32_t slot;
    };
    std::vector<Raw> raw;
    raw.reserve((size_t)nint * 4);
    int64_t slot = 0;
    for (int32_t i = 0; i < batch; ++i) {
        const rpp_result *r = results[i];
        for (int q = 0; q <= r->max_dim; ++q) {
            for (size_t k = 0; k < r->iv[q].size(); ++k, ++slot) {
                const rpp_critical &c = r->cr[q][k];
                const rpp_interval &iv = r->iv[q][k];
                if (c.bu >= 0) {
                    const int32_t u = (int32_t)(base[i] + c.bu), v = (int32_t)(base[i] + c.bv);
                    raw.push_back({u, v, (uint32_t)slot});
                    raw.push_back({v, u, (uint32_t)slot});
                }
                if (c.du >= 0 && std::isfinite(iv.death)) {
                    const int32_t u = (int32_t)(base[i] + c.du), v = (int32_t)(base[i] + c.dv);
                    raw.push_back({u, v, (uint32_t)slot | 0x80000000u});
                    raw.push_back({v, u, (uint32_t)slot | 0x80000000u});
                }
            }
        }
    }
    for (const Raw &x : raw) ++count[x.u + 1];
    for (int64_t u = 0; u < npoints; ++u) count[u + 1] += count[u];
    std::vector<int64_t> fill(count.begin(), count.end() - 1);
    std::vector<Contribution> csr(raw.size() + 1);
    for (const Raw &x : raw) csr[fill[x.u]++] = {x.other, x.slot};

    Workspace *ws = ctx->acquire();
    struct Guard {
        rpp_context *c;
        Workspace *w;
        ~Guard() { c->release(w); }
    } guard{ctx, ws};
    void *d_off, *d_csr, *h_off, *h_csr;
    Status st;
    if (!(st = ws->dev(ws->up, (count.size()) * 8, &d_off)).ok()) return report(st);
    if (!(st = ws->dev(ws->mst, csr.size() * sizeof(Contribution), &d_csr)).ok()) return report(st);
    if (!(st = ws->host(ws->h_up, count.size() * 8, &h_off)).ok()) return report(st);
    if (!(st = ws->host(ws->h_mst, csr.size() * sizeof(Contribution), &h_csr)).ok())
        return report(st);
    std::memcpy(h_off, count.data(), count.size() * 8);
    std::memcpy(h_csr, csr.data(), csr.size() * sizeof(Contribution));
    cudaMemcpyAsync(d_off, h_off, count.size() * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_csr, h_csr, csr.size() * sizeof(Contribution), cudaMemcpyHostToDevice, s);
    if (npoints > 0) {
        ++g_launches;
        k_backward<<<(unsigned)((npoints + 127) / 128), 128, 0, s>>>(
            points, dim, npoints, (const int64_t *)d_off, (const Contribution *)d_csr, grad_birth,
            grad_death, grad_points);
    }
    cudaError_t e = cudaStreamSynchronize(s);  // the staging buffers are reused
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string("rpp_barcodes_backward: ") + cudaGetErrorString(e));
        return RPP_E_CUDA;
    }
    return RPP_OK;
}
