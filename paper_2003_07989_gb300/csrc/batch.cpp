// batch.cpp -- many independent clouds per call.
//
// Clouds of up to BATCH_NMAX points asking for H0 and H1 go through the fused
// pass of batch.cu: they are grouped into size buckets (64, 128, 256, 512,
// 1024 points) and each bucket runs in launches of up to `cap` clouds, each
// launch a captured CUDA graph (control block upload, the fused kernel, and
// the download of the per-cloud outputs and H0 edges) that is re-instantiated
// only when a buffer moves. The launch shape of the fused kernel (threads per
// block, lanes per column of the apparent test) is chosen per bucket by the
// autotuner the first time the bucket runs in a context: every candidate runs
// on that launch's clouds and the fastest is kept. Clouds with leftover
// columns then get their distance rows and sorted neighbour lists (one more
// launch), and their submatrix reductions run on the host threads, one cloud
// per thread. Everything else (larger clouds, higher dimensions, recorded
// intermediate arrays) takes the per-instance pipeline.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

#include "pipeline.h"

using namespace rpp;

rpp::Tuning rpp_context::tuning_for(int64_t n, int p) {
    rpp::Tuning t;
    (void)p;
    t.group = n <= 256 ? 42 : 44;  // untuned default: 4 lanes, 2 or 4 candidate blocks a step
    return t;
}

namespace rpp {

namespace {

const int BUCKETS[] = {64, 128, 256, 512, BATCH_NMAX};
constexpr size_t D_SCRATCH_BYTES = 256ull << 20;  // distance matrices of one launch
constexpr uint64_t LEFT_CAP = 1ull << 20;         // leftover columns of one launch

int bucket_nmax(int64_t n) {
    for (int b : BUCKETS)
        if (n <= b) return b;
    return -1;
}

int ld_of(int n) { return (n + 3) & ~3; }

// Clouds per launch for a bucket: the distance scratch stays near 256 MB.
int bucket_cap(int nmax) {
    const size_t per = (size_t)nmax * ld_of(nmax) * 4;
    return (int)std::max<size_t>(1, std::min<size_t>(4096, D_SCRATCH_BYTES / per));
}

int dimcap_of(int dim) {
    int c = 2;
    while (c < dim) c <<= 1;
    return c;
}

// The device and host buffers of one fused launch of a bucket, sized for its
// capacity so that the captured graph stays valid from launch to launch.
struct Bufs {
    float *pts;
    BatchCloud *clouds;
    int32_t *order;
    BatchCtl *ctl;
    float *D;
    uint64_t *mst;
    BatchOut *outs;
    Leftover *left;
    int32_t *lcloud;
    uint16_t *app_w;  // per cloud and edge: the vertex of its apparent pair, or 0xFFFF
    float *h_pts;
    BatchCloud *h_clouds;
    int32_t *h_order;
    BatchCtl *h_ctl;  // [0] uploaded, [1] downloaded
    BatchOut *h_outs;
    uint64_t *h_mst;
    Leftover *h_left;
    int32_t *h_lcloud;
};

uint64_t pow2_ge(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Capacities of one fused launch, rounded up to powers of two so that launches
// of similar batches reuse the same buffers and captured graphs.
struct Caps {
    uint64_t clouds = 0, pts = 0, D = 0, mst = 0, left = 0, aw = 0;
};

Caps caps_of(const std::vector<Instance> &ins, const std::vector<int> &idx) {
    Caps c;
    uint64_t pts = 0, D = 0, mst = 0, cols = 0;
    for (int i : idx) {
        const uint64_t n = (uint64_t)ins[i].n;
        pts += n * (uint64_t)ins[i].dim;
        D += n * (uint64_t)ld_of((int)n);
        mst += n;
        cols += n * (n - 1) / 2;
    }
    c.clouds = pow2_ge(std::max<size_t>(idx.size(), 16));
    c.pts = pow2_ge(std::max<uint64_t>(pts, 1024));
    c.D = pow2_ge(std::max<uint64_t>(D, 1024));
    c.mst = pow2_ge(std::max<uint64_t>(mst, 1024));
    c.aw = pow2_ge(std::max<uint64_t>(cols, 1024));
    // leftover columns are a small share of the columns (the apparent-pair
    // rate); a launch that finds more runs the overflowing clouds alone
    c.left = std::min<uint64_t>(LEFT_CAP, pow2_ge(std::max<uint64_t>(cols / 16, 4096)));
    return c;
}

// Device bytes a fused launch over these clouds holds (buffers of caps_of,
// the growth slack of Workspace::dev, the rows of clouds with leftovers, and
// the device reduction's pool, outputs and sorted edges).
size_t launch_device_bytes(const Caps &c, uint64_t rows) {
    auto slack = [](size_t b) { return ((b + b / 4) + 255) & ~(size_t)255; };
    const uint64_t lcap = std::min(c.left, c.aw);  // leftovers are edges
    const size_t reduce = slack(reduce_small_vpool_words(lcap, 0) * 4 + rows / 2) +
                          slack(lcap * (sizeof(Leftover) + 20)) + slack(rows * 9) +
                          slack(radix_scratch_bound(rows / 2) + 64);
    return slack(c.pts * 4) + slack(c.clouds * (sizeof(BatchCloud) + 4 + sizeof(BatchOut) + 8)) +
           slack(c.D * 4) + slack(c.mst * 8) + slack(c.left * (sizeof(Leftover) + 4)) +
           slack(c.aw * 2) + slack(rows * 12) + slack(rows) + reduce + 8 * 256;
}

Status get_bufs(Workspace &ws, const Caps &c, Bufs &b) {
    void *p;
    RPP_TRY(ws.dev(ws.b_pts, c.pts * 4, &p));
    b.pts = (float *)p;
    RPP_TRY(ws.dev(ws.b_clouds, c.clouds * sizeof(BatchCloud), &p));
    b.clouds = (BatchCloud *)p;
    RPP_TRY(ws.dev(ws.b_order, c.clouds * 4, &p));
    b.order = (int32_t *)p;
    RPP_TRY(ws.dev(ws.b_ctl, sizeof(BatchCtl), &p));
    b.ctl = (BatchCtl *)p;
    RPP_TRY(ws.dev(ws.b_D, c.D * 4, &p));
    b.D = (float *)p;
    RPP_TRY(ws.dev(ws.b_mst, c.mst * 8, &p));
    b.mst = (uint64_t *)p;
    RPP_TRY(ws.dev(ws.b_outs, c.clouds * sizeof(BatchOut), &p));
    b.outs = (BatchOut *)p;
    RPP_TRY(ws.dev(ws.b_left, c.left * sizeof(Leftover), &p));
    b.left = (Leftover *)p;
    RPP_TRY(ws.dev(ws.b_lcloud, c.left * 4, &p));
    b.lcloud = (int32_t *)p;
    RPP_TRY(ws.dev(ws.b_aw, c.aw * 2, &p));
    b.app_w = (uint16_t *)p;
    RPP_TRY(ws.host(ws.hb_pts, c.pts * 4, &p));
    b.h_pts = (float *)p;
    RPP_TRY(ws.host(ws.hb_clouds, c.clouds * sizeof(BatchCloud), &p));
    b.h_clouds = (BatchCloud *)p;
    RPP_TRY(ws.host(ws.hb_order, c.clouds * 4, &p));
    b.h_order = (int32_t *)p;
    RPP_TRY(ws.host(ws.hb_ctl, 2 * sizeof(BatchCtl), &p));
    b.h_ctl = (BatchCtl *)p;
    RPP_TRY(ws.host(ws.hb_outs, c.clouds * sizeof(BatchOut), &p));
    b.h_outs = (BatchOut *)p;
    RPP_TRY(ws.host(ws.hb_mst, c.mst * 8, &p));
    b.h_mst = (uint64_t *)p;
    RPP_TRY(ws.host(ws.hb_left, c.left * sizeof(Leftover), &p));
    b.h_left = (Leftover *)p;
    RPP_TRY(ws.host(ws.hb_lcloud, c.left * 4, &p));
    b.h_lcloud = (int32_t *)p;
    return Status();
}

// The fused launch as a CUDA graph: upload the control block, run the fused
// kernel, download the per-cloud outputs, the control block and the H0 edges.
Status fused_graph(Workspace &ws, const BatchPlan &plan, const Caps &c, const Bufs &b,
                   cudaGraphExec_t *out) {
    const std::vector<uintptr_t> key = {
        (uintptr_t)plan.nmax,   (uintptr_t)plan.dimcap,  (uintptr_t)plan.cfg.threads,
        (uintptr_t)plan.cfg.group, (uintptr_t)plan.blocks, (uintptr_t)c.clouds,
        (uintptr_t)c.mst,       (uintptr_t)c.left,
        (uintptr_t)b.pts,       (uintptr_t)b.clouds,     (uintptr_t)b.order,
        (uintptr_t)b.ctl,       (uintptr_t)b.D,          (uintptr_t)b.mst,
        (uintptr_t)b.outs,      (uintptr_t)b.left,       (uintptr_t)b.lcloud,
        (uintptr_t)b.app_w,     (uintptr_t)c.aw,
        (uintptr_t)b.h_ctl,     (uintptr_t)b.h_outs,     (uintptr_t)b.h_mst};
    for (auto &g : ws.graphs)
        if (g.first == key) {
            *out = g.second;
            return Status();
        }
    if (ws.graphs.size() >= 16) {  // keep the most recent ones
        cudaGraphExecDestroy(ws.graphs.front().second);
        ws.graphs.erase(ws.graphs.begin());
    }
    if (!ws.capture_stream) RPP_CK(cudaStreamCreateWithFlags(&ws.capture_stream, cudaStreamNonBlocking));
    cudaStream_t cs = ws.capture_stream;
    RPP_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const long long l0 = g_launches;
    cudaMemcpyAsync(b.ctl, &b.h_ctl[0], sizeof(BatchCtl), cudaMemcpyHostToDevice, cs);
    launch_batch_h1(plan, b.pts, b.clouds, b.order, b.ctl, b.D, b.mst, b.outs, b.left, b.lcloud,
                    c.left, b.app_w, cs);
    cudaMemcpyAsync(b.h_outs, b.outs, c.clouds * sizeof(BatchOut), cudaMemcpyDeviceToHost, cs);
    cudaMemcpyAsync(&b.h_ctl[1], b.ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, cs);
    cudaMemcpyAsync(b.h_mst, b.mst, c.mst * 8, cudaMemcpyDeviceToHost, cs);
    g_launches = l0;  // nothing ran yet
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess || !g) {
        cudaGetLastError();
        return fail(RPP_E_CUDA, std::string("graph capture of the fused pass failed: ") +
                                    cudaGetErrorString(e));
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(RPP_E_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    ws.graphs.emplace_back(key, exec);
    *out = exec;
    return Status();
}

// Autotuner: time every candidate launch shape on this launch's clouds (the
// inputs are already on the device) and keep the fastest for the bucket.
Status autotune(rpp_context *ctx, const Bufs &b, const Caps &caps, int nmax, int dimcap,
                int nclouds, cudaStream_t s, BatchConfig *best) {
    // (threads, group, blocks per SM): group = lanes per column G, or 10 G + U
    // for U candidate blocks a step; a cap on the blocks per SM bounds the
    // distance matrices in flight (their sum should stay in L2)
    static const BatchConfig cands[] = {{128, 4, 0},   {128, 8, 0},  {256, 4, 0},  {256, 8, 0},
                                        {256, 16, 0},  {512, 8, 0},  {512, 16, 0}, {256, 42, 0},
                                        {256, 44, 0},  {512, 42, 0}, {512, 42, 1}, {512, 44, 1},
                                        {256, 42, 2},  {256, 44, 2}, {512, 8, 1},
                                        {1024, 42, 1}, {1024, 44, 1}, {1024, 8, 1}};
    cudaEvent_t e0, e1;
    RPP_CK(cudaEventCreate(&e0));
    RPP_CK(cudaEventCreate(&e1));
    float best_ms = INFINITY;
    for (const BatchConfig &c : cands) {
        const BatchPlan plan = plan_batch_h1(nmax, dimcap, c, ctx->sms);
        b.h_ctl[0].queue = 0;
        b.h_ctl[0].nclouds = nclouds;
        b.h_ctl[0].left_count = 0;
        float ms = 0.0f;
        for (int rep = 0; rep < 2; ++rep) {  // the first run warms the caches
            cudaMemcpyAsync(b.ctl, &b.h_ctl[0], sizeof(BatchCtl), cudaMemcpyHostToDevice, s);
            cudaEventRecord(e0, s);
            launch_batch_h1(plan, b.pts, b.clouds, b.order, b.ctl, b.D, b.mst, b.outs, b.left,
                            b.lcloud, caps.left, b.app_w, s);
            cudaEventRecord(e1, s);
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return fail(RPP_E_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
            }
            cudaEventElapsedTime(&ms, e0, e1);
        }
        if (ms < best_ms) {
            best_ms = ms;
            *best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return Status();
}

// Results of one cloud of a fused launch.
struct CloudWork {
    int slot = 0;                  // position in the launch
    std::vector<Leftover> left;    // its leftover columns
    int64_t job = -1;              // row job (distance rows and neighbour lists), -1: none
    bool fallback = false;         // leftover pool overflowed: run it alone
};

// One fused launch over clouds ins[idx[k]]: what its host half needs.
struct Launch {
    std::vector<int> idx;
    double t0 = 0.0;
    long long launches = 0;
    double dev_ms = 0.0;
    Bufs b{};
    std::vector<CloudWork> W;
    std::vector<int64_t> off, aoff;  // per row job: rows (n^2) and edges (C(n,2)) before it
    float *hD = nullptr;             // per job: distance rows, neighbour lists, apparent vertices
    uint64_t *hN = nullptr;
    uint16_t *hA = nullptr;
    // the device reduction: per row job its reduce job (-1: none); per reduce
    // job its leftovers' first position, status and additions; per leftover
    // (sorted by index within its cloud) the death index and diameter
    std::vector<int> rjob;
    std::vector<int64_t> rleft;
    // [0]: the first phase's (cursors), [1]: the second phase's (sweeps)
    const int32_t *rstat[2] = {nullptr, nullptr}, *radds[2] = {nullptr, nullptr};
    const uint64_t *rdeath[2] = {nullptr, nullptr};
    const float *rddiam[2] = {nullptr, nullptr};
    // recorded on the reduction's stream once a phase's results are in the
    // host buffers above (nullptr: that phase did not run in this launch)
    cudaEvent_t red[2] = {nullptr, nullptr};
    unsigned *cancel = nullptr;  // host side of the first phase's cancel flag
    bool *pending = nullptr;     // the workspace's reduce_pending
    int red_mode = 0;  // the context's device_reduce when launched
    int device = 0;
};

// Device half of a fused launch: the pass itself, then the distance rows,
// neighbour lists and apparent vertices of every cloud with leftovers, copied
// into ws's host buffers (which stay in use until the host half is done).
Status launch_device(rpp_context *ctx, Workspace &ws, const std::vector<Instance> &ins,
                     const std::vector<int> &idx, int nmax, int dimcap, cudaStream_t s,
                     Launch &L) {
    if (ws.reduce_pending) {  // a cancelled device reduction may still read these buffers
        RPP_CK(cudaEventSynchronize(ws.ev_reduce));
        ws.reduce_pending = false;
    }
    L.idx = idx;
    L.t0 = now_ms();
    const long long launches0 = g_launches;
    const int k = (int)idx.size();
    const Caps caps = caps_of(ins, idx);
    Bufs &b = L.b;
    RPP_TRY(get_bufs(ws, caps, b));

    // layout and inputs
    int64_t pt = 0, dd = 0, aw = 0;
    int32_t ms = 0;
    std::vector<const float *> dev_src(k, nullptr);
    bool any_dev = false, any_host = false;
    for (int j = 0; j < k; ++j) {
        const Instance &in = ins[idx[j]];
        BatchCloud &c = b.h_clouds[j];
        c.n = (int32_t)in.n;
        c.dim = in.dim;
        c.ld = ld_of(c.n);
        c.pt_off = pt;
        c.d_off = dd;
        c.mst_off = ms;
        c.t_user = in.quantile > 0.0 ? INFINITY : in.threshold;
        c.qrank = in.quantile > 0.0 ? quantile_rank(in.quantile, (uint64_t)in.n) : 0;
        c.max_dim = in.max_dim;
        c.aw_off = aw;
        const size_t cnt = (size_t)c.n * c.dim;
        if (is_device_pointer(in.data)) {
            dev_src[j] = in.data;
            any_dev = true;
        } else {
            std::memcpy(b.h_pts + pt, in.data, cnt * 4);
            any_host = true;
        }
        pt += (int64_t)cnt;
        dd += (int64_t)c.n * c.ld;
        aw += (int64_t)c.n * (c.n - 1) / 2;
        ms += std::max(0, c.n - 1);
        b.h_order[j] = j;
    }
    std::stable_sort(b.h_order, b.h_order + k,
                     [&](int32_t x, int32_t y) { return b.h_clouds[x].n > b.h_clouds[y].n; });
    RPP_CK(cudaMemcpyAsync(b.clouds, b.h_clouds, (size_t)k * sizeof(BatchCloud),
                           cudaMemcpyHostToDevice, s));
    RPP_CK(cudaMemcpyAsync(b.order, b.h_order, (size_t)k * 4, cudaMemcpyHostToDevice, s));
    if (any_host) RPP_CK(cudaMemcpyAsync(b.pts, b.h_pts, (size_t)pt * 4, cudaMemcpyHostToDevice, s));
    if (any_dev) {
        void *p, *hp;
        RPP_TRY(ws.dev(ws.b_src, (size_t)k * sizeof(void *), &p));
        RPP_TRY(ws.host(ws.hb_src, (size_t)k * sizeof(void *), &hp));
        std::memcpy(hp, dev_src.data(), (size_t)k * sizeof(void *));
        RPP_CK(cudaMemcpyAsync(p, hp, (size_t)k * sizeof(void *), cudaMemcpyHostToDevice, s));
        launch_gather_points((const float *const *)p, b.clouds, k, b.pts, s);
    }

    // launch shape: the bucket's tuned one (tuned now if this is its first run)
    BatchConfig cfg;
    bool have = false;
    {
        std::lock_guard<std::mutex> g(ctx->tune_mu);
        auto it = ctx->batch_tuning.find(nmax);
        if (it != ctx->batch_tuning.end()) {
            cfg = it->second;
            have = true;
        }
    }
    if (!have && ctx->autotune) {
        RPP_TRY(autotune(ctx, b, caps, nmax, dimcap, k, s, &cfg));
        std::lock_guard<std::mutex> g(ctx->tune_mu);
        ctx->batch_tuning.emplace(nmax, cfg);
    }
    const BatchPlan plan = plan_batch_h1(nmax, dimcap, cfg, ctx->sms);
    cudaGraphExec_t exec;
    RPP_TRY(fused_graph(ws, plan, caps, b, &exec));
    b.h_ctl[0].queue = 0;
    b.h_ctl[0].nclouds = k;
    b.h_ctl[0].left_count = 0;
    RPP_CK(cudaGraphLaunch(exec, s));
    ++g_launches;  // the fused kernel
    const double a = now_ms();
    RPP_CK(cudaStreamSynchronize(s));
    double dev_ms = now_ms() - a;

    // per-cloud outputs, leftovers grouped by cloud
    for (int j = 0; j < k; ++j) {
        const unsigned err = b.h_outs[j].err;
        if (err & ERR_INTERNAL)
            return fail(RPP_E_CUDA, "cloud " + std::to_string(idx[j]) +
                                        ": fused pass: spanning-forest root search exceeded its bound");
        if (err)
            return fail(RPP_E_INVALID, "cloud " + std::to_string(idx[j]) +
                                           ": invalid input: non-finite distance");
    }
    const uint64_t found = b.h_ctl[1].left_count, got = std::min(found, caps.left);
    if (got) {
        RPP_CK(cudaMemcpyAsync(b.h_left, b.left, got * sizeof(Leftover), cudaMemcpyDeviceToHost, s));
        RPP_CK(cudaMemcpyAsync(b.h_lcloud, b.lcloud, got * 4, cudaMemcpyDeviceToHost, s));
        RPP_CK(cudaStreamSynchronize(s));
    }
    std::vector<CloudWork> &W = L.W;
    W.assign(k, CloudWork());
    for (int j = 0; j < k; ++j) W[j].slot = j;
    for (uint64_t i = 0; i < got; ++i) W[b.h_lcloud[i]].left.push_back(b.h_left[i]);
    std::vector<int32_t> jobs;
    std::vector<int64_t> &off = L.off, &aoff = L.aoff;
    off.clear();
    aoff.clear();
    int64_t rows = 0, edges = 0;
    for (int j = 0; j < k; ++j) {
        if (W[j].left.size() < b.h_outs[j].nleft) {
            W[j].fallback = true;
            continue;
        }
        if (W[j].left.empty()) continue;
        W[j].job = (int64_t)jobs.size();
        jobs.push_back(j);
        off.push_back(rows);
        aoff.push_back(edges);
        rows += (int64_t)b.h_clouds[j].n * b.h_clouds[j].n;
        edges += (int64_t)b.h_clouds[j].n * (b.h_clouds[j].n - 1) / 2;
    }
    float *&hD = L.hD;
    uint64_t *&hN = L.hN;
    uint16_t *&hA = L.hA;
    hD = nullptr;
    hN = nullptr;
    hA = nullptr;
    if (!jobs.empty()) {  // distance rows and neighbour lists of the clouds with leftovers
        void *p, *hp;
        const size_t nj = jobs.size();
        RPP_TRY(ws.dev(ws.b_jobs, nj * 4, &p));
        int32_t *djobs = (int32_t *)p;
        RPP_TRY(ws.dev(ws.b_off, 2 * nj * 8, &p));
        int64_t *doff = (int64_t *)p;
        RPP_TRY(ws.dev(ws.b_Dout, (size_t)rows * 4, &p));
        float *dD = (float *)p;
        RPP_TRY(ws.dev(ws.b_nbr, (size_t)rows * 8, &p));
        uint64_t *dN = (uint64_t *)p;
        RPP_TRY(ws.dev(ws.b_awout, (size_t)std::max<int64_t>(edges, 1) * 2, &p));
        uint16_t *dA = (uint16_t *)p;
        RPP_TRY(ws.host(ws.hb_jobs, nj * 4 + 2 * nj * 8, &hp));
        std::memcpy(hp, jobs.data(), nj * 4);
        std::memcpy((char *)hp + nj * 4, off.data(), nj * 8);
        std::memcpy((char *)hp + nj * 4 + nj * 8, aoff.data(), nj * 8);
        RPP_CK(cudaMemcpyAsync(djobs, hp, nj * 4, cudaMemcpyHostToDevice, s));
        RPP_CK(cudaMemcpyAsync(doff, (char *)hp + nj * 4, 2 * nj * 8, cudaMemcpyHostToDevice, s));
        launch_batch_rows(b.D, b.clouds, djobs, (int)nj, doff, nmax, dD, dN, b.app_w, dA, s);
        RPP_CK(cudaGetLastError());
        // clouds of up to REDUCE_SMALL_NMAX points reduce their leftover
        // columns on the device, on a stream of their own: the rows' copies to
        // the host, the host half and the next launch's pass run meanwhile (a
        // cloud whose walks outgrow the device's budget is reduced by the host)
        L.rjob.assign(nj, -1);
        L.rleft.clear();
        for (int ph = 0; ph < 2; ++ph) {
            L.rstat[ph] = L.radds[ph] = nullptr;
            L.rdeath[ph] = nullptr;
            L.rddiam[ph] = nullptr;
            L.red[ph] = nullptr;
        }
        L.red_mode = ctx->device_reduce;
        L.cancel = nullptr;
        L.pending = &ws.reduce_pending;
        L.device = ws.device;
        if (ctx->device_reduce) {
            std::vector<ReduceJob> rj;
            int64_t lpos = 0;
            int rnmax = 0;
            uint64_t ecap = 0;  // edges inside the threshold of the reduced clouds
            int64_t vpos = 0;   // pool words of the reduced clouds
            for (size_t q = 0; q < nj; ++q) {
                const int j = jobs[q];
                const BatchCloud &c = b.h_clouds[j];
                if (c.n > REDUCE_SMALL_NMAX) continue;
                std::vector<Leftover> &Lv = W[j].left;
                std::sort(Lv.begin(), Lv.end(),
                          [](const Leftover &x, const Leftover &y) { return x.index < y.index; });
                ReduceJob R;
                R.d_off = off[q];
                R.aw_off = aoff[q];
                R.left_off = lpos;
                R.nleft = (int64_t)Lv.size();
                R.n = c.n;
                R.t = b.h_outs[j].t;
                R.v_off = vpos;
                R.v_cap = (int64_t)reduce_small_vpool_words(R.nleft, (uint64_t)c.n);
                vpos += R.v_cap;
                L.rjob[q] = (int)rj.size();
                L.rleft.push_back(lpos);
                rj.push_back(R);
                lpos += (int64_t)Lv.size();
                rnmax = std::max(rnmax, c.n);
                ecap += b.h_outs[j].ncols;
            }
            if (!rj.empty()) {
                const size_t nr = rj.size(), nl = (size_t)lpos;
                const size_t in_bytes = nr * sizeof(ReduceJob) + nl * sizeof(Leftover) + nr * 4;
                RPP_TRY(ws.host(ws.hr_in, in_bytes, &hp));
                std::memcpy(hp, rj.data(), nr * sizeof(ReduceJob));
                Leftover *hl = (Leftover *)((char *)hp + nr * sizeof(ReduceJob));
                // the second phase's blocks take the heaviest clouds first
                // (most leftover columns times points), so that no block
                // starts a long cloud at the end
                int32_t *hord = (int32_t *)(hl + nl);
                for (size_t q = 0; q < nr; ++q) hord[q] = (int32_t)q;
                std::stable_sort(hord, hord + nr, [&](int32_t x, int32_t y) {
                    return rj[x].nleft * rj[x].n > rj[y].nleft * rj[y].n;
                });
                for (size_t q = 0; q < nj; ++q)
                    if (L.rjob[q] >= 0) {
                        const std::vector<Leftover> &Lv = W[jobs[q]].left;
                        std::memcpy(hl + L.rleft[L.rjob[q]], Lv.data(), Lv.size() * sizeof(Leftover));
                    }
                if (!ws.reduce_stream)
                    RPP_CK(cudaStreamCreateWithFlags(&ws.reduce_stream, cudaStreamNonBlocking));
                if (!ws.ev_rows) RPP_CK(cudaEventCreateWithFlags(&ws.ev_rows, cudaEventDisableTiming));
                if (!ws.ev_reduce)
                    RPP_CK(cudaEventCreateWithFlags(&ws.ev_reduce, cudaEventDisableTiming));
                if (!ws.ev_reduce_b)
                    RPP_CK(cudaEventCreateWithFlags(&ws.ev_reduce_b, cudaEventDisableTiming));
                cudaStream_t rs = ws.reduce_stream;
                RPP_CK(cudaEventRecord(ws.ev_rows, s));
                RPP_CK(cudaStreamWaitEvent(rs, ws.ev_rows, 0));
                void *dj, *dl, *dvp, *dvs, *dvc, *dde, *ddd, *dst;
                void *dek = nullptr, *det = nullptr, *des = nullptr, *dea = nullptr;
                RPP_TRY(ws.dev(ws.r_jobs, nr * sizeof(ReduceJob) + nr * 4 + 16, &dj));
                int32_t *dord = (int32_t *)((char *)dj + nr * sizeof(ReduceJob));
                unsigned *dnext = (unsigned *)(dord + nr);
                RPP_TRY(ws.dev(ws.r_left, std::max<size_t>(nl, 1) * sizeof(Leftover), &dl));
                RPP_TRY(ws.dev(ws.r_vpool, std::max<size_t>((size_t)vpos, 1) * 4, &dvp));
                RPP_TRY(ws.dev(ws.r_vstart, std::max<size_t>(nl, 1) * 4, &dvs));
                RPP_TRY(ws.dev(ws.r_vcnt, std::max<size_t>(nl, 1) * 4, &dvc));
                ecap = std::max<uint64_t>(ecap, 2);
                const bool sweeps = ctx->device_reduce == 2;
                if (sweeps) {  // the sweeps' sorted edges
                    RPP_TRY(ws.dev(ws.r_ekeys, ecap * 8, &dek));
                    RPP_TRY(ws.dev(ws.r_etmp, ecap * 8, &det));
                    RPP_TRY(ws.dev(ws.r_ekaw, ecap * 2, &dea));
                    RPP_TRY(ws.dev(ws.r_esort, radix_scratch_bytes(ecap) + 64, &des));
                }
                RPP_TRY(ws.dev(ws.r_death, std::max<size_t>(nl, 1) * 8, &dde));
                RPP_TRY(ws.dev(ws.r_ddiam, std::max<size_t>(nl, 1) * 4, &ddd));
                RPP_TRY(ws.dev(ws.r_stat, nr * 16, &dst));
                RPP_CK(cudaMemcpyAsync(dj, hp, nr * sizeof(ReduceJob), cudaMemcpyHostToDevice, rs));
                RPP_CK(cudaMemcpyAsync(dord, hord, nr * 4, cudaMemcpyHostToDevice, rs));
                if (nl)
                    RPP_CK(cudaMemcpyAsync(dl, hl, nl * sizeof(Leftover), cudaMemcpyHostToDevice, rs));
                ReduceSmallArgs ra;
                ra.D = dD;
                ra.aw = dA;
                ra.jobs = (const ReduceJob *)dj;
                ra.njobs = (int)nr;
                ra.nmax = rnmax;
                ra.left = (const Leftover *)dl;
                ra.vpool = (uint32_t *)dvp;
                ra.vstart = (uint32_t *)dvs;
                ra.vcnt = (uint32_t *)dvc;
                ra.death = (uint64_t *)dde;
                ra.ddiam = (float *)ddd;
                ra.status = (int32_t *)dst;
                ra.adds = (int32_t *)dst + nr;
                ra.status_b = (int32_t *)dst + 2 * nr;
                ra.adds_b = (int32_t *)dst + 3 * nr;
                ra.ekeys = (uint64_t *)dek;
                ra.etmp = (uint64_t *)det;
                ra.ekaw = (uint16_t *)dea;
                ra.ecount = des ? (unsigned long long *)((char *)des + radix_scratch_bytes(ecap))
                                : nullptr;
                ra.eerr = des ? (unsigned *)((char *)des + radix_scratch_bytes(ecap) + 8) : nullptr;
                ra.escratch = des;
                ra.ecap = ecap;
                ra.order_b = dord;
                ra.next_b = dnext;
                if (!sweeps) {  // the host may finish every cloud first: let it stop the device
                    void *hc, *dc = nullptr;
                    RPP_TRY(ws.host(ws.hr_cancel, 64, &hc));
                    RPP_CK(cudaHostGetDevicePointer(&dc, hc, 0));
                    __atomic_store_n((unsigned *)hc, 0u, __ATOMIC_RELEASE);
                    L.cancel = (unsigned *)hc;
                    ra.cancel = (const unsigned *)dc;
                }
                // each phase's results (per leftover: death, diameter; per
                // job: status, additions) are copied out behind its own event
                const size_t out_bytes = nl * 8 + nl * 4 + nr * 8;
                for (int ph = 0; ph < (sweeps ? 2 : 1); ++ph) {
                    if (ph == 0) launch_reduce_small(ra, rs);
                    else launch_reduce_small_sweep(ra, rs);
                    RPP_CK(cudaGetLastError());
                    RPP_TRY(ws.host(ph == 0 ? ws.hr_out : ws.hr_out_b, std::max<size_t>(out_bytes, 8),
                                    &hp));
                    uint64_t *hde = (uint64_t *)hp;
                    float *hdd = (float *)(hde + nl);
                    int32_t *hst = (int32_t *)(hdd + nl);
                    if (nl) {
                        RPP_CK(cudaMemcpyAsync(hde, dde, nl * 8, cudaMemcpyDeviceToHost, rs));
                        RPP_CK(cudaMemcpyAsync(hdd, ddd, nl * 4, cudaMemcpyDeviceToHost, rs));
                    }
                    RPP_CK(cudaMemcpyAsync(hst, (int32_t *)dst + 2 * ph * nr, nr * 8,
                                           cudaMemcpyDeviceToHost, rs));
                    cudaEvent_t ev = ph == 0 ? ws.ev_reduce : ws.ev_reduce_b;
                    RPP_CK(cudaEventRecord(ev, rs));
                    L.red[ph] = ev;
                    L.rdeath[ph] = hde;
                    L.rddiam[ph] = hdd;
                    L.rstat[ph] = hst;
                    L.radds[ph] = hst + nr;
                }
            }
        }
        RPP_TRY(ws.host(ws.hb_Dout, (size_t)rows * 4, &hp));
        hD = (float *)hp;
        RPP_TRY(ws.host(ws.hb_nbr, (size_t)rows * 8, &hp));
        hN = (uint64_t *)hp;
        RPP_CK(cudaMemcpyAsync(hD, dD, (size_t)rows * 4, cudaMemcpyDeviceToHost, s));
        RPP_CK(cudaMemcpyAsync(hN, dN, (size_t)rows * 8, cudaMemcpyDeviceToHost, s));
        RPP_TRY(ws.host(ws.hb_awout, (size_t)std::max<int64_t>(edges, 1) * 2, &hp));
        hA = (uint16_t *)hp;
        RPP_CK(cudaMemcpyAsync(hA, dA, (size_t)edges * 2, cudaMemcpyDeviceToHost, s));
        const double a2 = now_ms();
        RPP_CK(cudaStreamSynchronize(s));
        dev_ms += now_ms() - a2;
    }
    L.launches = g_launches - launches0;
    L.dev_ms = dev_ms;
    return Status();
}

// Host half of a fused launch: H0 from the forest, the submatrix reductions
// and the barcodes; results into out[idx[k]]. Clouds whose leftover columns
// overflowed the pool are appended to `alone` (run by themselves later).
Status launch_host(rpp_context *ctx, Launch &L,
                   rpp_result **out, std::vector<int> &alone) {
    const std::vector<int> &idx = L.idx;
    const int k = (int)idx.size();
    const Bufs &b = L.b;
    std::vector<CloudWork> &W = L.W;
    const std::vector<int64_t> &off = L.off, &aoff = L.aoff;
    const float *hD = L.hD;
    const uint64_t *hN = L.hN;
    const uint16_t *hA = L.hA;
    const double t0 = L.t0, dev_ms = L.dev_ms;
    const long long launches = L.launches;
    const int inner = (int)off.size() >= ctx->host_threads ? 1 : ctx->host_threads;
    std::vector<rpp_result *> res(k, nullptr);
    // whether cloud j went to the device reduction
    auto sent = [&](int j) {
        return W[j].job >= 0 && !L.rjob.empty() && L.rjob[W[j].job] >= 0;
    };
    // Whether phase ph of the device reduction has its results on the host.
    // With red_mode 1 a thread that finds them missing reduces the cloud
    // itself (both give the same pairs); with red_mode 2 it waits for them.
    std::atomic<bool> red_done[2];
    for (int ph = 0; ph < 2; ++ph) red_done[ph].store(false);
    auto device_done = [&](int ph) {
        if (!L.red[ph]) return false;
        if (red_done[ph].load(std::memory_order_acquire)) return true;
        cudaSetDevice(L.device);
        const cudaError_t e =
            L.red_mode == 2 ? cudaEventSynchronize(L.red[ph]) : cudaEventQuery(L.red[ph]);
        if (e == cudaSuccess) {
            red_done[ph].store(true, std::memory_order_release);
            return true;
        }
        cudaGetLastError();  // not ready (or failed: reported by the final synchronize)
        return false;
    };
    // The phase whose result job rj takes (-1: the host reduces it).
    auto device_phase = [&](int rj) {
        if (rj < 0) return -1;
        if (device_done(0) && L.rstat[0][rj] == 0) return 0;
        if (device_done(1) && L.rstat[1][rj] == 0) return 1;
        return -1;
    };
    // clouds the device does not reduce first, then the heaviest reductions
    // first (most leftover columns, then most points), so that the threads do
    // not wait on one long cloud at the end and reach the lightest clouds,
    // which the device reduces, last
    std::vector<int> sched(k);
    for (int j = 0; j < k; ++j) sched[j] = j;
    std::stable_sort(sched.begin(), sched.end(), [&](int x, int y) {
        if (sent(x) != sent(y)) return !sent(x);
        if (W[x].left.size() != W[y].left.size()) return W[x].left.size() > W[y].left.size();
        return b.h_clouds[x].n > b.h_clouds[y].n;
    });
    parallel_for(ctx->host_threads, k, [&](int64_t jj) {
        const int j = sched[jj];
        if (W[j].fallback) return;
        const BatchCloud &c = b.h_clouds[j];
        const BatchOut &o = b.h_outs[j];
        const int n = c.n;
        rpp_result *r = new rpp_result();
        r->max_dim = c.max_dim;
        rpp_stats &S = r->stats;
        std::memset(&S, 0, sizeof S);
        S.n = n;
        S.max_dim = c.max_dim;
        S.threshold = o.t;
        S.enclosing_radius = o.R;
        S.kernel_launches = launches;
        S.ms_device = dev_ms;
        std::vector<uint64_t> store;
        Binomial B;
        fill_binomial(n, 3, store, B);
        for (uint32_t q = 0; q < o.nmst; ++q) {  // H0 deaths
            const uint64_t key = b.h_mst[c.mst_off + q];
            const float d = bits_to_float((uint32_t)(key >> 32));
            if (!(d > 0.0f)) continue;  // zero length (duplicate points)
            int v[2];
            decode_host(B, key & 0xffffffffull, 1, n, v);
            rpp_critical cr = {-1, -1, v[0], v[1]};
            add_interval(r, 0, 0.0f, d, cr);
        }
        for (int64_t q = 0; q < (int64_t)n - (int64_t)o.nmst; ++q) {
            rpp_critical cr = {-1, -1, -1, -1};
            add_interval(r, 0, 0.0f, INFINITY, cr);
        }
        if (n >= 2) {
            S.candidates[1] = (int64_t)n * (n - 1) / 2;
            S.cleared[1] = o.nmst;
            S.columns[1] = (int64_t)o.ncols - o.nmst;
        }
        if (c.max_dim >= 1) {
            S.apparent[1] = (int64_t)o.napp;
            S.leftover[1] = (int64_t)o.nleft;
            S.scanned[1] = (int64_t)o.scanned;
            if (W[j].job >= 0) {
                const double a3 = now_ms();
                const int rj = L.rjob.empty() ? -1 : L.rjob[W[j].job];
                HostInstance I;
                I.n = n;
                I.D = hD + off[W[j].job];
                I.ld = n;
                I.B = &B;
                I.nbr = hN + off[W[j].job];
                I.app_tau = nullptr;  // no sorted taus: the apparent vertex of each edge instead
                I.napp = 0;
                I.app_w = hA + aoff[W[j].job];  // the apparent pairs found on the GPU
                I.t = o.t;
                std::vector<Leftover> &Lv = W[j].left;
                std::vector<HostPair> pairs;
                ReduceStats rs;
                const int ph = device_phase(rj);
                if (ph >= 0) {  // reduced on the device
                    const int64_t base = L.rleft[rj];
                    for (size_t q = 0; q < Lv.size(); ++q) {
                        HostPair P;
                        P.sigma = Lv[q].sigma;
                        P.birth = Lv[q].diam;
                        P.tau = L.rdeath[ph][base + (int64_t)q];
                        P.death = P.tau == NO_PIVOT ? INFINITY : L.rddiam[ph][base + (int64_t)q];
                        pairs.push_back(P);
                    }
                    rs.additions = L.radds[ph][rj];
                    S.device_columns[1] = (int64_t)Lv.size();
                } else {
                    std::sort(Lv.begin(), Lv.end(), [](const Leftover &x, const Leftover &y) {
                        return x.index < y.index;
                    });
                    reduce_leftovers(I, 1, Lv.data(), (int64_t)Lv.size(), inner, pairs, rs);
                }
                S.free_pivot[1] = rs.free_pivot;
                S.additions[1] = rs.additions;
                S.store_reads[1] = rs.reads;
                S.entries[1] = rs.entries;
                S.sweep_levels[1] = rs.levels;
                S.sweep_pivots[1] = rs.sweep_pivots;
                S.sweep_idle[1] = rs.sweep_idle;
                S.ms_sweep_walks = rs.sweep_walk_ms;
                int vs[2], vt[3];
                for (const HostPair &P : pairs) {
                    if (P.tau != NO_PIVOT && !(P.death > P.birth)) continue;
                    rpp_critical cr = {-1, -1, -1, -1};
                    decode_host(B, P.sigma, 1, n, vs);
                    youngest_edge(I, vs, 2, &cr.bu, &cr.bv);
                    if (P.tau != NO_PIVOT) {
                        decode_host(B, P.tau, 2, n, vt);
                        youngest_edge(I, vt, 3, &cr.du, &cr.dv);
                    }
                    add_interval(r, 1, P.birth, P.death, cr);
                }
                S.ms_host_reduce = now_ms() - a3;
            }
        }
        for (int q = 0; q <= c.max_dim; ++q) {
            sort_result(r, q);
            S.intervals[q] = (int64_t)r->iv[q].size();
        }
        S.ms_total = now_ms() - t0;
        res[j] = r;
    });
    // every cloud has its pairs: the device's first phase may stop, and the
    // workspace's next launch waits for it (the results here need nothing more)
    if (L.cancel) {
        __atomic_store_n(L.cancel, 1u, __ATOMIC_RELEASE);
        if (L.red[0] && L.pending) *L.pending = true;
    }
    for (int ph = 0; ph < 2; ++ph) {  // the reduction's buffers stay in use until it is done
        if (!L.red[ph] || (ph == 0 && L.cancel)) continue;
        cudaSetDevice(L.device);
        const cudaError_t e = cudaEventSynchronize(L.red[ph]);
        if (e != cudaSuccess) {
            for (rpp_result *r : res) rpp_result_free(r);
            return fail(RPP_E_CUDA, std::string("device reduction of the batched clouds: ") +
                                        cudaGetErrorString(e));
        }
    }
    for (int j = 0; j < k; ++j) {
        if (W[j].fallback) alone.push_back(idx[j]);
        else out[idx[j]] = res[j];
    }
    return Status();
}

}  // namespace

bool batch_fused_eligible(const rpp_context *ctx, const Instance &in) {
    return ctx->batch_fused && in.kind == RPP_INPUT_POINTS && in.max_dim <= 1 &&
           in.n <= BATCH_NMAX && (ctx->record & (RPP_RECORD_COLUMNS | RPP_RECORD_APPARENT)) == 0;
}

int64_t batch_bucket(const Instance &in) {
    return ((int64_t)bucket_nmax(in.n) << 32) | (int64_t)dimcap_of(in.dim);
}

size_t batch_device_bytes(const std::vector<Instance> &ins) {
    std::vector<int> idx(ins.size());
    uint64_t rows = 0;
    for (size_t i = 0; i < ins.size(); ++i) {
        idx[i] = (int)i;
        rows += (uint64_t)ins[i].n * (uint64_t)ins[i].n;
    }
    return launch_device_bytes(caps_of(ins, idx), rows) + 2 * sizeof(void *) * ins.size();
}

Status run_batch(rpp_context *ctx, Workspace &ws, const std::vector<Instance> &ins,
                 cudaStream_t s, rpp_result **out, Workspace *ws2) {
    RPP_CK(cudaSetDevice(ws.device));
    std::map<std::pair<int, int>, std::vector<int>> buckets;  // (nmax, dimcap) -> clouds
    std::vector<int> alone;
    for (int i = 0; i < (int)ins.size(); ++i) {
        out[i] = nullptr;
        if (batch_fused_eligible(ctx, ins[i]))
            buckets[{bucket_nmax(ins[i].n), dimcap_of(ins[i].dim)}].push_back(i);
        else
            alone.push_back(i);
    }
    auto cleanup = [&]() {
        // a launch that failed before its host half may leave a device
        // reduction writing into the workspace's buffers
        for (Workspace *w : {&ws, ws2})
            if (w && w->reduce_stream) cudaStreamSynchronize(w->reduce_stream);
        for (size_t i = 0; i < ins.size(); ++i)
            if (out[i]) {
                rpp_result_free(out[i]);
                out[i] = nullptr;
            }
    };
    struct Planned {
        std::vector<int> idx;
        int nmax, dimcap;
    };
    std::vector<Planned> plan;
    for (auto &kv : buckets) {
        const int cap = bucket_cap(kv.first.first);
        const std::vector<int> &all = kv.second;
        for (size_t o = 0; o < all.size(); o += (size_t)cap)
            plan.push_back({std::vector<int>(all.begin() + o,
                                             all.begin() + std::min(all.size(), o + cap)),
                            kv.first.first, kv.first.second});
    }
    // With a second workspace the device half of launch i + 1 runs (from this
    // thread, on the stream) while the host threads finish launch i; each
    // launch's buffers belong to one workspace until its host half is done.
    Launch L[2];
    Workspace *wsp[2] = {&ws, ws2 ? ws2 : &ws};
    const bool overlap = ws2 && ws2 != &ws && plan.size() > 1;
    std::vector<int> overflow;
    Status st;
    if (!plan.empty())
        st = launch_device(ctx, ws, ins, plan[0].idx, plan[0].nmax, plan[0].dimcap, s, L[0]);
    for (size_t i = 0; st.ok() && i < plan.size(); ++i) {
        Launch &cur = L[i & 1];
        const bool more = i + 1 < plan.size();
        Workspace &wn = *wsp[overlap ? (i + 1) & 1 : 0];
        if (!overlap) {
            st = launch_host(ctx, cur, out, overflow);
            if (st.ok() && more)
                st = launch_device(ctx, wn, ins, plan[i + 1].idx, plan[i + 1].nmax,
                                   plan[i + 1].dimcap, s, L[(i + 1) & 1]);
            continue;
        }
        Status hs;
        std::thread host([&] {
            try {
                hs = launch_host(ctx, cur, out, overflow);
            } catch (const std::exception &e) {
                hs = fail(RPP_E_NOMEM, std::string("batched host reduction: ") + e.what());
            }
        });
        if (more)
            st = launch_device(ctx, wn, ins, plan[i + 1].idx, plan[i + 1].nmax, plan[i + 1].dimcap,
                               s, L[(i + 1) & 1]);
        host.join();
        if (st.ok()) st = hs;
    }
    if (!st.ok()) {
        cleanup();
        return st;
    }
    // clouds run alone: not fusable, or their leftover columns overflowed the pool
    std::sort(overflow.begin(), overflow.end());
    alone.insert(alone.end(), overflow.begin(), overflow.end());
    for (int i : alone) {
        rpp_result *r = new rpp_result();
        st = run_instance(ctx, ws, ins[i], s, r);
        if (!st.ok()) {
            delete r;
            cleanup();
            st.msg = "cloud " + std::to_string(i) + ": " + st.msg;
            return st;
        }
        out[i] = r;
    }
    return Status();
}

}  // namespace rpp

extern "C" rpp_status rpp_barcodes_batched(rpp_context *ctx, int32_t batch,
                                           const float *const *data, const int64_t *n,
                                           const int32_t *dim, int32_t max_dim,
                                           const float *thresholds, const double *quantiles,
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
        in.quantile = quantiles ? quantiles[i] : 0.0;
        Status v = validate_instance(in);
        if (!v.ok()) {
            v.msg = "cloud " + std::to_string(i) + ": " + v.msg;
            return report(v);
        }
    }
    if (batch == 0) return RPP_OK;
    Workspace *ws = ctx->acquire();
    // a second workspace lets launches overlap (not under a memory budget,
    // which holds per workspace)
    Workspace *ws2 = ctx->budget == 0 ? ctx->acquire() : nullptr;
    Status s = run_batch(ctx, *ws, ins, (cudaStream_t)stream, out, ws2);
    if (ws2) ctx->release(ws2);
    ctx->release(ws);
    if (!s.ok()) return report(s);
    return RPP_OK;
}

extern "C" rpp_status rpp_context_set_device_reduce(rpp_context *ctx, int32_t mode) {
    if (!ctx) {
        set_last_error("rpp_context_set_device_reduce: ctx is NULL");
        return RPP_E_INVALID;
    }
    if (mode < 0 || mode > 2) {
        set_last_error("rpp_context_set_device_reduce: mode must be 0, 1 or 2");
        return RPP_E_INVALID;
    }
    ctx->device_reduce = mode;
    return RPP_OK;
}

extern "C" rpp_status rpp_context_set_batch(rpp_context *ctx, int32_t fused, int32_t autotune) {
    if (!ctx) {
        set_last_error("rpp_context_set_batch: ctx is NULL");
        return RPP_E_INVALID;
    }
    ctx->batch_fused = fused != 0;
    ctx->autotune = autotune != 0;
    return RPP_OK;
}

extern "C" rpp_status rpp_context_batch_tuning(rpp_context *ctx, int32_t nmax, int32_t *threads,
                                               int32_t *group) {
    if (!ctx || !threads || !group) {
        set_last_error("rpp_context_batch_tuning: NULL argument");
        return RPP_E_INVALID;
    }
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    auto it = ctx->batch_tuning.find(nmax);
    if (it == ctx->batch_tuning.end()) {
        *threads = 0;
        *group = 0;
        return RPP_OK;
    }
    *threads = it->second.threads;
    *group = it->second.group;
    return RPP_OK;
}
