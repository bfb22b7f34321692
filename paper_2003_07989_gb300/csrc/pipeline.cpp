// pipeline.cpp -- one instance end to end: distances, threshold, H0, and per
// dimension p the filtration with clearing, the apparent-pair pass, the
// partition and the submatrix reduction (the flow of Fig. "framework" (b)).
//
// Host <-> device crossings (the paper's hybrid design, with H0 moved to the
// device: the minimum spanning forest is found by Boruvka rounds on the GPU
// and its edges are marked cleared there; only its n - 1 keys come back):
//   * after the partition of dimension p, the leftover columns and the apparent
//     pairs (sorted by tau) go to the host for the submatrix reduction;
//   * the deaths the host found return to the device as the clearing bitmap of
//     dimension p + 1, together with the apparent taus already there.
#include "pipeline.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <thread>

namespace rpp {

double now_ms() {
    return std::chrono::duration<double, std::milli>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

uint64_t quantile_rank(double q, uint64_t n) {
    const uint64_t m = n * (n - 1) / 2;
    uint64_t r = (uint64_t)std::ceil(q * (double)m);
    return std::max<uint64_t>(1, std::min<uint64_t>(r, m));
}

int bits_for(uint64_t x) {  // bits needed to write x (0 for x = 0)
    int b = 0;
    while (b < 64 && (x >> b)) ++b;
    return b;
}

Status fail(rpp_status code, const std::string &msg) {
    Status s;
    s.code = code;
    s.msg = msg;
    return s;
}

float bits_to_float(uint32_t b) {
    float f;
    std::memcpy(&f, &b, sizeof f);
    return f;
}

// ---------------------------------------------------------------------------
// workspace

Workspace::~Workspace() {
    if (reduce_stream) cudaStreamSynchronize(reduce_stream);  // nothing may still read the buffers
    DevBuf *d[] = {&X,    &Dsrc,  &D,      &state,   &binom,     &key_hi, &key_lo,
                   &tmp_hi, &tmp_lo, &tmp_val, &tiles, &hist,      &status, &pivot,
                   &pdiam, &app_tau, &app_sigma, &left, &bitmap, &mst,    &up, &nbr, &h0,
                   &state_tune, &csr_off, &csr_nbr, &sp_a, &sp_b, &sp_c, &sp_cnt, &aw,
                   &order};
    for (DevBuf *b : d)
        if (b->p) cudaFree(b->p);
    HostBuf *h[] = {&h_hi,    &h_lo,  &h_tau, &h_sigma, &h_left, &h_D,  &h_state,
                    &h_mst,   &h_up,  &h_nbr, &h_ehi,   &h_eab,  &h_aw};
    for (HostBuf *b : h)
        if (b->p) cudaFreeHost(b->p);
    DevBuf *bd[] = {&b_pts, &b_clouds, &b_order, &b_ctl, &b_D,   &b_mst,  &b_outs,
                    &b_left, &b_lcloud, &b_jobs, &b_off, &b_Dout, &b_nbr, &b_src,
                    &b_aw, &b_awout, &r_jobs, &r_left, &r_vpool, &r_vstart, &r_vcnt, &r_death, &r_ddiam,
                    &r_ekeys, &r_etmp, &r_esort, &r_ekaw,
                    &r_stat};
    for (DevBuf *b : bd)
        if (b->p) cudaFree(b->p);
    HostBuf *bh[] = {&hb_pts,  &hb_clouds, &hb_order, &hb_ctl, &hb_outs, &hb_mst,  &hb_left,
                     &hb_lcloud, &hb_jobs, &hb_off,   &hb_Dout, &hb_nbr, &hb_src, &hb_awout,
                     &hr_in,   &hr_out, &hr_out_b, &hr_cancel};
    if (ev_reduce) cudaEventDestroy(ev_reduce);
    if (ev_reduce_b) cudaEventDestroy(ev_reduce_b);
    if (ev_rows) cudaEventDestroy(ev_rows);
    if (reduce_stream) cudaStreamDestroy(reduce_stream);
    for (HostBuf *b : bh)
        if (b->p) cudaFreeHost(b->p);
    for (auto &g : graphs) cudaGraphExecDestroy(g.second);
    if (capture_stream) cudaStreamDestroy(capture_stream);
    for (cudaEvent_t e : events) cudaEventDestroy(e);
}

namespace {

// Per-stage device time from CUDA events recorded on the pipeline's stream
// around each stage (rpp_stats.stage_ms), plus kernel launch counts.
struct StageTimer {
    bool on = false;
    cudaStream_t s = nullptr;
    Workspace *ws = nullptr;
    size_t used = 0;
    int cur = -1;
    long long l0 = 0;
    cudaEvent_t start = nullptr;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
    int64_t launches[8] = {};
    cudaEvent_t get() {
        if (used == ws->events.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            ws->events.push_back(e);
        }
        return ws->events[used++];
    }
    void begin(int stage) {
        cur = stage;
        l0 = g_launches;
        if (!on) return;
        start = get();
        cudaEventRecord(start, s);
    }
    void end() {
        if (cur >= 0) launches[cur] += g_launches - l0;
        if (on) {
            cudaEvent_t e = get();
            cudaEventRecord(e, s);
            marks.push_back({cur, {start, e}});
        }
        cur = -1;
    }
    // after the stream is synchronised
    void collect(rpp_stats &S) {
        for (auto &m : marks) {
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, m.second.first, m.second.second);
            S.stage_ms[m.first] += ms;
        }
        for (int i = 0; i < 8; ++i) S.stage_launches[i] = launches[i];
    }
};

enum { ST_DIST = 0, ST_RADIUS, ST_BUILD, ST_SORT, ST_APPARENT, ST_PARTITION, ST_PAIRSORT, ST_OTHER };

// Neighbour lists on the host, for matrices too large for the GPU row sort.
void sort_rows_host(const float *D, int64_t ld, int64_t n, uint64_t *out, int threads) {
    std::atomic<int64_t> next(0);
    auto work = [&]() {
        for (int64_t r; (r = next.fetch_add(1)) < n;) {
            uint64_t *row = out + r * n;
            const float *d = D + r * ld;
            for (int64_t i = 0; i < n; ++i) {
                uint32_t bits;
                std::memcpy(&bits, d + i, 4);
                row[i] = ((uint64_t)bits << 32) | (uint64_t)i;
            }
            std::sort(row, row + n);
        }
    };
    std::vector<std::thread> pool;
    for (int i = 1; i < std::max(1, threads); ++i) pool.emplace_back(work);
    work();
    for (auto &t : pool) t.join();
}

}  // namespace

Status Workspace::dev(DevBuf &b, size_t bytes, void **out) {
    if (bytes == 0) bytes = 256;
    if (b.bytes < bytes) {
        size_t want = ((bytes + bytes / 4) + 255) & ~(size_t)255;
        const size_t others = device_bytes - b.bytes;
        if (budget && others + want > budget) want = (bytes + 255) & ~(size_t)255;
        if (budget && others + want > budget)
            return fail(RPP_E_NOMEM, "device workspace would exceed the context's memory budget");
        if (b.p) {
            cudaFree(b.p);
            device_bytes -= b.bytes;
            b.p = nullptr;
            b.bytes = 0;
        }
        cudaError_t e = cudaMalloc(&b.p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            return fail(RPP_E_NOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
        }
        b.bytes = want;
        device_bytes += want;
    }
    *out = b.p;
    return Status();
}

Status Workspace::host(HostBuf &b, size_t bytes, void **out) {
    if (bytes == 0) bytes = 256;
    if (b.bytes < bytes) {
        size_t want = ((bytes + bytes / 4) + 4095) & ~(size_t)4095;
        if (b.p) cudaFreeHost(b.p);
        b.p = nullptr;
        b.bytes = 0;
        cudaError_t e = cudaMallocHost(&b.p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(RPP_E_NOMEM, std::string("cudaMallocHost failed: ") + cudaGetErrorString(e));
        }
        b.bytes = want;
    }
    *out = b.p;
    return Status();
}

// ---------------------------------------------------------------------------
// helpers

void fill_binomial(int64_t n, int kmax, std::vector<uint64_t> &store, Binomial &B) {
    store.assign((size_t)(kmax + 1) * (n + 1), 0);
    const uint64_t SAT = ~0ull;
    for (int64_t v = 0; v <= n; ++v) {
        store[v] = 1;  // C(v, 0)
        for (int k = 1; k <= kmax; ++k) {
            if (v == 0) {
                store[(size_t)k * (n + 1)] = 0;
                continue;
            }
            // C(v, k) = C(v-1, k-1) + C(v-1, k)
            const uint64_t a = store[(size_t)(k - 1) * (n + 1) + v - 1];
            const uint64_t b = store[(size_t)k * (n + 1) + v - 1];
            store[(size_t)k * (n + 1) + v] =
                (a == SAT || b == SAT || a + b < a || a + b > (1ull << 63)) ? SAT : a + b;
        }
    }
    B.n = n;
    B.kmax = kmax;
    B.host = store.data();
}

cudaError_t allow_dynamic_smem(const void *fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> allowed;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(mu);
    size_t &a = allowed[{dev, fn}];
    if (bytes <= a) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) a = bytes;
    return e;
}

bool is_device_pointer(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

Status validate_instance(const Instance &in) {
    if (!in.data) return fail(RPP_E_INVALID, "data is NULL");
    if (in.n < 1) return fail(RPP_E_INVALID, "n must be >= 1");
    if (in.n > (1ll << 31) - 2) return fail(RPP_E_INVALID, "n too large");
    if (in.max_dim < 0 || in.max_dim > RPP_MAX_DIM)
        return fail(RPP_E_INVALID, "max_dim must be in [0, RPP_MAX_DIM]");
    if (in.kind != RPP_INPUT_POINTS && in.kind != RPP_INPUT_DISTANCES)
        return fail(RPP_E_INVALID, "unknown input kind");
    if (in.kind == RPP_INPUT_POINTS && in.dim < 1) return fail(RPP_E_INVALID, "dim must be >= 1");
    if (std::isnan(in.threshold) || in.threshold < 0.0f)
        return fail(RPP_E_INVALID, "threshold must be >= 0 or +INFINITY");
    if (in.quantile != 0.0 && !(in.quantile > 0.0 && in.quantile <= 1.0))
        return fail(RPP_E_INVALID, "quantile must be in (0, 1]");
    // every index up to dimension max_dim + 1 must fit in 63 bits
    std::vector<uint64_t> store;
    Binomial B;
    fill_binomial(in.n, in.max_dim + 2, store, B);
    if (B.at(in.max_dim + 2, in.n) == ~0ull)
        return fail(RPP_E_OVERFLOW, "C(n, max_dim + 2) does not fit the 63-bit index");
    // H0's forest keys hold 32-bit edge indices (for max_dim = 0 too)
    if ((uint64_t)in.n * (uint64_t)(in.n - 1) / 2 >= (1ull << 32))
        return fail(RPP_E_OVERFLOW, "C(n, 2) does not fit the 32-bit edge index (n > 92682)");
    return Status();
}

// Device bytes run_instance requests for an instance, including the growth
// slack of Workspace::dev (what a workspace holds after running it).
size_t instance_device_bytes(const Instance &in) {
    std::vector<uint64_t> store;
    Binomial B;
    const int kmax = in.max_dim + 2 < 3 ? 3 : in.max_dim + 2;
    fill_binomial(in.n, kmax, store, B);
    const int64_t n = in.n, ld = (n + 31) / 32 * 32;
    uint64_t maxcand = 0;
    for (int p = 1; p <= std::max(1, in.max_dim); ++p) maxcand = std::max(maxcand, B.at(p + 1, n));
    auto slack = [](size_t b) { return ((b + b / 4) + 255) & ~(size_t)255; };
    size_t total = 0;
    total += slack(store.size() * 8) + slack(sizeof(DevState)) + slack((size_t)n * ld * 4);
    if (in.kind == RPP_INPUT_POINTS) total += slack((size_t)n * in.dim * 4);
    else total += slack((size_t)n * n * 4);
    const size_t per = 4 + 8 + 4 + 8 + 8 + 1 + 8 + 4 + 8 + 8 + sizeof(Leftover);
    total += slack(maxcand * per) + slack(radix_scratch_bytes(maxcand));
    total += slack((size_t)n * 4) + slack(maxcand / 8 + 8) + slack(maxcand * 8);
    total += slack((size_t)n * n * 8);  // neighbour lists
    total += slack(512 + (size_t)n * 32);  // the H0 forest
    total += slack(build_order_bytes(maxcand));  // the ordered build's look-back
    return total + 64 * 256;  // per-buffer rounding
}

// ---------------------------------------------------------------------------
// the pipeline

namespace {

struct DimOutput {
    std::vector<HostPair> pairs;  // host-found pairs (zero-length included) and essentials
};

}  // namespace

void add_interval(rpp_result *res, int q, float b, float d, const rpp_critical &c) {
    rpp_interval iv;
    iv.birth = b;
    iv.death = d;
    res->iv[q].push_back(iv);
    res->cr[q].push_back(c);
}

void sort_result(rpp_result *res, int q) {
    std::vector<size_t> idx(res->iv[q].size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
    auto &iv = res->iv[q];
    auto &cr = res->cr[q];
    std::sort(idx.begin(), idx.end(), [&](size_t a, size_t b) {
        if (iv[a].birth != iv[b].birth) return iv[a].birth < iv[b].birth;
        if (iv[a].death != iv[b].death) return iv[a].death < iv[b].death;
        const int32_t ka[4] = {cr[a].bu, cr[a].bv, cr[a].du, cr[a].dv};
        const int32_t kb[4] = {cr[b].bu, cr[b].bv, cr[b].du, cr[b].dv};
        return std::lexicographical_compare(ka, ka + 4, kb, kb + 4);
    });
    std::vector<rpp_interval> iv2(idx.size());
    std::vector<rpp_critical> cr2(idx.size());
    for (size_t i = 0; i < idx.size(); ++i) {
        iv2[i] = iv[idx[i]];
        cr2[i] = cr[idx[i]];
    }
    iv.swap(iv2);
    cr.swap(cr2);
}

// Launch shape of the single-instance apparent pass for dimension p and the
// size bucket of n (the next power of two): the context's tuned one, or, on
// the bucket's first instance (with autotuning on), the fastest of the
// candidate shapes timed on this instance's columns (the default shape unless
// another is more than 3% faster). Every shape writes the
// same outputs; the timing launches count into a scratch copy of the state,
// so the call's counters are those of the one real launch.
static Status apparent_shape(rpp_context *ctx, Workspace &ws, int p, int64_t n, DevState *st,
                             const std::function<void(int, DevState *)> &launch, cudaStream_t s,
                             int *group) {
    int64_t bucket = 1;
    while (bucket < n) bucket <<= 1;
    const std::pair<int, int64_t> key(p, bucket);
    *group = ctx->tuning_for(n, p).group;
    {
        std::lock_guard<std::mutex> g(ctx->tune_mu);
        auto it = ctx->apparent_tuning.find(key);
        if (it != ctx->apparent_tuning.end()) {
            *group = it->second;
            return Status();
        }
    }
    if (!ctx->autotune) return Status();
    void *vp;
    RPP_TRY(ws.dev(ws.state_tune, sizeof(DevState), &vp));
    DevState *scratch = (DevState *)vp;
    RPP_CK(cudaMemcpyAsync(scratch, st, sizeof(DevState), cudaMemcpyDeviceToDevice, s));
    cudaEvent_t e0, e1;
    RPP_CK(cudaEventCreate(&e0));
    RPP_CK(cudaEventCreate(&e1));
    // each shape: one warm-up launch, then the best of three; the default
    // shape keeps the bucket unless another is more than 3% faster
    const int fallback = *group;
    float base_ms = 0.0f, best = 0.0f;
    std::vector<std::pair<int, float>> timed;
    for (int g : {fallback, 8, 82, 42, 44, 4, 141, 142, 181, 121, 143, 144, 122}) {
        if (g == fallback && !timed.empty()) continue;
        float ms = 0.0f, low = 0.0f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, s);
            launch(g, scratch);
            cudaEventRecord(e1, s);
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return fail(RPP_E_CUDA, std::string("apparent-pass tuning: ") + cudaGetErrorString(e));
            }
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep == 1 || (rep > 1 && ms < low)) low = ms;
        }
        timed.push_back({g, low});
    }
    base_ms = timed[0].second;
    best = base_ms;
    for (const auto &gt : timed)
        if (gt.second < best && gt.second < 0.97f * base_ms) {
            best = gt.second;
            *group = gt.first;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    ctx->apparent_tuning.emplace(key, *group);
    return Status();
}

// The stages every entry point starts with: the binomial table (rows
// 0..kmax, cached per workspace), the zeroed device state, the distance
// matrix (from points with the fixed formula, or a caller's matrix copied and
// validated) with row stride ld = n rounded up to 32, the enclosing radius R
// and the threshold st->t = min(t, R) (+inf for a quantile, set later).
struct Prologue {
    uint64_t *d_binom = nullptr;
    DevState *st = nullptr;
    DevState *hst = nullptr;  // pinned host copy for read-backs
    float *D = nullptr;
};

static Status prologue(Workspace &ws, const Instance &in, int kmax, cudaStream_t s, StageTimer &T,
                       Prologue &P) {
    const int64_t n = in.n;
    const int64_t ld = (n + 31) / 32 * 32;
    void *vp;
    if (ws.binom_n != n || ws.binom_k < kmax) {
        fill_binomial(n, kmax, ws.binom_store, ws.binom_host);
        ws.binom_n = n;
        ws.binom_k = kmax;
        ws.binom_on_device = false;
    }
    RPP_TRY(ws.dev(ws.binom, ws.binom_store.size() * 8, &vp));
    uint64_t *d_binom = (uint64_t *)vp;
    if (!ws.binom_on_device) {
        RPP_CK(cudaMemcpyAsync(d_binom, ws.binom_store.data(), ws.binom_store.size() * 8,
                               cudaMemcpyHostToDevice, s));
        RPP_CK(cudaStreamSynchronize(s));  // the host table may be refilled later
        ws.binom_on_device = true;
    }

    // device state
    RPP_TRY(ws.dev(ws.state, sizeof(DevState), &vp));
    DevState *st = (DevState *)vp;
    RPP_TRY(ws.host(ws.h_state, sizeof(DevState), &vp));
    DevState *hst = (DevState *)vp;
    RPP_CK(cudaMemsetAsync(st, 0, sizeof(DevState), s));

    // distances
    RPP_TRY(ws.dev(ws.D, (size_t)n * ld * sizeof(float), &vp));
    float *D = (float *)vp;
    if (in.kind == RPP_INPUT_POINTS) {
        const float *X = in.data;
        if (!is_device_pointer(X)) {
            RPP_TRY(ws.dev(ws.X, (size_t)n * in.dim * sizeof(float), &vp));
            RPP_CK(cudaMemcpyAsync(vp, X, (size_t)n * in.dim * sizeof(float),
                                   cudaMemcpyHostToDevice, s));
            X = (const float *)vp;
        }
        T.begin(ST_DIST);
        launch_distance_matrix(X, n, in.dim, D, ld, s);
        T.end();
    } else {
        const float *src = in.data;
        if (!is_device_pointer(src)) {
            RPP_TRY(ws.dev(ws.Dsrc, (size_t)n * n * sizeof(float), &vp));
            RPP_CK(cudaMemcpyAsync(vp, src, (size_t)n * n * sizeof(float), cudaMemcpyHostToDevice,
                                   s));
            src = (const float *)vp;
        }
        T.begin(ST_DIST);
        launch_copy_validate_distances(src, n, D, ld, st, s);
        T.end();
    }
    const float t_user = in.quantile > 0.0 ? INFINITY : in.threshold;
    T.begin(ST_RADIUS);
    launch_enclosing_radius(D, n, ld, st, t_user, s);
    T.end();
    RPP_CK(cudaGetLastError());
    P.d_binom = d_binom;
    P.st = st;
    P.hst = hst;
    P.D = D;
    return Status();
}

// The filtration construction of dimension p alone (no clearing): the
// prologue, every p-simplex with diameter <= min(t, R) built and sorted in
// coboundary order, then optionally copied to the caller's arrays (device or
// host memory). The sort's key count stays on the device until the end.
Status run_filtration(rpp_context *ctx, Workspace &ws, const Instance &in, int p, cudaStream_t s,
                      float *diam_out, uint64_t *cidx_out, int64_t capacity, int64_t *count,
                      rpp_stats &S) {
    const double t0 = now_ms();
    RPP_TRY(validate_instance(in));
    if (p < 1 || p > in.max_dim) return fail(RPP_E_INVALID, "p must be in [1, RPP_MAX_DIM]");
    if (in.n < p + 1) return fail(RPP_E_INVALID, "n must be at least p + 1");
    RPP_CK(cudaSetDevice(ws.device));
    const int64_t n = in.n;
    const int64_t ld = (n + 31) / 32 * 32;
    std::memset(&S, 0, sizeof S);
    S.n = n;
    S.max_dim = p;
    StageTimer T;
    T.on = (ctx->record & RPP_RECORD_TIMING) != 0;
    T.s = s;
    T.ws = &ws;
    const long long launches0 = g_launches;
    Prologue pro;
    RPP_TRY(prologue(ws, in, std::max(3, p + 2), s, T, pro));
    const Binomial &B = ws.binom_host;
    const uint64_t cand = B.at(p + 1, n);
    if (cand >= (1ull << 32))
        return fail(RPP_E_NOMEM, "more than 2^32 candidate simplices in dimension p");
    S.candidates[p] = (int64_t)cand;
    uint32_t *key_hi, *tmp_hi;
    uint64_t *key_lo, *tmp_lo;
    void *sort_scratch;
    RPP_TRY(ws.dev(ws.key_hi, cand * 4, (void **)&key_hi));
    RPP_TRY(ws.dev(ws.key_lo, cand * 8, (void **)&key_lo));
    RPP_TRY(ws.dev(ws.tmp_hi, cand * 4, (void **)&tmp_hi));
    RPP_TRY(ws.dev(ws.tmp_lo, cand * 8, (void **)&tmp_lo));
    RPP_TRY(ws.dev(ws.tiles, radix_scratch_bytes(cand), &sort_scratch));
    unsigned long long *order;
    RPP_TRY(ws.dev(ws.order, build_order_bytes(cand), (void **)&order));
    T.begin(ST_BUILD);
    launch_build_columns(pro.D, ld, n, p, pro.d_binom, cand, nullptr, pro.st, key_hi, key_lo, s,
                         order);
    T.end();
    T.begin(ST_SORT);  // the columns arrive in index order: the diameter digits alone
    radix_sort(key_hi, key_lo, nullptr, tmp_hi, tmp_lo, nullptr, sort_scratch, cand,
               &pro.st->ncols, 0, &pro.st->err, s, &pro.st->sort_passes[p]);
    T.end();
    RPP_CK(cudaGetLastError());
    const double a = now_ms();
    RPP_CK(cudaMemcpyAsync(pro.hst, pro.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    RPP_CK(cudaStreamSynchronize(s));
    S.ms_device = now_ms() - a;
    const DevState &h = *pro.hst;
    if (h.err & ~(unsigned)ERR_INTERNAL) return fail(RPP_E_INVALID, "invalid input distances");
    if (h.err & ERR_INTERNAL) return fail(RPP_E_CUDA, "a bounded device wait ran out (sort)");
    const uint64_t N = h.ncols;
    S.threshold = h.t;
    S.enclosing_radius = h.R;
    S.columns[p] = (int64_t)N;
    S.sort_passes[p] = (int64_t)h.sort_passes[p];
    *count = (int64_t)N;
    if (diam_out || cidx_out) {
        if ((int64_t)N > capacity)
            return fail(RPP_E_INVALID, "capacity is below the column count (" + std::to_string(N) +
                                           ")");
        if (N > 0) {
            if (diam_out) {  // ~bits(diameter) back to diameters, in the scratch buffer
                launch_invert_u32(key_hi, N, tmp_hi, s);
                RPP_CK(cudaMemcpyAsync(diam_out, tmp_hi, N * 4, cudaMemcpyDefault, s));
            }
            if (cidx_out) RPP_CK(cudaMemcpyAsync(cidx_out, key_lo, N * 8, cudaMemcpyDefault, s));
            RPP_CK(cudaStreamSynchronize(s));
        }
    }
    if (T.on) RPP_CK(cudaStreamSynchronize(s));
    T.collect(S);
    S.kernel_launches = g_launches - launches0;
    S.ms_total = now_ms() - t0;
    return Status();
}

Status run_instance(rpp_context *ctx, Workspace &ws, const Instance &in, cudaStream_t s,
                    rpp_result *res) {
    const double t0 = now_ms();
    double dev_ms = 0.0, red_ms = 0.0, h0_ms = 0.0;
    RPP_TRY(validate_instance(in));
    RPP_CK(cudaSetDevice(ws.device));
    const int64_t n = in.n;
    const int max_dim = in.max_dim;
    const int64_t ld = (n + 31) / 32 * 32;
    res->max_dim = max_dim;
    for (int q = 0; q <= RPP_MAX_DIM; ++q) {
        res->iv[q].clear();
        res->cr[q].clear();
    }
    rpp_stats &S = res->stats;
    std::memset(&S, 0, sizeof S);
    S.n = n;
    S.max_dim = max_dim;
    StageTimer T;
    T.on = (ctx->record & RPP_RECORD_TIMING) != 0;
    T.s = s;
    T.ws = &ws;
    const long long launches0 = g_launches;
    unsigned long long scanned_prev = 0;

    // binomial table, state, distances, enclosing radius and threshold
    const int kmax = max_dim + 2 < 3 ? 3 : max_dim + 2;
    void *vp;
    Prologue pro;
    RPP_TRY(prologue(ws, in, kmax, s, T, pro));
    const Binomial &B = ws.binom_host;
    uint64_t *d_binom = pro.d_binom;
    DevState *st = pro.st;
    DevState *hst = pro.hst;
    float *D = pro.D;
    if (in.census) {  // every edge: neither a threshold nor the enclosing radius
        static const float inf = INFINITY;
        RPP_CK(cudaMemcpyAsync(&st->t, &inf, sizeof(float), cudaMemcpyHostToDevice, s));
    }

    // host copy of D for the reduction and the realising edges
    RPP_TRY(ws.host(ws.h_D, (size_t)n * ld * sizeof(float), &vp));
    float *hD = (float *)vp;
    RPP_CK(cudaMemcpyAsync(hD, D, (size_t)n * ld * sizeof(float), cudaMemcpyDeviceToHost, s));

    // buffers sized for the largest dimension
    // sized for dimension 1 here; dimensions p >= 2 grow them to their need
    const uint64_t maxcand = std::max<uint64_t>(1, B.at(2, n));
    uint32_t *key_hi, *tmp_hi;
    void *sort_scratch;
    uint64_t *key_lo, *tmp_lo, *tmp_val, *pivot, *app_tau, *app_sigma;
    uint8_t *status;
    float *pdiam;
    Leftover *left;
    RPP_TRY(ws.dev(ws.key_hi, maxcand * 4, (void **)&key_hi));
    RPP_TRY(ws.dev(ws.key_lo, maxcand * 8, (void **)&key_lo));
    RPP_TRY(ws.dev(ws.tmp_hi, maxcand * 4, (void **)&tmp_hi));
    RPP_TRY(ws.dev(ws.tmp_lo, maxcand * 8, (void **)&tmp_lo));
    RPP_TRY(ws.dev(ws.tmp_val, maxcand * 8, (void **)&tmp_val));
    RPP_TRY(ws.dev(ws.tiles, radix_scratch_bytes(maxcand), &sort_scratch));
    RPP_TRY(ws.dev(ws.status, maxcand, (void **)&status));
    RPP_TRY(ws.dev(ws.pivot, maxcand * 8, (void **)&pivot));
    RPP_TRY(ws.dev(ws.pdiam, maxcand * 4, (void **)&pdiam));
    RPP_TRY(ws.dev(ws.app_tau, maxcand * 8, (void **)&app_tau));
    RPP_TRY(ws.dev(ws.app_sigma, maxcand * 8, (void **)&app_sigma));
    RPP_TRY(ws.dev(ws.left, maxcand * sizeof(Leftover), (void **)&left));
    // Growth for a dimension p >= 2 of `cap` columns: the key arrays and the
    // sort's scratch before its build (they hold nothing live then), the
    // per-column outputs after it (the build may read the previous
    // dimension's apparent taus). A buffer that grows is reallocated, so the
    // stream is drained first.
    auto grow_columns = [&](uint64_t cap) -> Status {
        cap = std::max<uint64_t>(1, cap);
        if (ws.key_lo.bytes < cap * 8 || ws.tiles.bytes < radix_scratch_bytes(cap))
            RPP_CK(cudaStreamSynchronize(s));
        RPP_TRY(ws.dev(ws.key_hi, cap * 4, (void **)&key_hi));
        RPP_TRY(ws.dev(ws.key_lo, cap * 8, (void **)&key_lo));
        RPP_TRY(ws.dev(ws.tmp_hi, cap * 4, (void **)&tmp_hi));
        RPP_TRY(ws.dev(ws.tmp_lo, cap * 8, (void **)&tmp_lo));
        RPP_TRY(ws.dev(ws.tiles, radix_scratch_bytes(cap), &sort_scratch));
        return Status();
    };
    auto grow_outputs = [&](uint64_t cap) -> Status {
        cap = std::max<uint64_t>(1, cap);
        if (ws.app_tau.bytes < cap * 8 || ws.left.bytes < cap * sizeof(Leftover))
            RPP_CK(cudaStreamSynchronize(s));
        RPP_TRY(ws.dev(ws.tmp_val, cap * 8, (void **)&tmp_val));
        RPP_TRY(ws.dev(ws.status, cap, (void **)&status));
        RPP_TRY(ws.dev(ws.pivot, cap * 8, (void **)&pivot));
        RPP_TRY(ws.dev(ws.pdiam, cap * 4, (void **)&pdiam));
        RPP_TRY(ws.dev(ws.app_tau, cap * 8, (void **)&app_tau));
        RPP_TRY(ws.dev(ws.app_sigma, cap * 8, (void **)&app_sigma));
        RPP_TRY(ws.dev(ws.left, cap * sizeof(Leftover), (void **)&left));
        return Status();
    };
    // the thresholded construction's state (dimensions p >= 2)
    unsigned long long *csr_off = nullptr;
    uint32_t *csr_nbr = nullptr;
    uint64_t *sp_prev = nullptr;  // every simplex of the last sparse dimension
    uint64_t sp_prev_count = 0;
    bool sp_prev_valid = false;

    auto read_state = [&]() -> Status {
        double a = now_ms();
        RPP_CK(cudaMemcpyAsync(hst, st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
        RPP_CK(cudaStreamSynchronize(s));
        dev_ms += now_ms() - a;
        return Status();
    };

    RPP_TRY(read_state());
    if (hst->err) {
        std::string m = "invalid input:";
        if (hst->err & ERR_NONFINITE) m += " non-finite value;";
        if (hst->err & ERR_NEGATIVE) m += " negative distance;";
        if (hst->err & ERR_ASYMMETRIC) m += " asymmetric matrix;";
        if (hst->err & ERR_DIAGONAL) m += " nonzero diagonal;";
        return fail(RPP_E_INVALID, m);
    }
    S.enclosing_radius = hst->R;
    float t = hst->t;

    HostInstance I;
    I.n = n;
    I.D = hD;
    I.ld = ld;
    I.B = &B;

    // H0 on the device: forest edges (keys (bits(d) << 32) | ~index), their
    // count, and their positions among the dimension-1 columns
    unsigned long long *h0_mst = nullptr, *h0_best = nullptr;
    unsigned *h0_count = nullptr, *h0_flags = nullptr;
    uint32_t *h0_pos = nullptr;
    int32_t *h0_comp = nullptr, *h0_parent = nullptr, *h0_next = nullptr;
    unsigned char *h0_host = nullptr;  // pinned: count (16 B), keys, positions
    if (n >= 2) {
        unsigned char *q;
        const size_t nb = (size_t)n;
        RPP_TRY(ws.dev(ws.h0, 512 + nb * (3 * 4 + 8 + 8 + 4), (void **)&q));
        RPP_TRY(ws.host(ws.h_mst, 16 + nb * (8 + 4), (void **)&h0_host));
        h0_comp = (int32_t *)q;
        h0_parent = h0_comp + nb;
        h0_next = h0_parent + nb;
        h0_best = (unsigned long long *)(q + ((nb * 12 + 15) & ~(size_t)15));
        h0_mst = h0_best + nb;
        h0_pos = (uint32_t *)(h0_mst + nb);
        h0_count = (unsigned *)(h0_pos + nb);
        h0_flags = h0_count + 1;  // 64 words
    }
    uint64_t edges_begin = 0, edges_count = 0;  // dimension-1 columns (MST edges included)
    // the apparent vertex of every edge (dimension 1), for vertices that fit 16 bits
    const bool use_aw = !in.census && max_dim >= 1 && n <= 65535;
    uint16_t *d_aw = nullptr;
    std::vector<uint64_t> prev_deaths;  // host-found deaths of the previous dimension
    uint64_t prev_napp = 0;

    if (n >= 2) {
        // ---- dimension 1 columns: every edge inside the threshold, sorted ----
        const uint64_t m = B.at(2, n);
        S.candidates[1] = (int64_t)m;
        // build, sort, forest, apparent pass and partition are queued without
        // a host round trip: their column count stays in device memory
        // (st->ncols), and grids are sized for the m candidates
        unsigned long long *order;
        RPP_TRY(ws.dev(ws.order, build_order_bytes(m), (void **)&order));
        T.begin(ST_BUILD);
        launch_build_columns(D, ld, n, 1, d_binom, m, nullptr, st, key_hi, key_lo, s, order);
        T.end();
        RPP_CK(cudaGetLastError());
        T.begin(ST_SORT);  // the edges arrive in index order: the diameter digits alone
        radix_sort(key_hi, key_lo, nullptr, tmp_hi, tmp_lo, nullptr, sort_scratch, m, &st->ncols,
                   0, &st->err, s, &st->sort_passes[1]);
        T.end();
        RPP_CK(cudaGetLastError());
        uint64_t begin = 0;
        uint64_t cols = m;  // a bound until the state is read back
        const unsigned long long *d_cols = &st->ncols;
        if (in.quantile > 0.0) {
            RPP_TRY(read_state());
            const uint64_t N = hst->ncols;
            // threshold = ceil(q m)-th smallest distance; distances above R were
            // dropped, and if the quantile lies above R, R itself is used.
            const uint64_t r = quantile_rank(in.quantile, (uint64_t)n);
            if (r <= N) {
                uint32_t kh;
                RPP_CK(cudaMemcpyAsync(&kh, key_hi + (N - r), 4, cudaMemcpyDeviceToHost, s));
                RPP_CK(cudaStreamSynchronize(s));
                t = bits_to_float(~kh);
                T.begin(ST_OTHER);
                launch_lower_bound_u32(key_hi, N, kh, &st->begin, s);
                T.end();
                RPP_CK(cudaMemcpyAsync(&st->t, &t, sizeof(float), cudaMemcpyHostToDevice, s));
                RPP_TRY(read_state());
                begin = hst->begin;
            }
            cols = N - begin;
            d_cols = nullptr;
        }
        S.threshold = t;
        I.t = t;
        edges_begin = begin;

        // ---- H0: the minimum spanning forest inside t, on the device ----
        const double a0 = now_ms();
        T.begin(ST_OTHER);
        launch_h0_forest(D, ld, n, st, h0_comp, h0_parent, h0_next, h0_best, h0_mst, h0_count,
                         h0_flags, s);
        T.end();
        RPP_CK(cudaGetLastError());
        const uint32_t *hi1 = key_hi + begin;
        const uint64_t *lo1 = key_lo + begin;
        const bool dim1 = max_dim >= 1 && cols > 0;
        if (dim1) {  // its edges are the cleared dimension-1 columns
            RPP_CK(cudaMemsetAsync(status, 0, cols, s));
            T.begin(ST_OTHER);
            launch_h0_clear(h0_mst, h0_count, n, hi1, lo1, cols, d_cols, status, h0_pos, s);
            T.end();
            RPP_CK(cudaGetLastError());
        }
        RPP_CK(cudaMemcpyAsync(h0_host, h0_count, 4, cudaMemcpyDeviceToHost, s));
        RPP_CK(cudaMemcpyAsync(h0_host + 16, h0_mst, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
        if (dim1)
            RPP_CK(cudaMemcpyAsync(h0_host + 16 + (size_t)n * 8, h0_pos, (size_t)n * 4,
                                   cudaMemcpyDeviceToHost, s));
        h0_ms += now_ms() - a0;
        if ((ctx->record & RPP_RECORD_COLUMNS) && max_dim >= 1) {
            if (d_cols) {
                RPP_TRY(read_state());
                cols = hst->ncols;
                d_cols = nullptr;
            }
            std::vector<uint32_t> hh(cols);
            std::vector<uint64_t> ll(cols);
            RPP_CK(cudaMemcpyAsync(hh.data(), key_hi + begin, cols * 4, cudaMemcpyDeviceToHost, s));
            RPP_CK(cudaMemcpyAsync(ll.data(), key_lo + begin, cols * 8, cudaMemcpyDeviceToHost, s));
            RPP_CK(cudaStreamSynchronize(s));
            const unsigned nm = *(const unsigned *)h0_host;
            const uint32_t *pos = (const uint32_t *)(h0_host + 16 + (size_t)n * 8);
            std::vector<char> cl(cols, 0);
            for (unsigned i = 0; i < nm && cols > 0; ++i) cl[pos[i]] = 1;
            for (uint64_t i = 0; i < cols; ++i)
                if (!cl[i]) {
                    res->col_diam[1].push_back(bits_to_float(~hh[i]));
                    res->col_idx[1].push_back(ll[i]);
                }
            res->has_cols[1] = true;
        }

        if (dim1) {
            // each edge's apparent vertex: the host's owner test for
            // dimension 1 reads it directly, so the apparent taus need no
            // sort (they still clear dimension 2)
            if (use_aw) {
                RPP_TRY(ws.dev(ws.aw, B.at(2, n) * 2, (void **)&d_aw));
                RPP_CK(cudaMemsetAsync(d_aw, 0xFF, B.at(2, n) * 2, s));
            }
            // the apparent taus of dimension 1 are read only to clear
            // dimension 2, to be recorded, or as the sorted owner test when
            // the apparent vertices are not kept; otherwise the pass skips
            // their indices and the partition only counts the pairs
            const bool taus1 = d_aw == nullptr || max_dim >= 2 ||
                               (ctx->record & RPP_RECORD_APPARENT) != 0;
            auto run = [&](int g, DevState *state) {
                launch_apparent(D, ld, n, 1, d_binom, hi1, lo1, cols, d_cols, state, status,
                                pivot, pdiam, d_aw, g, ctx->sms, s, taus1);
            };
            int group;
            RPP_TRY(apparent_shape(ctx, ws, 1, n, st, run, s, &group));
            T.begin(ST_APPARENT);
            run(group, st);
            T.end();
            T.begin(ST_PARTITION);
            launch_partition(status, hi1, lo1, pivot, pdiam, cols, d_cols,
                             taus1 ? app_tau : nullptr, taus1 ? app_sigma : nullptr, left, st, s);
            T.end();
            RPP_CK(cudaGetLastError());
        }
    } else {
        S.threshold = t;
        I.t = t;
    }

    // H0 intervals: one death per forest edge, one essential class per component
    {
        unsigned nm = 0;
        if (n >= 2) {
            RPP_TRY(read_state());  // the forest's copies are in
            if (hst->err & ERR_INTERNAL)
                return fail(RPP_E_CUDA, "a bounded device loop or wait ran out (H0 forest or sort)");
            edges_count = hst->ncols - edges_begin;
            nm = *(const unsigned *)h0_host;
            const unsigned long long *keys = (const unsigned long long *)(h0_host + 16);
            int v[2];
            for (unsigned i = 0; i < nm; ++i) {
                const float d = bits_to_float((uint32_t)(keys[i] >> 32));
                if (!(d > 0.0f)) continue;  // zero-length (duplicate points)
                decode_host(B, (uint64_t)(~(uint32_t)keys[i]), 1, n, v);
                rpp_critical c = {-1, -1, v[0], v[1]};
                add_interval(res, 0, 0.0f, d, c);
            }
            S.cleared[1] = (int64_t)nm;
            S.columns[1] = (int64_t)edges_count - S.cleared[1];
        }
        for (int64_t i = 0; i < n - (int64_t)nm; ++i) {
            rpp_critical c = {-1, -1, -1, -1};
            add_interval(res, 0, 0.0f, INFINITY, c);
        }
    }

    // Dimensions p >= 2 take the thresholded construction (cliques of the
    // threshold graph) when the edges inside t are a small share of all
    // edges, or when some C(n, p+1) is too large to enumerate; else every
    // index. One choice for all of them: a thresholded dimension builds its
    // simplices from the full list the one below it left.
    bool sparse_dims = false;
    if (max_dim >= 2 && n >= 2) {
        const uint64_t m1 = B.at(2, n);
        const double density = m1 ? (double)edges_count / (double)m1 : 1.0;
        bool huge = false;
        for (int p = 2; p <= max_dim; ++p) huge |= B.at(p + 1, n) >= (1ull << 32);
        sparse_dims = ctx->sparse_mode == 1 ||
                      (ctx->sparse_mode == 0 && (density < SPARSE_DENSITY || huge));
    }

    // ---- dimensions p = 1 .. max_dim ----
    for (int p = 1; p <= max_dim && n >= 2; ++p) {
        if (p >= 2) {
            const uint64_t cand = B.at(p + 1, n);
            S.candidates[p] = (int64_t)cand;
            S.cleared[p] = (int64_t)(prev_napp + prev_deaths.size());
            const bool sparse = sparse_dims;
            if (!sparse && cand >= (1ull << 32))
                return fail(RPP_E_NOMEM, "more than 2^32 candidate simplices in dimension " +
                                             std::to_string(p) + " (the thresholded path is off)");
            // the previous dimension's deaths: apparent taus (sorted on the
            // device) and the host's pairs, sorted here
            std::sort(prev_deaths.begin(), prev_deaths.end());
            uint64_t *up = nullptr;
            if (!prev_deaths.empty()) {
                RPP_TRY(ws.dev(ws.up, prev_deaths.size() * 8, (void **)&up));
                RPP_TRY(ws.host(ws.h_up, prev_deaths.size() * 8, &vp));
                std::memcpy(vp, prev_deaths.data(), prev_deaths.size() * 8);
                RPP_CK(cudaMemcpyAsync(up, vp, prev_deaths.size() * 8, cudaMemcpyHostToDevice, s));
            }
            uint64_t cap = cand;  // columns the build may write
            RPP_CK(cudaMemsetAsync(&st->ncols, 0, sizeof(unsigned long long), s));
            if (!sparse) {
                RPP_TRY(grow_columns(cap));
                // clearing bitmap from the deaths of dimension p-1
                uint32_t *bitmap;
                RPP_TRY(ws.dev(ws.bitmap, (cand + 31) / 32 * 4, (void **)&bitmap));
                RPP_CK(cudaMemsetAsync(bitmap, 0, (cand + 31) / 32 * 4, s));
                T.begin(ST_OTHER);
                launch_bitmap_set(app_tau, prev_napp, bitmap, s);
                if (up) launch_bitmap_set(up, prev_deaths.size(), bitmap, s);
                T.end();
                T.begin(ST_BUILD);
                unsigned long long *order;
                RPP_TRY(ws.dev(ws.order, build_order_bytes(cand), (void **)&order));
                launch_build_columns(D, ld, n, p, d_binom, cand, bitmap, st, key_hi, key_lo, s,
                                     order);
                T.end();
            } else {
                S.sparse[p] = 1;
                if (!csr_off) {  // the threshold graph, once per instance
                    RPP_TRY(ws.dev(ws.csr_off, (size_t)(n + 1) * 8, (void **)&csr_off));
                    T.begin(ST_OTHER);
                    launch_csr_build(D, ld, n, st, csr_off, nullptr, false, s);
                    T.end();
                    unsigned long long total = 0;
                    RPP_CK(cudaMemcpyAsync(&total, csr_off + n, 8, cudaMemcpyDeviceToHost, s));
                    RPP_CK(cudaStreamSynchronize(s));
                    RPP_TRY(ws.dev(ws.csr_nbr, std::max<size_t>(4, total * 4), (void **)&csr_nbr));
                    T.begin(ST_OTHER);
                    launch_csr_build(D, ld, n, st, csr_off, csr_nbr, true, s);
                    T.end();
                }
                // the (p-1)-simplices inside t: the edges (dimension 1's sorted
                // keys, copied aside) or every simplex the previous sparse
                // build listed
                const uint64_t *prev;
                uint64_t nprev;
                if (p == 2) {
                    RPP_TRY(ws.dev(ws.sp_a, std::max<uint64_t>(1, edges_count) * 8, &vp));
                    if (edges_count)
                        RPP_CK(cudaMemcpyAsync(vp, key_lo + edges_begin, edges_count * 8,
                                               cudaMemcpyDeviceToDevice, s));
                    prev = (const uint64_t *)vp;
                    nprev = edges_count;
                } else if (sp_prev_valid) {
                    prev = sp_prev;
                    nprev = sp_prev_count;
                } else {
                    return fail(RPP_E_CUDA, "thresholded build: no list of the previous dimension");
                }
                const bool keep_all = p < max_dim;
                unsigned long long *cnt;
                RPP_TRY(ws.dev(ws.sp_cnt, 16, (void **)&cnt));
                RPP_CK(cudaMemsetAsync(cnt, 0, 16, s));
                T.begin(ST_BUILD);
                launch_sparse_build(D, ld, n, p, d_binom, prev, nprev, csr_off, csr_nbr, st,
                                    app_tau, prev_napp, up, up ? prev_deaths.size() : 0, false,
                                    cnt, nullptr, nullptr, 0, nullptr, 0, s);
                T.end();
                unsigned long long counts[2];
                RPP_CK(cudaMemcpyAsync(counts, cnt, 16, cudaMemcpyDeviceToHost, s));
                RPP_CK(cudaStreamSynchronize(s));
                cap = counts[1];
                RPP_TRY(grow_columns(cap));
                uint64_t *all_out = nullptr;
                if (keep_all) {  // the other list buffer (prev may live in one of them)
                    DevBuf &dst = (p == 2 || prev == (const uint64_t *)ws.sp_b.p) ? ws.sp_c : ws.sp_b;
                    RPP_TRY(ws.dev(dst, std::max<uint64_t>(1, counts[0]) * 8, &vp));
                    all_out = (uint64_t *)vp;
                }
                RPP_CK(cudaMemsetAsync(cnt, 0, 16, s));
                T.begin(ST_BUILD);
                launch_sparse_build(D, ld, n, p, d_binom, prev, nprev, csr_off, csr_nbr, st,
                                    app_tau, prev_napp, up, up ? prev_deaths.size() : 0, true,
                                    cnt, key_hi, key_lo, cap, all_out, counts[0], s);
                T.end();
                RPP_CK(cudaMemcpyAsync(&st->ncols, cnt + 1, 8, cudaMemcpyDeviceToDevice, s));
                sp_prev = all_out;
                sp_prev_count = counts[0];
                sp_prev_valid = keep_all;
            }
            RPP_CK(cudaGetLastError());
            // the apparent taus of p-1 have been read: the per-column outputs
            // may grow now
            RPP_TRY(grow_outputs(cap));
            // as in dimension 1, the count stays on the device until the
            // partition has run
            uint64_t N = cap;
            const unsigned long long *d_n = &st->ncols;
            T.begin(ST_SORT);
            // the dense build writes its columns in index order (the
            // diameter digits alone); the thresholded one does not
            radix_sort(key_hi, key_lo, nullptr, tmp_hi, tmp_lo, nullptr, sort_scratch, cap,
                       &st->ncols, S.sparse[p] ? bits_for(cand - 1) : 0, &st->err, s,
                       &st->sort_passes[p]);
            T.end();
            if (ctx->record & RPP_RECORD_COLUMNS) {
                RPP_TRY(read_state());
                N = hst->ncols;
                d_n = nullptr;
                std::vector<uint32_t> hh(N);
                res->col_idx[p].resize(N);
                RPP_CK(cudaMemcpyAsync(hh.data(), key_hi, N * 4, cudaMemcpyDeviceToHost, s));
                RPP_CK(cudaMemcpyAsync(res->col_idx[p].data(), key_lo, N * 8,
                                       cudaMemcpyDeviceToHost, s));
                RPP_CK(cudaStreamSynchronize(s));
                res->col_diam[p].resize(N);
                for (uint64_t i = 0; i < N; ++i) res->col_diam[p][i] = bits_to_float(~hh[i]);
                res->has_cols[p] = true;
            }
            RPP_CK(cudaMemsetAsync(status, 0, N, s));
            RPP_CK(cudaMemsetAsync(&st->napp, 0, 2 * sizeof(unsigned long long), s));
            if (S.sparse[p]) {
                T.begin(ST_APPARENT);
                launch_apparent_sparse(D, ld, n, p, d_binom, csr_off, csr_nbr, key_hi, key_lo, N,
                                       d_n, st, status, pivot, pdiam, ctx->sms, s);
                T.end();
            } else {
                auto run = [&](int g, DevState *state) {
                    launch_apparent(D, ld, n, p, d_binom, key_hi, key_lo, N, d_n, state, status,
                                    pivot, pdiam, nullptr, g, ctx->sms, s);
                };
                int group;
                RPP_TRY(apparent_shape(ctx, ws, p, n, st, run, s, &group));
                T.begin(ST_APPARENT);
                run(group, st);
                T.end();
            }
            T.begin(ST_PARTITION);
            launch_partition(status, key_hi, key_lo, pivot, pdiam, N, d_n, app_tau, app_sigma,
                             left, st, s);
            T.end();
            RPP_CK(cudaGetLastError());
        }
        RPP_TRY(read_state());
        if (hst->err & ERR_INTERNAL)
            return fail(RPP_E_CUDA, "a bounded device wait ran out (sort)");
        if (p >= 2) S.columns[p] = (int64_t)hst->ncols;
        S.sort_passes[p] = (int64_t)hst->sort_passes[p];
        const uint64_t napp = hst->napp, nleft = hst->nleft;
        S.apparent[p] = (int64_t)napp;
        S.leftover[p] = (int64_t)nleft;
        S.scanned[p] = (int64_t)(hst->scanned - scanned_prev);
        scanned_prev = hst->scanned;
        if (in.census) {  // the census ends with the apparent-pair pass
            RPP_CK(cudaStreamSynchronize(s));
            T.collect(S);
            S.kernel_launches = g_launches - launches0;
            S.ms_device = dev_ms;
            S.ms_host_h0 = h0_ms;
            S.ms_total = now_ms() - t0;
            return Status();
        }
        const bool record_app = (ctx->record & RPP_RECORD_APPARENT) != 0;
        const bool next_sparse = p < max_dim && sparse_dims;
        const bool by_vertex = p == 1 && d_aw != nullptr;  // owner test from the vertices
        if (record_app || (nleft > 0 && !by_vertex) || next_sparse) {
            // the apparent taus sorted: the second layer of the pair store (the
            // sigmas ride along only when the pairs are recorded; the host
            // reduction takes the owner of an apparent tau as its youngest facet)
            T.begin(ST_PAIRSORT);
            radix_sort(nullptr, app_tau, record_app ? app_sigma : nullptr, nullptr, tmp_lo,
                       tmp_val, sort_scratch, napp, nullptr, bits_for(B.at(p + 2, n) - 1),
                       &st->err, s);
            T.end();
            RPP_CK(cudaGetLastError());
        }
        if (record_app) {
            res->app_tau[p].resize(napp);
            res->app_sigma[p].resize(napp);
            RPP_CK(cudaMemcpyAsync(res->app_tau[p].data(), app_tau, napp * 8,
                                   cudaMemcpyDeviceToHost, s));
            RPP_CK(cudaMemcpyAsync(res->app_sigma[p].data(), app_sigma, napp * 8,
                                   cudaMemcpyDeviceToHost, s));
            RPP_CK(cudaStreamSynchronize(s));
            res->has_app[p] = true;
        }
        DimOutput out;
        if (nleft > 0) {
            Leftover *hleft;
            uint64_t *htau;
            RPP_TRY(ws.host(ws.h_left, nleft * sizeof(Leftover), (void **)&hleft));
            if (by_vertex) {
                uint16_t *haw;
                RPP_TRY(ws.host(ws.h_aw, B.at(2, n) * 2, (void **)&haw));
                RPP_CK(cudaMemcpyAsync(haw, d_aw, B.at(2, n) * 2, cudaMemcpyDeviceToHost, s));
                I.app_w = haw;
                I.app_tau = nullptr;
                I.napp = 0;
            } else {
                RPP_TRY(ws.host(ws.h_tau, napp * 8, (void **)&htau));
                RPP_CK(cudaMemcpyAsync(htau, app_tau, napp * 8, cudaMemcpyDeviceToHost, s));
                I.app_w = nullptr;
                I.app_tau = htau;
                I.napp = napp;
            }
            if (p == 1 && edges_count > 0 && n <= 65535) {
                // the sorted edges as vertex pairs, for the sweep of long walks
                // (tmp_hi is free once the pair sort, if any, has run)
                uint32_t *he, *hab;
                RPP_TRY(ws.host(ws.h_ehi, edges_count * 4, (void **)&he));
                RPP_TRY(ws.host(ws.h_eab, edges_count * 4, (void **)&hab));
                T.begin(ST_OTHER);
                launch_edge_pairs(key_lo + edges_begin, edges_count, tmp_hi, s);
                T.end();
                RPP_CK(cudaMemcpyAsync(he, key_hi + edges_begin, edges_count * 4,
                                       cudaMemcpyDeviceToHost, s));
                RPP_CK(cudaMemcpyAsync(hab, tmp_hi, edges_count * 4, cudaMemcpyDeviceToHost, s));
                I.edge_hi = he;
                I.edge_ab = hab;
                I.nedges = (int64_t)edges_count;
            } else {
                I.edge_hi = nullptr;
                I.edge_ab = nullptr;
                I.nedges = 0;
            }
            // the state again (the pair sort's wait flag), read with the copies below
            RPP_CK(cudaMemcpyAsync(hst, st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
            if (!I.nbr) {  // neighbour lists for the lazy coboundaries, once per instance
                uint64_t *dn, *hn;
                RPP_TRY(ws.dev(ws.nbr, (size_t)n * n * 8, (void **)&dn));
                RPP_TRY(ws.host(ws.h_nbr, (size_t)n * n * 8, (void **)&hn));
                T.begin(ST_OTHER);
                const bool gpu_sorted = launch_sort_rows(D, ld, n, dn, s);
                T.end();
                if (gpu_sorted)
                    RPP_CK(cudaMemcpyAsync(hn, dn, (size_t)n * n * 8, cudaMemcpyDeviceToHost, s));
                RPP_CK(cudaMemcpyAsync(hleft, left, nleft * sizeof(Leftover),
                                       cudaMemcpyDeviceToHost, s));
                double a = now_ms();
                RPP_CK(cudaStreamSynchronize(s));
                dev_ms += now_ms() - a;
                if (!gpu_sorted) sort_rows_host(hD, ld, n, hn, ctx->host_threads);
                I.nbr = hn;
            } else {
                double a = now_ms();
                RPP_CK(cudaMemcpyAsync(hleft, left, nleft * sizeof(Leftover),
                                       cudaMemcpyDeviceToHost, s));
                RPP_CK(cudaStreamSynchronize(s));
                dev_ms += now_ms() - a;
            }
            if (hst->err & ERR_INTERNAL)
                return fail(RPP_E_CUDA, "a bounded device wait ran out (pair sort)");
            double a = now_ms();
            std::sort(hleft, hleft + nleft,
                      [](const Leftover &x, const Leftover &y) { return x.index < y.index; });
            ReduceStats rs;
            reduce_leftovers(I, p, hleft, (int64_t)nleft, ctx->host_threads, out.pairs, rs);
            S.free_pivot[p] = rs.free_pivot;
            S.additions[p] = rs.additions;
            S.store_reads[p] = rs.reads;
            S.entries[p] = rs.entries;
            S.sweep_levels[p] = rs.levels;
            S.sweep_pivots[p] = rs.sweep_pivots;
            S.sweep_idle[p] = rs.sweep_idle;
            S.ms_sweep_walks += rs.sweep_walk_ms;
            red_ms += now_ms() - a;
        }
        // intervals of dimension p and the deaths that clear dimension p + 1
        prev_deaths.clear();
        int vs[RPP_MAX_DIM + 2], vt[RPP_MAX_DIM + 3];
        for (const HostPair &P : out.pairs) {
            if (P.tau != NO_PIVOT) prev_deaths.push_back(P.tau);
            if (P.tau != NO_PIVOT && !(P.death > P.birth)) continue;  // zero length
            rpp_critical c = {-1, -1, -1, -1};
            decode_host(B, P.sigma, p, n, vs);
            youngest_edge(I, vs, p + 1, &c.bu, &c.bv);
            if (P.tau != NO_PIVOT) {
                decode_host(B, P.tau, p + 1, n, vt);
                youngest_edge(I, vt, p + 2, &c.du, &c.dv);
            }
            add_interval(res, p, P.birth, P.death, c);
        }
        prev_napp = napp;
    }
    if ((n >= 2 && max_dim >= 1) || T.on) RPP_CK(cudaStreamSynchronize(s));
    T.collect(S);
    S.kernel_launches = g_launches - launches0;

    for (int q = 0; q <= max_dim; ++q) {
        sort_result(res, q);
        S.intervals[q] = (int64_t)res->iv[q].size();
    }
    S.ms_device = dev_ms;
    S.ms_host_reduce = red_ms;
    S.ms_host_h0 = h0_ms;
    S.ms_total = now_ms() - t0;
    return Status();
}

}  // namespace rpp
