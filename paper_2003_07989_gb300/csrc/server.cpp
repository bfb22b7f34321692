// server.cpp -- serving: requests of point clouds arrive over time and are
// admitted, as device memory and slots free up, onto slot workers that each own
// a CUDA stream and a workspace. Admitted requests overlap on the device (one
// stream per slot) and in their host reductions (one thread per slot).
//
// Admission: a request's device footprint is estimated from its simplex counts
// (the same buffer sizes the pipeline requests). A slot may take the request
// when the bytes held by the other slots plus the larger of its own held bytes
// and the estimate stay within the budget; an idle slot holding more than the
// request needs returns its buffers first. The queue is served first-fit in
// arrival order; a request passed over too often blocks later ones until it
// fits, so large requests are not starved.
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

#include "pipeline.h"

using namespace rpp;

namespace {

struct Request {
    uint64_t ticket = 0;
    std::vector<float> pts;
    Instance in;
    size_t est = 0;
    bool fused = false;  // runs in fused batches (clouds of the fused pass, max_batch > 1)
    int skipped = 0;
    bool done = false;
    rpp_result *res = nullptr;
    Status status;
};

}  // namespace

struct rpp_server {
    rpp_context *ctx = nullptr;
    rpp_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> reqs;
    std::deque<uint64_t> finished;  // tickets in completion order (rpp_server_next)
    std::vector<size_t> held;  // bytes reserved per slot
    std::vector<std::thread> workers;
    uint64_t next_ticket = 1;
    bool stop = false;

    size_t held_others(int k) const {
        size_t s = 0;
        for (size_t j = 0; j < held.size(); ++j)
            if ((int)j != k) s += held[j];
        return s;
    }
    void worker(int k);
};

void rpp_server::worker(int k) {
    cudaSetDevice(ctx->device);
    cudaStream_t s;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    Workspace *ws = new Workspace();
    ws->device = ctx->device;
    const size_t budget = cfg.device_bytes;
    const int max_skips = 8;
    std::vector<Request *> batch;
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> g(mu);
            for (;;) {
                if (stop && queue.empty()) break;
                // first fit in arrival order, with aging of passed-over requests
                for (auto it = queue.begin(); it != queue.end(); ++it) {
                    Request *q = *it;
                    bool fits = budget == 0 || held_others(k) + std::max(held[k], q->est) <= budget;
                    if (!fits && budget && held_others(k) + q->est <= budget &&
                        ws->device_bytes > q->est) {
                        // this slot's cached buffers are in the way: return them
                        delete ws;
                        ws = new Workspace();
                        ws->device = ctx->device;
                        held[k] = 0;
                        fits = true;
                    }
                    if (fits) {
                        r = q;
                        queue.erase(it);
                        break;
                    }
                    if (++q->skipped > max_skips) break;  // nobody may pass it any longer
                }
                if (r) break;
                if (!queue.empty() && held[k] > 0) {
                    // nothing fits: an idle slot gives its cached buffers back so
                    // that admission can always make progress
                    delete ws;
                    ws = new Workspace();
                    ws->device = ctx->device;
                    held[k] = 0;
                    cv_work.notify_all();
                    continue;
                }
                cv_work.wait(g);
            }
            if (!r) break;
            batch.assign(1, r);
            if (r->fused) {
                // continuous batching: waiting requests of the same size bucket
                // join this launch (one fused launch per batch) while the
                // batch's footprint fits next to the other slots
                std::vector<Instance> ins(1, r->in);
                size_t est = r->est;
                const int64_t bucket = batch_bucket(r->in);
                for (auto it = queue.begin();
                     it != queue.end() && (int)batch.size() < cfg.max_batch;) {
                    Request *q = *it;
                    if (!q->fused || batch_bucket(q->in) != bucket) {
                        ++it;
                        continue;
                    }
                    ins.push_back(q->in);
                    const size_t e = batch_device_bytes(ins);
                    if (budget == 0 || held_others(k) + std::max(held[k], e) <= budget) {
                        batch.push_back(q);
                        est = e;
                        it = queue.erase(it);
                    } else {
                        ins.pop_back();
                        ++it;
                    }
                }
                held[k] = std::max(held[k], est);
            } else {
                held[k] = std::max(held[k], r->est);
            }
        }
        std::vector<rpp_result *> res(batch.size(), nullptr);
        std::vector<Status> st(batch.size());
        if (batch.size() > 1 || batch[0]->fused) {
            std::vector<Instance> ins;
            for (Request *q : batch) ins.push_back(q->in);
            Status bs = run_batch(ctx, *ws, ins, s, res.data());
            if (!bs.ok()) {  // find the failing request: run each one alone
                for (size_t i = 0; i < batch.size(); ++i) {
                    res[i] = new rpp_result();
                    st[i] = run_instance(ctx, *ws, batch[i]->in, s, res[i]);
                    if (!st[i].ok()) {
                        delete res[i];
                        res[i] = nullptr;
                    }
                }
            }
        } else {
            res[0] = new rpp_result();
            st[0] = run_instance(ctx, *ws, batch[0]->in, s, res[0]);
            if (!st[0].ok()) {
                delete res[0];
                res[0] = nullptr;
            }
        }
        {
            std::lock_guard<std::mutex> g(mu);
            held[k] = ws->device_bytes;
            for (size_t i = 0; i < batch.size(); ++i) {
                batch[i]->res = res[i];
                batch[i]->status = st[i];
                batch[i]->done = true;
                finished.push_back(batch[i]->ticket);
            }
            // tickets taken by rpp_server_poll stay queued until skipped:
            // drop them now and then so that a poll-only user stays bounded
            if (finished.size() > 4096 && finished.size() > 2 * reqs.size()) {
                std::deque<uint64_t> keep;
                for (uint64_t t : finished)
                    if (reqs.count(t)) keep.push_back(t);
                finished.swap(keep);
            }
        }
        cv_done.notify_all();
        cv_work.notify_all();
    }
    delete ws;
    cudaStreamDestroy(s);
}

extern "C" {

rpp_status rpp_server_create(rpp_context *ctx, const rpp_server_config *cfg, rpp_server **out) {
    if (!ctx || !cfg || !out || cfg->max_slots < 1) {
        set_last_error("rpp_server_create: invalid arguments");
        return RPP_E_INVALID;
    }
    rpp_server *srv = new rpp_server();
    srv->ctx = ctx;
    srv->cfg = *cfg;
    srv->held.assign(cfg->max_slots, 0);
    for (int k = 0; k < cfg->max_slots; ++k) srv->workers.emplace_back(&rpp_server::worker, srv, k);
    *out = srv;
    return RPP_OK;
}

rpp_status rpp_server_submit(rpp_server *srv, const float *points, int64_t n, int32_t dim,
                             int32_t max_dim, float threshold, double quantile, uint64_t *ticket) {
    if (!srv || !points || !ticket) {
        set_last_error("rpp_server_submit: invalid arguments");
        return RPP_E_INVALID;
    }
    Request *r = new Request();
    r->in.kind = RPP_INPUT_POINTS;
    r->in.n = n;
    r->in.dim = dim;
    r->in.max_dim = max_dim;
    r->in.threshold = threshold;
    r->in.quantile = quantile;
    r->in.data = points;
    Status v = validate_instance(r->in);
    if (!v.ok()) {
        delete r;
        return report(v);
    }
    r->pts.resize((size_t)n * dim);
    if (is_device_pointer(points)) {
        cudaSetDevice(srv->ctx->device);
        if (cudaMemcpy(r->pts.data(), points, r->pts.size() * 4, cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
            delete r;
            set_last_error("rpp_server_submit: copying the points failed");
            return RPP_E_CUDA;
        }
    } else {
        std::memcpy(r->pts.data(), points, r->pts.size() * 4);
    }
    r->in.data = r->pts.data();
    r->fused = srv->cfg.max_batch > 1 && batch_fused_eligible(srv->ctx, r->in);
    r->est = r->fused ? batch_device_bytes({r->in}) : instance_device_bytes(r->in);
    if (srv->cfg.device_bytes && r->est > srv->cfg.device_bytes) {
        delete r;
        set_last_error("rpp_server_submit: request can never fit the server's memory bound");
        return RPP_E_BUSY;
    }
    {
        std::lock_guard<std::mutex> g(srv->mu);
        if (srv->stop) {
            delete r;
            set_last_error("rpp_server_submit: server is shutting down");
            return RPP_E_BUSY;
        }
        r->ticket = srv->next_ticket++;
        srv->reqs[r->ticket] = r;
        srv->queue.push_back(r);
        *ticket = r->ticket;
    }
    srv->cv_work.notify_one();
    return RPP_OK;
}

rpp_status rpp_server_poll(rpp_server *srv, uint64_t ticket, int32_t timeout_ms, rpp_result **out) {
    if (!srv || !out) {
        set_last_error("rpp_server_poll: invalid arguments");
        return RPP_E_INVALID;
    }
    *out = nullptr;
    std::unique_lock<std::mutex> g(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) {
        set_last_error("rpp_server_poll: unknown ticket");
        return RPP_E_INVALID;
    }
    Request *r = it->second;
    if (timeout_ms < 0) {
        srv->cv_done.wait(g, [&] { return r->done; });
    } else if (!srv->cv_done.wait_for(g, std::chrono::milliseconds(timeout_ms),
                                      [&] { return r->done; })) {
        return RPP_E_TIMEOUT;
    }
    srv->reqs.erase(it);
    g.unlock();
    rpp_status code = r->status.code;
    if (code != RPP_OK) set_last_error(r->status.msg);
    *out = r->res;
    delete r;
    return code;
}

rpp_status rpp_server_next(rpp_server *srv, int32_t timeout_ms, uint64_t *ticket,
                           rpp_result **out) {
    if (!srv || !ticket || !out) {
        set_last_error("rpp_server_next: invalid arguments");
        return RPP_E_INVALID;
    }
    *out = nullptr;
    *ticket = 0;
    std::unique_lock<std::mutex> g(srv->mu);
    Request *r = nullptr;
    auto ready = [&] {  // the oldest finished request not yet taken by rpp_server_poll
        while (!srv->finished.empty()) {
            auto it = srv->reqs.find(srv->finished.front());
            srv->finished.pop_front();
            if (it != srv->reqs.end()) {
                r = it->second;
                srv->reqs.erase(it);
                return true;
            }
        }
        return false;
    };
    if (timeout_ms < 0) {
        srv->cv_done.wait(g, ready);
    } else if (!srv->cv_done.wait_for(g, std::chrono::milliseconds(timeout_ms), ready)) {
        return RPP_E_TIMEOUT;
    }
    g.unlock();
    *ticket = r->ticket;
    rpp_status code = r->status.code;
    if (code != RPP_OK) set_last_error(r->status.msg);
    *out = r->res;
    delete r;
    return code;
}

void rpp_server_destroy(rpp_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    for (auto &t : srv->workers) t.join();
    for (auto &kv : srv->reqs) {
        rpp_result_free(kv.second->res);
        delete kv.second;
    }
    delete srv;
}

}  // extern "C"
