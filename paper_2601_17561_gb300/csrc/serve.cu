// Serving form: a request loop that keeps the encrypted database resident, admits query eyes as
// they arrive, batches them (continuous batching: a batch starts when it is full or its oldest
// eye has waited `window_us`, and requests that arrive while a batch runs join the next one), and
// runs query preparation, the grouped CCMM and the fold per batch (Section 5: computing servers
// batch up to 32 query eyes; Appendix C.5 batch scaling).
//
// Device resources: one set of compute buffers (prepared query, scores, CRT scratch) used by the
// compute stream, and two I/O slots, each with its own copy stream, device buffers for the batch's
// query ciphertext and folded scores, and page-locked host staging.  Batch k+1's gather and
// host-to-device copy and batch k-1's device-to-host copy and scatter overlap batch k's compute.
// Every wait is bounded (condition-variable waits with timeouts, event polling).
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "icm_internal.h"

using namespace icm;

namespace icm {
icm_status api_fail(icm_status s, const char *msg);
}

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t ticket;
    const uint64_t *host_ct;     // [Lq][rho][K]
    uint64_t *host_out;          // sum_c [L][G][M_c]
    Clock::time_point t_submit, t_done;
    int state = 0;               // 0 pending, 1 running, 2 done, 3 failed
    icm_status status = ICM_OK;
};

struct Slot {
    cudaStream_t cs = nullptr;           // copy stream
    cudaEvent_t h2d = nullptr, comp = nullptr, d2h = nullptr;
    void *d_ct = nullptr;                // [Lq][max_eyes*rho][K]
    std::vector<void *> d_fold;          // per chunk [L][max_eyes*G][M_c]
    uint64_t *h_ct = nullptr;            // pinned staging
    std::vector<uint64_t *> h_fold;      // pinned staging per chunk
    std::vector<Req *> reqs;
    bool busy = false;
};

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

struct icm_server {
    icm_ctx *ctx;
    std::vector<const icm_db *> dbs;
    icm_server_cfg cfg;
    uint32_t G = 0;
    size_t eye_ct_words = 0, eye_out_words = 0;
    cudaStream_t comp = nullptr;
    void *d_op = nullptr, *d_ws = nullptr;
    std::vector<void *> d_sc;
    size_t op_bytes = 0, ws_bytes = 0;
    std::vector<size_t> sc_bytes, fo_bytes;
    Slot slots[2];
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req *> pending;
    std::unordered_map<uint64_t, Req *> reqs;
    uint64_t next_ticket = 1, n_done = 0, n_batches = 0, eyes_batched = 0;
    bool stop = false;
    std::thread worker;

    ~icm_server();
    void run();
    icm_status launch(Slot &s, std::vector<Req *> &batch);
    void finish(Slot &s, icm_status st);
};

namespace {

// Device layout of the server workspace: compute buffers, then the two slots.
struct Carve {
    size_t op, sc_total, ws, slot_ct, slot_fo_total, total;
};

Carve carve(const icm_ctx *c, const icm_db *const *dbs, size_t n, const icm_server_cfg *cfg) {
    Carve k{};
    const icm_form f = cfg->form;
    icm_query_op_bytes(c, cfg->max_eyes, f, &k.op);
    for (size_t i = 0; i < n; ++i) {
        size_t sc = 0, fo = 0;
        icm_scores_bytes(c, dbs[i], cfg->max_eyes, 0, &sc);
        icm_scores_bytes(c, dbs[i], cfg->max_eyes, 1, &fo);
        k.sc_total += a256(sc);
        k.slot_fo_total += a256(fo);
    }
    icm_match_batch_workspace_bytes(c, dbs, n, cfg->max_eyes, f, &k.ws);
    icm_query_ct_bytes(c, cfg->max_eyes, &k.slot_ct);
    k.total = a256(k.op) + k.sc_total + a256(k.ws) + 2 * (a256(k.slot_ct) + k.slot_fo_total);
    return k;
}

}  // namespace

icm_server::~icm_server() {
    for (auto &s : slots) {
        if (s.cs) cudaStreamDestroy(s.cs);
        if (s.h2d) cudaEventDestroy(s.h2d);
        if (s.comp) cudaEventDestroy(s.comp);
        if (s.d2h) cudaEventDestroy(s.d2h);
        if (s.h_ct) cudaFreeHost(s.h_ct);
        for (auto *p : s.h_fold) cudaFreeHost(p);
    }
    if (comp) cudaStreamDestroy(comp);
    for (auto &kv : reqs) delete kv.second;
}

icm_status icm_server::launch(Slot &s, std::vector<Req *> &batch) {
    const uint32_t n = (uint32_t)batch.size();
    const uint32_t Lq = ctx->p.n_limbs_q, rho = ctx->p.rho, K = ctx->K;
    // gather the eyes' ciphertexts into the staging layout [Lq][n*rho][K]
    for (uint32_t l = 0; l < Lq; ++l)
        for (uint32_t e = 0; e < n; ++e)
            std::memcpy(s.h_ct + ((size_t)l * n * rho + (size_t)e * rho) * K, batch[e]->host_ct + (size_t)l * rho * K,
                        (size_t)rho * K * 8);
    size_t ct_bytes = 0;
    icm_query_ct_bytes(ctx, n, &ct_bytes);
    cudaError_t e = cudaMemcpyAsync(s.d_ct, s.h_ct, ct_bytes, cudaMemcpyHostToDevice, s.cs);
    if (e == cudaSuccess) e = cudaEventRecord(s.h2d, s.cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(comp, s.h2d, 0);
    if (e != cudaSuccess) return api_fail(ICM_ECUDA, cudaGetErrorString(e));
    icm_query *q = nullptr;
    icm_status st = icm_query_prepare(ctx, s.d_ct, n, cfg.form, d_op, op_bytes, comp, &q);
    std::vector<icm_scores *> sc(dbs.size(), nullptr), fo(dbs.size(), nullptr);
    if (st == ICM_OK)
        st = icm_match_batch(ctx, dbs.data(), dbs.size(), q, d_sc.data(), sc_bytes.data(), d_ws, ws_bytes, comp, sc.data());
    for (size_t i = 0; st == ICM_OK && i < dbs.size(); ++i)
        st = icm_fold(ctx, sc[i], s.d_fold[i], fo_bytes[i], comp, &fo[i]);
    icm_query_destroy(q);
    for (auto *p : sc) icm_scores_destroy(p);
    for (auto *p : fo) icm_scores_destroy(p);
    if (st != ICM_OK) return st;
    e = cudaEventRecord(s.comp, comp);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s.cs, s.comp, 0);
    for (size_t i = 0; e == cudaSuccess && i < dbs.size(); ++i) {
        const size_t bytes = (size_t)ctx->p.n_limbs * n * G * dbs[i]->lay.M * 8;
        e = cudaMemcpyAsync(s.h_fold[i], s.d_fold[i], bytes, cudaMemcpyDeviceToHost, s.cs);
    }
    if (e == cudaSuccess) e = cudaEventRecord(s.d2h, s.cs);
    if (e != cudaSuccess) return api_fail(ICM_ECUDA, cudaGetErrorString(e));
    return ICM_OK;
}

// Scatter every eye's folded scores to its output, then mark the requests done (or failed).
void icm_server::finish(Slot &s, icm_status st) {
    const uint32_t n = (uint32_t)s.reqs.size();
    const uint32_t L = ctx->p.n_limbs;
    if (st == ICM_OK) {
        for (uint32_t e = 0; e < n; ++e) {
            uint64_t *dst = s.reqs[e]->host_out;
            for (size_t i = 0; i < dbs.size(); ++i) {
                const uint64_t M = dbs[i]->lay.M;
                for (uint32_t l = 0; l < L; ++l) {
                    std::memcpy(dst, s.h_fold[i] + ((size_t)l * n * G + (size_t)e * G) * M, (size_t)G * M * 8);
                    dst += (size_t)G * M;
                }
            }
        }
    }
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(mu);
    for (Req *r : s.reqs) {
        r->t_done = now;
        r->status = st;
        r->state = st == ICM_OK ? 2 : 3;
        ++n_done;
    }
    s.reqs.clear();
    s.busy = false;
    cv.notify_all();
}

void icm_server::run() {
    cudaSetDevice(ctx->device);
    for (;;) {
        // completions
        for (auto &s : slots) {
            if (!s.busy || s.reqs.empty()) continue;
            const cudaError_t q = cudaEventQuery(s.d2h);
            if (q == cudaErrorNotReady) continue;
            finish(s, q == cudaSuccess ? ICM_OK : ICM_ECUDA);
        }
        std::vector<Req *> batch;
        Slot *free_slot = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            bool busy = slots[0].busy || slots[1].busy;
            if (stop && pending.empty() && !busy) return;
            for (auto &s : slots) if (!s.busy) { free_slot = &s; break; }
            bool go = false;
            if (free_slot && !pending.empty()) {
                const auto waited = std::chrono::duration_cast<std::chrono::microseconds>(Clock::now() - pending.front()->t_submit).count();
                go = pending.size() >= cfg.max_eyes || waited >= (long long)cfg.window_us || stop;
            }
            if (go) {
                while (!pending.empty() && batch.size() < cfg.max_eyes) {
                    batch.push_back(pending.front());
                    pending.front()->state = 1;
                    pending.pop_front();
                }
                free_slot->busy = true;
                free_slot->reqs = batch;
                ++n_batches;
                eyes_batched += batch.size();
            } else {
                // nothing to launch: sleep until a request arrives or a poll interval passes
                cv.wait_for(lk, std::chrono::microseconds(busy ? 200 : 2000));
                continue;
            }
        }
        const icm_status st = launch(*free_slot, batch);
        if (st != ICM_OK) finish(*free_slot, st);
    }
}

extern "C" {

icm_status icm_server_device_bytes(const icm_ctx *c, const icm_db *const *dbs, size_t n_dbs, const icm_server_cfg *cfg,
                                   size_t *bytes) {
    if (!c || !dbs || !cfg || !bytes || n_dbs == 0 || n_dbs > ICM_MAX_CHUNKS || cfg->max_eyes == 0 || cfg->max_eyes > 32)
        return api_fail(ICM_EINVAL, "bad arguments");
    *bytes = carve(c, dbs, n_dbs, cfg).total;
    return ICM_OK;
}

icm_status icm_server_create(icm_ctx *c, const icm_db *const *dbs, size_t n_dbs, const icm_server_cfg *cfg, void *dev_ws,
                             size_t ws_bytes, icm_server **out) {
    size_t need = 0;
    icm_status st = icm_server_device_bytes(c, dbs, n_dbs, cfg, &need);
    if (st != ICM_OK) return st;
    if (!out || !dev_ws || ws_bytes < need) return api_fail(ICM_ENOMEM, "server workspace too small");
    if (!c->have_keys) return api_fail(ICM_EINVAL, "icm_keygen has not run");
    icm_server *s = new (std::nothrow) icm_server();
    if (!s) return api_fail(ICM_ENOMEM, "host allocation");
    s->ctx = c;
    s->dbs.assign(dbs, dbs + n_dbs);
    s->cfg = *cfg;
    if (s->cfg.max_pending == 0) s->cfg.max_pending = 4096;
    s->G = (c->p.rho + c->p.fold_k - 1) / c->p.fold_k;
    s->eye_ct_words = (size_t)c->p.n_limbs_q * c->p.rho * c->K;
    for (size_t i = 0; i < n_dbs; ++i) s->eye_out_words += (size_t)c->p.n_limbs * s->G * dbs[i]->lay.M;
    const Carve k = carve(c, dbs, n_dbs, cfg);
    char *w = (char *)dev_ws;
    s->d_op = w; s->op_bytes = k.op; w += a256(k.op);
    for (size_t i = 0; i < n_dbs; ++i) {
        size_t sc = 0, fo = 0;
        icm_scores_bytes(c, dbs[i], cfg->max_eyes, 0, &sc);
        icm_scores_bytes(c, dbs[i], cfg->max_eyes, 1, &fo);
        s->d_sc.push_back(w); s->sc_bytes.push_back(sc); w += a256(sc);
        s->fo_bytes.push_back(fo);
    }
    s->d_ws = k.ws ? w : nullptr; s->ws_bytes = k.ws; w += a256(k.ws);
    cudaError_t e = cudaStreamCreateWithFlags(&s->comp, cudaStreamNonBlocking);
    for (auto &sl : s->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.h2d, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.comp, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.d2h, cudaEventDisableTiming);
        sl.d_ct = w; w += a256(k.slot_ct);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_ct, k.slot_ct);
        for (size_t i = 0; i < n_dbs; ++i) {
            sl.d_fold.push_back(w); w += a256(s->fo_bytes[i]);
            uint64_t *h = nullptr;
            if (e == cudaSuccess) e = cudaMallocHost((void **)&h, s->fo_bytes[i]);
            sl.h_fold.push_back(h);
        }
    }
    if (e != cudaSuccess) { delete s; return api_fail(ICM_ECUDA, cudaGetErrorString(e)); }
    try {
        s->worker = std::thread([s] { s->run(); });
    } catch (...) {
        delete s;
        return api_fail(ICM_ENOMEM, "worker thread");
    }
    *out = s;
    return ICM_OK;
}

icm_status icm_server_eye_words(const icm_server *s, size_t *ct_words, size_t *out_words) {
    if (!s) return api_fail(ICM_EINVAL, "null server");
    if (ct_words) *ct_words = s->eye_ct_words;
    if (out_words) *out_words = s->eye_out_words;
    return ICM_OK;
}

icm_status icm_server_submit(icm_server *s, const uint64_t *host_ct, uint64_t *host_out, uint64_t *ticket) {
    if (!s || !host_ct || !host_out || !ticket) return api_fail(ICM_EINVAL, "null argument");
    Req *r = new (std::nothrow) Req();
    if (!r) return api_fail(ICM_ENOMEM, "host allocation");
    r->host_ct = host_ct;
    r->host_out = host_out;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) { delete r; return api_fail(ICM_EINVAL, "server is stopping"); }
        if (s->pending.size() >= s->cfg.max_pending) { delete r; return api_fail(ICM_ENOMEM, "admission queue full"); }
        r->ticket = s->next_ticket++;
        s->reqs[r->ticket] = r;
        s->pending.push_back(r);
    }
    s->cv.notify_all();
    *ticket = r->ticket;
    return ICM_OK;
}

icm_status icm_server_wait(icm_server *s, uint64_t ticket, uint32_t timeout_ms, double *latency_ms) {
    if (!s) return api_fail(ICM_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return api_fail(ICM_EINVAL, "unknown ticket");
    Req *r = it->second;
    if (!s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [r] { return r->state >= 2; }))
        return api_fail(ICM_ETIMEOUT, "request not finished in time");
    const icm_status st = r->status;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    s->reqs.erase(it);
    delete r;
    if (st != ICM_OK) return api_fail(st, "batch failed");
    return ICM_OK;
}

icm_status icm_server_stats(icm_server *s, uint64_t *n_done, uint64_t *n_batches, double *mean_batch) {
    if (!s) return api_fail(ICM_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (n_done) *n_done = s->n_done;
    if (n_batches) *n_batches = s->n_batches;
    if (mean_batch) *mean_batch = s->n_batches ? (double)s->eyes_batched / s->n_batches : 0.0;
    return ICM_OK;
}

icm_status icm_server_destroy(icm_server *s, uint32_t timeout_ms) {
    if (!s) return ICM_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    // the worker drains pending and in-flight batches; bound the wait
    const auto t0 = Clock::now();
    icm_status st = ICM_OK;
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->pending.empty() && !s->slots[0].busy && !s->slots[1].busy) break;
        }
        if (std::chrono::duration_cast<std::chrono::milliseconds>(Clock::now() - t0).count() > timeout_ms) {
            st = api_fail(ICM_ETIMEOUT, "server did not drain in time");
            break;
        }
        std::this_thread::sleep_for(std::chrono::milliseconds(1));
    }
    if (st == ICM_OK) {
        s->worker.join();
        delete s;
    } else {
        s->worker.detach();      // still draining: the object stays alive for the worker
    }
    return st;
}

}  // extern "C"
