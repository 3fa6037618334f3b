// Serving form: a request loop that keeps the encrypted database resident, admits query eyes as
// they arrive, batches them (continuous batching: a batch starts when it is full or its oldest
// eye has waited `window_us`, and requests that arrive while batches run join a later one), and
// runs query preparation, the grouped CCMM and the fold per batch (Section 5: computing servers
// batch up to 32 query eyes; Appendix C.5 batch scaling).
//
// Admission by device memory: the caller's workspace is a pool.  Every batch of n eyes reserves,
// for its whole life, the bytes its buffers take at n eyes (prepared query with its residue
// planes, scores, CRT scratch, ciphertext, folded scores), first fit in the pool.  A batch starts
// when a batch slot (compute stream, copy stream, page-locked staging) is free and the pool holds
// the buffers of at least one waiting eye; it takes as many waiting eyes (up to max_eyes) as the
// free memory allows.  With the workspace of icm_server_device_bytes, max_batches full batches fit.
//
// Overlap on the device: each batch runs its preparation, CCMM and folds on its slot's compute
// stream and its copies on its slot's copy stream.  The CCMM of a batch waits for the previous
// batch's CCMM (the persistent product kernel occupies every SM; two at once would only compete),
// so one batch's gather, host-to-device copy and query preparation, and another's folds,
// device-to-host copy and scatter, run while a third (or the same) batch's CCMM runs.
// Every wait is bounded (condition-variable waits with timeouts, event polling).
#include <algorithm>
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

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

// Buffers of one batch of n eyes, carved from its reservation in this order.
struct BatchBytes {
    size_t op = 0, ws = 0, ct = 0, total = 0;
    std::vector<size_t> sc, fo;
};

BatchBytes batch_bytes(const icm_ctx *c, const std::vector<const icm_db *> &dbs, icm_form f, uint32_t n) {
    BatchBytes b;
    icm_query_op_bytes(c, n, f, &b.op);
    icm_match_batch_workspace_bytes(c, dbs.data(), dbs.size(), n, f, &b.ws);
    icm_query_ct_bytes(c, n, &b.ct);
    b.total = a256(b.op) + a256(b.ws) + a256(b.ct);
    for (const icm_db *d : dbs) {
        size_t sc = 0, fo = 0;
        icm_scores_bytes(c, d, n, 0, &sc);
        icm_scores_bytes(c, d, n, 1, &fo);
        b.sc.push_back(sc);
        b.fo.push_back(fo);
        b.total += a256(sc) + a256(fo);
    }
    return b;
}

struct Slot {
    cudaStream_t comp = nullptr, cs = nullptr;           // compute and copy streams
    cudaEvent_t h2d = nullptr, match = nullptr, done = nullptr, d2h = nullptr;
    uint64_t *h_ct = nullptr;                            // pinned staging, max_eyes
    std::vector<uint64_t *> h_fold;                      // pinned staging per chunk, max_eyes
    std::vector<Req *> reqs;
    bool busy = false;
    size_t off = 0, bytes = 0;                           // reservation in the pool
};

}  // namespace

struct icm_server {
    icm_ctx *ctx;
    std::vector<const icm_db *> dbs;
    icm_server_cfg cfg;
    uint32_t G = 0;
    size_t eye_ct_words = 0, eye_out_words = 0;
    char *pool = nullptr;
    size_t pool_bytes = 0, full_batch_bytes = 0;
    std::vector<std::pair<size_t, size_t>> used;         // reservations (offset, bytes), by offset
    std::vector<Slot> slots;
    cudaEvent_t last_match = nullptr;                    // CCMM of the last launched batch
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req *> pending;
    std::unordered_map<uint64_t, Req *> reqs;
    uint64_t next_ticket = 1, n_done = 0, n_batches = 0, eyes_batched = 0;
    size_t cur_bytes = 0, peak_bytes = 0;
    uint32_t inflight = 0, peak_inflight = 0;
    bool stop = false;
    std::thread worker;

    ~icm_server();
    void run();
    bool reserve(size_t bytes, size_t &off);
    void release(size_t off);
    bool any_busy() const {
        for (const Slot &s : slots) if (s.busy) return true;
        return false;
    }
    icm_status launch(Slot &s, std::vector<Req *> &batch);
    void finish(Slot &s, icm_status st);
};

icm_server::~icm_server() {
    for (auto &s : slots) {
        if (s.comp) cudaStreamDestroy(s.comp);
        if (s.cs) cudaStreamDestroy(s.cs);
        if (s.h2d) cudaEventDestroy(s.h2d);
        if (s.match) cudaEventDestroy(s.match);
        if (s.done) cudaEventDestroy(s.done);
        if (s.d2h) cudaEventDestroy(s.d2h);
        if (s.h_ct) cudaFreeHost(s.h_ct);
        for (auto *p : s.h_fold) cudaFreeHost(p);
    }
    for (auto &kv : reqs) delete kv.second;
}

// First fit in the pool (offsets and sizes in 256-byte units of the workspace).
bool icm_server::reserve(size_t bytes, size_t &off) {
    size_t at = 0;
    for (const auto &u : used) {
        if (u.first >= at + bytes) break;
        at = std::max(at, u.first + u.second);
    }
    if (at + bytes > pool_bytes) return false;
    used.emplace_back(at, bytes);
    std::sort(used.begin(), used.end());
    off = at;
    cur_bytes += bytes;
    peak_bytes = std::max(peak_bytes, cur_bytes);
    return true;
}

void icm_server::release(size_t off) {
    for (size_t i = 0; i < used.size(); ++i)
        if (used[i].first == off) {
            cur_bytes -= used[i].second;
            used.erase(used.begin() + (long)i);
            return;
        }
}

icm_status icm_server::launch(Slot &s, std::vector<Req *> &batch) {
    const uint32_t n = (uint32_t)batch.size();
    const uint32_t Lq = ctx->p.n_limbs_q, rho = ctx->p.rho, K = ctx->K;
    const BatchBytes b = batch_bytes(ctx, dbs, cfg.form, n);
    // carve the batch's buffers from its reservation
    char *w = pool + s.off;
    void *d_op = w; w += a256(b.op);
    void *d_ws = b.ws ? w : nullptr; w += a256(b.ws);
    void *d_ct = w; w += a256(b.ct);
    std::vector<void *> d_sc, d_fo;
    for (size_t i = 0; i < dbs.size(); ++i) { d_sc.push_back(w); w += a256(b.sc[i]); }
    for (size_t i = 0; i < dbs.size(); ++i) { d_fo.push_back(w); w += a256(b.fo[i]); }
    // gather the eyes' ciphertexts into the staging layout [Lq][n*rho][K]
    for (uint32_t l = 0; l < Lq; ++l)
        for (uint32_t e = 0; e < n; ++e)
            std::memcpy(s.h_ct + ((size_t)l * n * rho + (size_t)e * rho) * K, batch[e]->host_ct + (size_t)l * rho * K,
                        (size_t)rho * K * 8);
    cudaError_t e = cudaMemcpyAsync(d_ct, s.h_ct, b.ct, cudaMemcpyHostToDevice, s.cs);
    if (e == cudaSuccess) e = cudaEventRecord(s.h2d, s.cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s.comp, s.h2d, 0);
    if (e != cudaSuccess) return api_fail(ICM_ECUDA, cudaGetErrorString(e));
    icm_query *q = nullptr;
    icm_status st = icm_query_prepare(ctx, d_ct, n, cfg.form, d_op, b.op, s.comp, &q);
    // one CCMM at a time on the device: after the previous batch's
    if (st == ICM_OK && last_match && cudaStreamWaitEvent(s.comp, last_match, 0) != cudaSuccess)
        st = api_fail(ICM_ECUDA, "stream wait");
    std::vector<icm_scores *> sc(dbs.size(), nullptr), fo(dbs.size(), nullptr);
    if (st == ICM_OK)
        st = icm_match_batch(ctx, dbs.data(), dbs.size(), q, d_sc.data(), b.sc.data(), d_ws, b.ws, s.comp, sc.data());
    if (st == ICM_OK) {
        if (cudaEventRecord(s.match, s.comp) != cudaSuccess) st = api_fail(ICM_ECUDA, "event record");
        else last_match = s.match;
    }
    for (size_t i = 0; st == ICM_OK && i < dbs.size(); ++i)
        st = icm_fold(ctx, sc[i], d_fo[i], b.fo[i], s.comp, &fo[i]);
    icm_query_destroy(q);
    for (auto *p : sc) icm_scores_destroy(p);
    for (auto *p : fo) icm_scores_destroy(p);
    if (st != ICM_OK) return st;
    e = cudaEventRecord(s.done, s.comp);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s.cs, s.done, 0);
    for (size_t i = 0; e == cudaSuccess && i < dbs.size(); ++i) {
        const size_t bytes = (size_t)ctx->p.n_limbs * n * G * dbs[i]->lay.M * 8;
        e = cudaMemcpyAsync(s.h_fold[i], d_fo[i], bytes, cudaMemcpyDeviceToHost, s.cs);
    }
    if (e == cudaSuccess) e = cudaEventRecord(s.d2h, s.cs);
    if (e != cudaSuccess) return api_fail(ICM_ECUDA, cudaGetErrorString(e));
    return ICM_OK;
}

// Scatter every eye's folded scores to its output, then mark the requests done (or failed) and
// return the batch's memory to the pool.
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
    release(s.off);
    s.busy = false;
    --inflight;
    cv.notify_all();
}

void icm_server::run() {
    cudaSetDevice(ctx->device);
    for (;;) {
        // completions
        for (auto &s : slots) {
            if (!s.busy) continue;
            const cudaError_t q = cudaEventQuery(s.d2h);
            if (q == cudaErrorNotReady) continue;
            finish(s, q == cudaSuccess ? ICM_OK : ICM_ECUDA);
        }
        std::vector<Req *> batch;
        Slot *free_slot = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            const bool busy = any_busy();
            if (stop && pending.empty() && !busy) return;
            for (auto &s : slots) if (!s.busy) { free_slot = &s; break; }
            bool go = false;
            if (free_slot && !pending.empty()) {
                const auto waited = std::chrono::duration_cast<std::chrono::microseconds>(Clock::now() - pending.front()->t_submit).count();
                go = pending.size() >= cfg.max_eyes || waited >= (long long)cfg.window_us || stop;
            }
            uint32_t n = 0;
            if (go) {
                // admission by memory: the most waiting eyes (up to max_eyes) whose buffers fit
                n = (uint32_t)std::min<size_t>(pending.size(), cfg.max_eyes);
                while (n > 0 && !reserve(batch_bytes(ctx, dbs, cfg.form, n).total, free_slot->off)) --n;
            }
            if (n > 0) {
                free_slot->bytes = batch_bytes(ctx, dbs, cfg.form, n).total;
                while (batch.size() < n) {
                    batch.push_back(pending.front());
                    pending.front()->state = 1;
                    pending.pop_front();
                }
                free_slot->busy = true;
                free_slot->reqs = batch;
                ++n_batches;
                eyes_batched += batch.size();
                peak_inflight = std::max(peak_inflight, ++inflight);
            } else {
                // nothing to launch (no slot, no eye, window still open, or no memory until a
                // batch completes): sleep until a request arrives or a poll interval passes
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
    if (!c || !dbs || !cfg || !bytes || n_dbs == 0 || n_dbs > ICM_MAX_CHUNKS || cfg->max_eyes == 0 || cfg->max_eyes > 32 ||
        cfg->max_batches > 4)
        return api_fail(ICM_EINVAL, "bad arguments");
    const std::vector<const icm_db *> v(dbs, dbs + n_dbs);
    *bytes = (size_t)(cfg->max_batches ? cfg->max_batches : 2) * batch_bytes(c, v, cfg->form, cfg->max_eyes).total;
    return ICM_OK;
}

icm_status icm_server_create(icm_ctx *c, const icm_db *const *dbs, size_t n_dbs, const icm_server_cfg *cfg, void *dev_ws,
                             size_t ws_bytes, icm_server **out) {
    size_t need = 0;
    icm_status st = icm_server_device_bytes(c, dbs, n_dbs, cfg, &need);
    if (st != ICM_OK) return st;
    const std::vector<const icm_db *> v(dbs, dbs + n_dbs);
    const size_t full = batch_bytes(c, v, cfg->form, cfg->max_eyes).total;
    if (!out || !dev_ws || ws_bytes < full) return api_fail(ICM_ENOMEM, "server workspace holds less than one full batch");
    if (!c->have_keys) return api_fail(ICM_EINVAL, "icm_keygen has not run");
    icm_server *s = new (std::nothrow) icm_server();
    if (!s) return api_fail(ICM_ENOMEM, "host allocation");
    s->ctx = c;
    s->dbs = v;
    s->cfg = *cfg;
    if (s->cfg.max_pending == 0) s->cfg.max_pending = 4096;
    if (s->cfg.max_batches == 0) s->cfg.max_batches = 2;
    s->G = (c->p.rho + c->p.fold_k - 1) / c->p.fold_k;
    s->eye_ct_words = (size_t)c->p.n_limbs_q * c->p.rho * c->K;
    for (size_t i = 0; i < n_dbs; ++i) s->eye_out_words += (size_t)c->p.n_limbs * s->G * dbs[i]->lay.M;
    s->pool = (char *)dev_ws;
    s->pool_bytes = ws_bytes / 256 * 256;
    s->full_batch_bytes = full;
    size_t ct_bytes = 0;
    icm_query_ct_bytes(c, cfg->max_eyes, &ct_bytes);
    const BatchBytes fb = batch_bytes(c, v, cfg->form, cfg->max_eyes);
    s->slots.resize(s->cfg.max_batches);
    cudaError_t e = cudaSuccess;
    for (auto &sl : s->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.comp, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.h2d, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.match, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.d2h, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_ct, ct_bytes);
        for (size_t i = 0; i < n_dbs; ++i) {
            uint64_t *h = nullptr;
            if (e == cudaSuccess) e = cudaMallocHost((void **)&h, fb.fo[i]);
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

icm_status icm_server_memory(icm_server *s, size_t *pool_bytes, size_t *full_batch_bytes, size_t *peak_bytes,
                             uint32_t *peak_batches) {
    if (!s) return api_fail(ICM_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (pool_bytes) *pool_bytes = s->pool_bytes;
    if (full_batch_bytes) *full_batch_bytes = s->full_batch_bytes;
    if (peak_bytes) *peak_bytes = s->peak_bytes;
    if (peak_batches) *peak_batches = s->peak_inflight;
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
            if (s->pending.empty() && !s->any_busy()) break;
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
