// Batching form: one CCMM over several database chunks (each its own MSRLWE database with its own
// a-part, uneven sizes) for one query batch, the fold of every chunk, and the whole pass captured
// into a CUDA graph that is replayed per batch; plus the autotuner of the product kernel's tile.
//
// For the small-modulus CRT forms every limb, chunk, row tile, modulus and column tile of a
// column round goes into one persistent launch (launch_ppmm_crt_grouped).  The u64 and digit forms
// loop over chunks.
#include <algorithm>
#include <new>
#include <vector>

#include "icm_internal.h"

using namespace icm;

namespace icm {
icm_status api_fail(icm_status s, const char *msg);
}

struct icm_plan {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~icm_plan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
};

namespace {

bool crt_form(icm_form f) { return f == ICM_FORM_I8_CRT || f == ICM_FORM_F16_CRT; }

// Bytes per chunk of scores, and the batch workspace split (match scratch only).
size_t batch_ws_bytes(const icm_ctx *c, const icm_db *const *dbs, size_t n, size_t n_eyes, icm_form form) {
    if (!crt_form(form)) return 0;
    uint64_t Mall = 0;
    for (size_t i = 0; i < n; ++i) Mall += dbs[i]->lay.M;
    return crt_scratch_bytes(c->p.n_limbs, c->i8_crt.n_mod, (uint64_t)n_eyes * c->p.rho, Mall);
}

icm_status enqueue_batch(icm_ctx *c, const icm_db *const *dbs, size_t n, const icm_query *q, void *const *dev_outs,
                         void *dev_ws, int bn, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (crt_form(q->form)) {
        std::vector<const uint64_t *> A(n);
        std::vector<uint64_t *> C(n);
        std::vector<uint64_t> M(n);
        for (size_t i = 0; i < n; ++i) { A[i] = dbs[i]->dev; C[i] = (uint64_t *)dev_outs[i]; M[i] = dbs[i]->lay.M; }
        ChunkTab tab;
        if (!make_chunk_tab(A.data(), C.data(), M.data(), (uint32_t)n, tab)) return api_fail(ICM_EINVAL, "1..16 chunks");
        tab.a_digits = 1;
        const void *planes = (const char *)q->dev + (size_t)c->p.n_limbs * q->n_cols * c->K * 8;
        e = launch_ppmm_crt_grouped(q->form == ICM_FORM_F16_CRT, bn, c->i8_crt, tab, planes, q->n_cols, c->K,
                                    i8_kpad(c->K), dev_ws, st);
    } else {
        for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
            if (q->form == ICM_FORM_U64)
                e = launch_ppmm_u64(c->lt, dbs[i]->dev, (const uint64_t *)q->dev, (uint64_t *)dev_outs[i], dbs[i]->lay.M,
                                    q->n_cols, c->K, true, st);
            else
                e = launch_ppmm_i8(ICM_FORM_I8_DIGITS, c->i8_digits, dbs[i]->dev, true,
                                   (const int8_t *)q->dev + (size_t)c->p.n_limbs * q->n_cols * c->K * 8,
                                   (uint64_t *)dev_outs[i], dbs[i]->lay.M, q->n_cols, c->K, i8_kpad(c->K), st);
        }
    }
    if (e != cudaSuccess) return api_fail(ICM_ECUDA, cudaGetErrorString(e));
    return ICM_OK;
}

}  // namespace

extern "C" {

icm_status icm_match_batch_workspace_bytes(const icm_ctx *c, const icm_db *const *dbs, size_t n_dbs, size_t n_eyes,
                                           icm_form form, size_t *bytes) {
    if (!c || !dbs || !bytes || n_dbs == 0 || n_dbs > ICM_MAX_CHUNKS) return api_fail(ICM_EINVAL, "bad arguments");
    for (size_t i = 0; i < n_dbs; ++i) if (!dbs[i]) return api_fail(ICM_EINVAL, "null database handle");
    *bytes = batch_ws_bytes(c, dbs, n_dbs, n_eyes, form);
    return ICM_OK;
}

icm_status icm_match_batch(icm_ctx *c, const icm_db *const *dbs, size_t n_dbs, const icm_query *q, void *const *dev_outs,
                           const size_t *out_bytes, void *dev_ws, size_t ws_bytes, void *stream, icm_scores **outs) {
    if (!c || !dbs || !q || !dev_outs || !out_bytes || !outs || n_dbs == 0 || n_dbs > ICM_MAX_CHUNKS)
        return api_fail(ICM_EINVAL, "bad arguments");
    for (size_t i = 0; i < n_dbs; ++i) {
        if (!dbs[i] || dbs[i]->ctx != c || !dev_outs[i]) return api_fail(ICM_EINVAL, "bad chunk handle or output");
        const size_t need = (size_t)c->p.n_limbs * q->n_cols * dbs[i]->lay.M * 8;
        if (out_bytes[i] < need) return api_fail(ICM_ENOMEM, "scores buffer too small");
    }
    if (q->ctx != c) return api_fail(ICM_EINVAL, "query from another context");
    const size_t wneed = batch_ws_bytes(c, dbs, n_dbs, q->n_eyes, q->form);
    if (wneed && (!dev_ws || ws_bytes < wneed)) return api_fail(ICM_ENOMEM, "batch workspace too small");
    std::vector<icm_scores *> made(n_dbs, nullptr);
    for (size_t i = 0; i < n_dbs; ++i) {
        made[i] = new (std::nothrow) icm_scores();
        if (!made[i]) { for (auto *p : made) delete p; return api_fail(ICM_ENOMEM, "host allocation"); }
    }
    icm_status s = enqueue_batch(c, dbs, n_dbs, q, dev_outs, dev_ws, c->crt_bn, (cudaStream_t)stream);
    if (s != ICM_OK) { for (auto *p : made) delete p; return s; }
    for (size_t i = 0; i < n_dbs; ++i) {
        icm_scores *sc = made[i];
        sc->ctx = c; sc->lay = dbs[i]->lay; sc->n_eyes = q->n_eyes; sc->n_cols = q->n_cols; sc->folded = 0;
        sc->dev = (uint64_t *)dev_outs[i]; sc->bytes = out_bytes[i];
        outs[i] = sc;
    }
    return ICM_OK;
}

icm_status icm_plan_create(icm_ctx *c, const icm_db *const *dbs, size_t n_dbs, size_t n_eyes, icm_form form,
                           const void *dev_ct, void *dev_op, size_t op_bytes, void *const *dev_scores,
                           const size_t *scores_bytes, void *const *dev_folded, const size_t *folded_bytes, void *dev_ws,
                           size_t ws_bytes, void *stream, icm_plan **out) {
    if (!c || !dbs || !dev_ct || !dev_op || !dev_scores || !dev_folded || !out || n_dbs == 0 || n_dbs > ICM_MAX_CHUNKS)
        return api_fail(ICM_EINVAL, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    if (!st) return api_fail(ICM_EINVAL, "graph capture needs a non-default stream");
    icm_plan *plan = new (std::nothrow) icm_plan();
    if (!plan) return api_fail(ICM_ENOMEM, "host allocation");
    // everything below is host-side validation plus enqueues, recorded by stream capture
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { delete plan; return api_fail(ICM_ECUDA, cudaGetErrorString(e)); }
    icm_query *q = nullptr;
    std::vector<icm_scores *> sc(n_dbs, nullptr), fo(n_dbs, nullptr);
    icm_status s = icm_query_prepare(c, dev_ct, n_eyes, form, dev_op, op_bytes, stream, &q);
    if (s == ICM_OK) s = icm_match_batch(c, dbs, n_dbs, q, dev_scores, scores_bytes, dev_ws, ws_bytes, stream, sc.data());
    for (size_t i = 0; s == ICM_OK && i < n_dbs; ++i) s = icm_fold(c, sc[i], dev_folded[i], folded_bytes[i], stream, &fo[i]);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(st, &g);
    icm_query_destroy(q);
    for (auto *p : sc) icm_scores_destroy(p);
    for (auto *p : fo) icm_scores_destroy(p);
    if (s != ICM_OK) { if (g) cudaGraphDestroy(g); delete plan; return s; }
    if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); delete plan; return api_fail(ICM_ECUDA, cudaGetErrorString(e)); }
    plan->graph = g;
    e = cudaGraphInstantiate(&plan->exec, g, 0);
    if (e != cudaSuccess) { delete plan; return api_fail(ICM_ECUDA, cudaGetErrorString(e)); }
    *out = plan;
    return ICM_OK;
}

icm_status icm_plan_launch(icm_plan *plan, void *stream) {
    if (!plan || !plan->exec) return api_fail(ICM_EINVAL, "null plan");
    cudaError_t e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return api_fail(ICM_ECUDA, cudaGetErrorString(e));
    return ICM_OK;
}

void icm_plan_destroy(icm_plan *plan) { delete plan; }

icm_status icm_autotune(icm_ctx *c, const icm_db *const *dbs, size_t n_dbs, const icm_query *q, void *const *dev_outs,
                        const size_t *out_bytes, void *dev_ws, size_t ws_bytes, void *stream, int *best_tile_n,
                        float *ms_per_choice, size_t n_choices) {
    if (!c || !q || !best_tile_n) return api_fail(ICM_EINVAL, "bad arguments");
    if (!crt_form(q->form)) { *best_tile_n = 0; return ICM_OK; }      // single kernel variant
    // the tcgen05 variants where they apply (fp16 form, even K), else the two mma.sync tiles;
    // ms_per_choice keeps the fixed order 128, 256, 1, 2, 3 (0 for variants not timed)
    const int choices[5] = {128, 256, 1, 2, 3};
    const bool tc = q->form == ICM_FORM_F16_CRT && crt_tc_supported(c->K);
    float best_ms = 1e30f;
    int best = c->crt_bn;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    icm_status s = ICM_OK;
    for (int i = 0; i < 5 && s == ICM_OK; ++i) {
        if (ms_per_choice && (size_t)i < n_choices) ms_per_choice[i] = 0.0f;
        if (tc != crt_tc_variant(choices[i])) continue;
        c->crt_bn = choices[i];
        std::vector<icm_scores *> outs(n_dbs, nullptr);
        cudaEventRecord(a, st);
        s = icm_match_batch(c, dbs, n_dbs, q, dev_outs, out_bytes, dev_ws, ws_bytes, stream, outs.data());
        cudaEventRecord(b, st);
        for (auto *p : outs) icm_scores_destroy(p);
        if (s != ICM_OK) break;
        cudaError_t e = cudaEventSynchronize(b);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e != cudaSuccess) { s = api_fail(ICM_ECUDA, cudaGetErrorString(e)); break; }
        if (ms_per_choice && (size_t)i < n_choices) ms_per_choice[i] = ms;
        if (ms < best_ms) { best_ms = ms; best = choices[i]; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    c->crt_bn = best;
    *best_tile_n = best;
    if (s == ICM_OK && device_status(true) != 0) return api_fail(ICM_ETIMEOUT, "a kernel gave up a bounded wait");
    return s;
}

icm_status icm_ctx_set_device_wait(icm_ctx *c, uint64_t wait_ns, int inject_stall) {
    if (!c) return api_fail(ICM_EINVAL, "null context");
    c->i8_crt.tc_wait_ns = wait_ns;
    c->i8_crt.tc_inject_stall = inject_stall ? 1u : 0u;
    return ICM_OK;
}

icm_status icm_ctx_set_variant(icm_ctx *c, int variant) {
    if (!c || (variant != 0 && !crt_tc_variant(variant) && variant != 128 && variant != 256))
        return api_fail(ICM_EINVAL, "variant must be 0, 1..3, 128 or 256");
    c->crt_bn = variant == 0 ? 2 : variant;
    return ICM_OK;
}

icm_status icm_device_status(int clear) {
    const uint32_t v = device_status(clear != 0);
    if (v == 0xFFFFFFFFu) return api_fail(ICM_ECUDA, "status word unreadable");
    return v ? api_fail(ICM_ETIMEOUT, "a kernel gave up a bounded wait") : ICM_OK;
}

}  // extern "C"
