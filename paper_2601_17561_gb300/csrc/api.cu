// Host side of the libicm C ABI (include/icm.h): parameter checks, prime selection, noise and
// decoding bounds, key generation, buffer sizing and the launch sequence of every call.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>

#include "icm_internal.h"

namespace icm {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }

using u128 = unsigned __int128;

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)((u128)a * b % q); }
static uint64_t powmod(uint64_t b, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    b %= q;
    while (e) { if (e & 1) r = mulmod(r, b, q); b = mulmod(b, b, q); e >>= 1; }
    return r;
}
uint64_t shoup_of(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }

// Deterministic Miller-Rabin for 64-bit integers (the first twelve primes as bases).
static bool is_prime64(uint64_t n) {
    static const uint64_t bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (uint64_t p : bases) if (n % p == 0) return n == p;
    uint64_t d = n - 1; int s = 0;
    while ((d & 1) == 0) { d >>= 1; ++s; }
    for (uint64_t a : bases) {
        uint64_t x = powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < s; ++i) { x = mulmod(x, x, n); if (x == n - 1) { comp = false; break; } }
        if (comp) return false;
    }
    return true;
}

// The `count` largest primes below 2^bits congruent to 1 modulo 2^17, decreasing.
static std::vector<uint64_t> pick_primes(uint32_t bits, uint32_t count) {
    const uint64_t step = 1ull << 17;
    std::vector<uint64_t> out;
    for (uint64_t c = ((1ull << bits) - 2) / step; c > 0 && out.size() < count; --c) {
        const uint64_t cand = c * step + 1;
        if (is_prime64(cand)) out.push_back(cand);
    }
    return out;
}

LimbTable make_limb_table(const std::vector<uint64_t> &q) {
    LimbTable t{};
    t.n = (uint32_t)q.size();
    for (size_t l = 0; l < q.size(); ++l) {
        t.q[l] = q[l];
        t.r64[l] = (uint64_t)(((u128)1 << 64) / q[l]);            // floor(2^64 / q), q >= 3
        t.pw64[l] = powmod(2, 64, q[l]);
        t.pw64s[l] = shoup_of(t.pw64[l], q[l]);
        t.pw128[l] = powmod(2, 128, q[l]);
        t.pw128s[l] = shoup_of(t.pw128[l], q[l]);
    }
    return t;
}

DbLayout make_layout(uint64_t n_real, uint32_t N, uint32_t rho) {
    DbLayout L{};
    L.N = N; L.n_real = n_real; L.n_tpl = n_real;
    L.n_full = (uint32_t)(n_real / N);
    L.rem = (uint32_t)(n_real % N);
    L.tail_lo = N;
    uint64_t M = N + (uint64_t)L.n_full * N;
    if (L.rem) {
        const uint32_t lo = N > rho - 1 ? N - (rho - 1) : 0;
        L.tail_lo = L.rem > lo ? L.rem : lo;
        M += L.rem + (N - L.tail_lo);
    }
    L.M = M;
    return L;
}

// log2(2^a + 2^b)
static long double lse2(long double a, long double b) {
    const long double m = a > b ? a : b;
    return m + log2l(exp2l(a - m) + exp2l(b - m));
}

static icm_status fail(icm_status s, const std::string &msg) { set_error(msg); return s; }
icm_status api_fail(icm_status s, const char *msg) { set_error(msg); return s; }

#define CUDA_TRY(expr)                                                                 \
    do {                                                                               \
        cudaError_t _e = (expr);                                                       \
        if (_e != cudaSuccess) return fail(ICM_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

}  // namespace icm

using namespace icm;

icm_ctx::~icm_ctx() {
    if (d_sdb_pos) cudaFree(d_sdb_pos);
    if (d_sdb_sgn) cudaFree(d_sdb_sgn);
    if (d_sq_pos) cudaFree(d_sq_pos);
    if (d_sq_sgn) cudaFree(d_sq_sgn);
    if (slot_tab) icm::free_slot_tables(slot_tab);
}

extern "C" {

const char *icm_status_str(icm_status s) {
    switch (s) {
        case ICM_OK: return "ok";
        case ICM_EINVAL: return "invalid argument";
        case ICM_ENOMEM: return "out of memory or buffer too small";
        case ICM_ECUDA: return "CUDA error";
        case ICM_ETIMEOUT: return "timed out";
        case ICM_EBOUND: return "bound violated";
        case ICM_EUNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *icm_last_error(void) { return g_err.c_str(); }

icm_status icm_ctx_create(const icm_params *p, icm_ctx **out) {
    if (!p || !out) return fail(ICM_EINVAL, "null argument");
    const icm_params P = *p;
    if (P.log_n_db < 5 || P.log_n_db > 16 || P.log_n_q < 5 || P.log_n_q > 16)
        return fail(ICM_EINVAL, "ring degrees must be 2^5 .. 2^16");
    if (P.n_limbs < 2 || P.n_limbs > ICM_MAX_LIMBS) return fail(ICM_EINVAL, "n_limbs must be 2..8");
    if (P.n_limbs_q < 1 || P.n_limbs_q > 2 || P.n_limbs_q >= P.n_limbs)
        return fail(ICM_EUNSUPPORTED, "n_limbs_q must be 1 or 2 and below n_limbs");
    if (P.prime_bits < 30 || P.prime_bits > 60) return fail(ICM_EINVAL, "prime_bits must be 30..60");
    if (P.code_bits != 12800) return fail(ICM_EUNSUPPORTED, "code_bits must be 12800 (16 x 200 x 4 layout)");
    const uint32_t Nq = 1u << P.log_n_q, Ndb = 1u << P.log_n_db;
    if (P.d2 < P.code_bits || P.d2 % Nq) return fail(ICM_EINVAL, "d2 must cover code_bits and be a multiple of N_q");
    if (P.rho == 0 || P.rho % 2 == 0 || P.rho > 199 || P.rho > Ndb) return fail(ICM_EINVAL, "rho must be odd, <= 199 and <= N_db");
    uint32_t lk = 0;
    while ((1u << lk) < P.fold_k) ++lk;
    if (P.fold_k == 0 || P.fold_k > P.rho || P.prime_bits + lk > 64)
        return fail(ICM_EINVAL, "fold_k must be in 1..rho and fold_k * 2^prime_bits <= 2^64");
    if (P.hamming_weight == 0 || P.hamming_weight > Nq || P.hamming_weight > Ndb) return fail(ICM_EINVAL, "bad hamming weight");
    if (P.noise_eta == 0 || P.noise_eta > 32) return fail(ICM_EINVAL, "noise_eta must be 1..32");
    if (P.log2_delta == 0 || P.log2_delta > 120) return fail(ICM_EINVAL, "log2_delta must be 1..120");
    const uint64_t K = (uint64_t)P.d2 + Nq;
    if (K >= (1ull << 32)) return fail(ICM_EUNSUPPORTED, "K too large");

    std::vector<uint64_t> q = pick_primes(P.prime_bits, P.n_limbs);
    if (q.size() != P.n_limbs) return fail(ICM_EINVAL, "not enough primes");

    // Bounds (worst case).  Decrypted product D = Q' Delta M_db M_q + Q' M_db E_q + E1 B_q + E2 A_q:
    //  (a) no wrap modulo Q_db:  Q' Delta cb + Q' cb eta + eta (d2 + N_q) Q / 2 < Q Q' / 2
    //  (b) exact rounding:       Q' cb eta + eta (d2 + N_q) Q / 2 < Q' Delta / 2
    //  (c) fixed-point CRT of the decryption check: L 2^bits 2^-128 Q / Delta < 1/8
    long double lQ = 0, lQp = 0;
    for (uint32_t l = 0; l < P.n_limbs; ++l) (l < P.n_limbs_q ? lQ : lQp) += log2l((long double)q[l]);
    const long double lcb = log2l((long double)P.code_bits), leta = log2l((long double)P.noise_eta);
    const long double lnoise_q = leta + log2l((long double)K) + lQ - 1;     // eta (d2+Nq) Q / 2
    const long double lerr = lse2(lQp + lcb + leta, lnoise_q);
    const long double lmsg = lQp + P.log2_delta + lcb;
    if (lse2(lmsg, lerr) > lQ + lQp - 1 - 1) return fail(ICM_EBOUND, "message plus noise may wrap modulo Q_db (raise Q or lower Delta)");
    if (lerr > lQp + P.log2_delta - 1 - 1) return fail(ICM_EBOUND, "noise may exceed Q' Delta / 2 (raise Delta)");
    if (log2l((long double)P.n_limbs) + P.prime_bits - 128 + lQ - P.log2_delta > -3)
        return fail(ICM_EBOUND, "fixed-point CRT of the decryption check is too coarse for Q / Delta");

    icm_ctx *c = new (std::nothrow) icm_ctx();
    if (!c) return fail(ICM_ENOMEM, "host allocation");
    c->p = P;
    c->N_db = Ndb; c->N_q = Nq; c->K = (uint32_t)K; c->n_qblk = P.d2 / Nq;
    c->q = q;
    c->lt = make_limb_table(q);
    c->qp_mod.resize(P.n_limbs); c->qp_mods.resize(P.n_limbs);
    c->delta_mod.resize(P.n_limbs); c->delta_mods.resize(P.n_limbs);
    for (uint32_t l = 0; l < P.n_limbs; ++l) {
        uint64_t v = 1 % q[l];
        for (uint32_t j = P.n_limbs_q; j < P.n_limbs; ++j) v = mulmod(v, q[j] % q[l], q[l]);
        c->qp_mod[l] = v; c->qp_mods[l] = shoup_of(v, q[l]);
        c->delta_mod[l] = powmod(2, P.log2_delta, q[l]); c->delta_mods[l] = shoup_of(c->delta_mod[l], q[l]);
        // CRT decoding constants
        uint64_t hat = 1 % q[l];
        for (uint32_t j = 0; j < P.n_limbs; ++j) if (j != l) hat = mulmod(hat, q[j] % q[l], q[l]);
        c->crt.inv[l] = powmod(hat, q[l] - 2, q[l]);
        c->crt.invs[l] = shoup_of(c->crt.inv[l], q[l]);
        const u128 R = (~(u128)0) / q[l];            // floor((2^128 - 1) / q) = floor(2^128 / q), q odd
        c->crt.rhi[l] = (uint64_t)(R >> 64);
        c->crt.rlo[l] = (uint64_t)R;
    }
    {
        const char *why = nullptr;
        make_i8_consts(ICM_FORM_I8_DIGITS, q.data(), q.size(), K, c->i8_digits, &why);
        c->i8_crt_ok = make_i8_consts(ICM_FORM_I8_CRT, q.data(), q.size(), K, c->i8_crt, &why);
    }
    long double qod = 1;
    for (uint32_t l = 0; l < P.n_limbs_q; ++l) qod *= (long double)q[l];
    c->crt.q_over_delta = (double)(qod / exp2l((long double)P.log2_delta));
    // decoding at the rescaled level (modulus Q, L_q limbs; same Q / Delta) and the rescaling
    c->crt_q = c->crt;
    c->rs = icm::RescaleConsts{};
    c->rs.L = P.n_limbs; c->rs.Lq = P.n_limbs_q;
    for (uint32_t l = 0; l < P.n_limbs; ++l) c->rs.q[l] = q[l];
    for (uint32_t l = 0; l < P.n_limbs_q; ++l) {
        uint64_t hat = 1 % q[l];
        for (uint32_t j = 0; j < P.n_limbs_q; ++j) if (j != l) hat = mulmod(hat, q[j] % q[l], q[l]);
        c->crt_q.inv[l] = powmod(hat, q[l] - 2, q[l]);
        c->crt_q.invs[l] = shoup_of(c->crt_q.inv[l], q[l]);
    }
    for (uint32_t i = P.n_limbs_q; i < P.n_limbs; ++i) {
        uint64_t hat = 1 % q[i];
        for (uint32_t k = P.n_limbs_q; k < P.n_limbs; ++k) if (k != i) hat = mulmod(hat, q[k] % q[i], q[i]);
        c->rs.yinv[i] = powmod(hat, q[i] - 2, q[i]);
        c->rs.yinvs[i] = shoup_of(c->rs.yinv[i], q[i]);
        c->rs.rhi[i] = c->crt.rhi[i]; c->rs.rlo[i] = c->crt.rlo[i];
    }
    for (uint32_t j = 0; j < P.n_limbs_q; ++j) {
        uint64_t qp = 1 % q[j];
        for (uint32_t i = P.n_limbs_q; i < P.n_limbs; ++i) {
            uint64_t hat = 1 % q[j];
            for (uint32_t k = P.n_limbs_q; k < P.n_limbs; ++k) if (k != i) hat = mulmod(hat, q[k] % q[j], q[j]);
            c->rs.w[j][i] = hat;
            c->rs.ws[j][i] = shoup_of(hat, q[j]);
            qp = mulmod(qp, q[i] % q[j], q[j]);
        }
        c->rs.qp[j] = qp; c->rs.qps[j] = shoup_of(qp, q[j]);
        c->rs.qpinv[j] = powmod(qp, q[j] - 2, q[j]); c->rs.qpinvs[j] = shoup_of(c->rs.qpinv[j], q[j]);
    }
    *out = c;
    return ICM_OK;
}

void icm_ctx_destroy(icm_ctx *ctx) { delete ctx; }

icm_status icm_ctx_primes(const icm_ctx *ctx, uint64_t *primes, size_t n) {
    if (!ctx || !primes || n < ctx->q.size()) return fail(ICM_EINVAL, "bad arguments");
    for (size_t l = 0; l < ctx->q.size(); ++l) primes[l] = ctx->q[l];
    return ICM_OK;
}

icm_status icm_ctx_crt_moduli(const icm_ctx *ctx, int32_t *moduli, size_t cap, size_t *n_moduli) {
    if (!ctx || !n_moduli || (cap && !moduli)) return fail(ICM_EINVAL, "bad arguments");
    if (!ctx->i8_crt_ok) return fail(ICM_EBOUND, "CRT forms unavailable for these primes / K");
    *n_moduli = ctx->i8_crt.n_mod;
    for (size_t i = 0; i < cap && i < ctx->i8_crt.n_mod; ++i) moduli[i] = ctx->i8_crt.mod[i];
    return ICM_OK;
}

}  // extern "C"

namespace icm {
// Sparse ternary secret with exactly h non-zeros: positions floor(w n / 2^64) drawn in stream
// order (skipping positions already taken), sign -1 when the word's lowest bit is set.
static SecretSupport sample_secret(uint64_t key, uint32_t n, uint32_t h) {
    std::vector<int8_t> s(n, 0);
    uint32_t cnt = 0;
    for (uint64_t j = 0; cnt < h; ++j) {
        const uint64_t w = sm64(key, j);
        const uint64_t pos = (uint64_t)(((u128)w * n) >> 64);
        if (!s[pos]) { s[pos] = (w & 1) ? -1 : 1; ++cnt; }
    }
    SecretSupport sp;
    for (uint32_t i = 0; i < n; ++i) if (s[i]) { sp.pos.push_back((int32_t)i); sp.sgn.push_back(s[i]); }
    return sp;
}
}  // namespace icm

extern "C" {

icm_status icm_keygen(icm_ctx *c) {
    if (!c) return fail(ICM_EINVAL, "null context");
    CUDA_TRY(cudaGetDevice(&c->device));
    const uint32_t h = c->p.hamming_weight;
    // database secrets for up to 2^17 / N_db blocks plus one (a chunk of up to 2^17 + N_db templates)
    const uint32_t max_blocks = (1u << 17) / c->N_db + 2;
    std::vector<int32_t> dpos((size_t)max_blocks * h), qpos((size_t)c->n_qblk * h);
    std::vector<int8_t> dsg((size_t)max_blocks * h), qsg((size_t)c->n_qblk * h);
    for (uint32_t t = 0; t < max_blocks; ++t) {
        SecretSupport s = sample_secret(stream_key(c->p.seed, ICM_KIND_SK_DB, t, 0), c->N_db, h);
        std::copy(s.pos.begin(), s.pos.end(), dpos.begin() + (size_t)t * h);
        std::copy(s.sgn.begin(), s.sgn.end(), dsg.begin() + (size_t)t * h);
    }
    for (uint32_t t = 0; t < c->n_qblk; ++t) {
        SecretSupport s = sample_secret(stream_key(c->p.seed, ICM_KIND_SK_Q, t, 0), c->N_q, h);
        std::copy(s.pos.begin(), s.pos.end(), qpos.begin() + (size_t)t * h);
        std::copy(s.sgn.begin(), s.sgn.end(), qsg.begin() + (size_t)t * h);
    }
    int32_t *a = nullptr, *b = nullptr; int8_t *x = nullptr, *y = nullptr;
    cudaError_t e = cudaMalloc(&a, dpos.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&x, dsg.size());
    if (e == cudaSuccess) e = cudaMalloc(&b, qpos.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&y, qsg.size());
    if (e == cudaSuccess) e = cudaMemcpy(a, dpos.data(), dpos.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(x, dsg.data(), dsg.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b, qpos.data(), qpos.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(y, qsg.data(), qsg.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(a); cudaFree(b); cudaFree(x); cudaFree(y);
        return fail(ICM_ECUDA, std::string("keygen upload: ") + cudaGetErrorString(e));
    }
    if (c->d_sdb_pos) { cudaFree(c->d_sdb_pos); cudaFree(c->d_sdb_sgn); cudaFree(c->d_sq_pos); cudaFree(c->d_sq_sgn); }
    c->d_sdb_pos = a; c->d_sdb_sgn = x; c->d_sq_pos = b; c->d_sq_sgn = y;
    c->max_db_blocks = max_blocks;
    c->have_keys = true;
    // shared-memory opt-ins of the product kernels are set once here, outside any stream capture
    e = crt_set_attributes();
    if (e != cudaSuccess) return fail(ICM_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
    return ICM_OK;
}

icm_status icm_db_bytes(const icm_ctx *c, size_t n_db, size_t *bytes, size_t *m_rows) {
    if (!c || !bytes) return fail(ICM_EINVAL, "null argument");
    const DbLayout L = make_layout(n_db, c->N_db, c->p.rho);
    *bytes = (size_t)c->p.n_limbs * L.M * c->K * 8;
    if (m_rows) *m_rows = L.M;
    return ICM_OK;
}

icm_status icm_db_encrypt(icm_ctx *c, const uint8_t *codes, const uint8_t *masks, size_t n_db, uint64_t chunk_id,
                          void *dev_buf, size_t bytes, void *stream, icm_db **out) {
    if (!c || !out || !dev_buf || (n_db && (!codes || !masks))) return fail(ICM_EINVAL, "null argument");
    if (!c->have_keys) return fail(ICM_EINVAL, "icm_keygen has not run");
    const DbLayout L = make_layout(n_db, c->N_db, c->p.rho);
    if (L.n_blocks() > c->max_db_blocks) return fail(ICM_EUNSUPPORTED, "chunk larger than 2^17 templates");
    const size_t need = (size_t)c->p.n_limbs * L.M * c->K * 8;
    if (bytes < need) return fail(ICM_ENOMEM, "database buffer too small");
    if ((uintptr_t)dev_buf % 16) return fail(ICM_EINVAL, "database buffer must be 16-byte aligned");
    if (L.M > 0xFFFFFFFFull) return fail(ICM_EUNSUPPORTED, "chunk too large");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t tb = c->p.code_bits / 8;
    uint8_t *d_t = nullptr;
    if (n_db) {
        CUDA_TRY(cudaMallocAsync((void **)&d_t, 2 * n_db * tb, st));
        cudaError_t e = cudaMemcpyAsync(d_t, codes, n_db * tb, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_t + n_db * tb, masks, n_db * tb, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { cudaFreeAsync(d_t, st); return fail(ICM_ECUDA, cudaGetErrorString(e)); }
    }
    icm_db *db = new (std::nothrow) icm_db();
    if (!db) { if (d_t) cudaFreeAsync(d_t, st); return fail(ICM_ENOMEM, "host allocation"); }
    uint64_t *d = (uint64_t *)dev_buf;
    cudaError_t e = launch_db_messages(c, to_dev(L), d_t, d_t ? d_t + n_db * tb : nullptr, d, st);
    if (e == cudaSuccess) e = launch_db_apart_and_b(c, to_dev(L), chunk_id, d, st);
    if (d_t) cudaFreeAsync(d_t, st);
    if (e != cudaSuccess) { delete db; return fail(ICM_ECUDA, std::string("db encrypt: ") + cudaGetErrorString(e)); }
    db->ctx = c; db->lay = L; db->chunk_id = chunk_id; db->dev = d; db->bytes = bytes;
    *out = db;
    return ICM_OK;
}

void icm_db_destroy(icm_db *db) { delete db; }

icm_status icm_query_ct_bytes(const icm_ctx *c, size_t n_eyes, size_t *bytes) {
    if (!c || !bytes) return fail(ICM_EINVAL, "null argument");
    *bytes = (size_t)c->p.n_limbs_q * n_eyes * c->p.rho * c->K * 8;
    return ICM_OK;
}

icm_status icm_query_encrypt(icm_ctx *c, const uint8_t *codes, const uint8_t *masks, const uint64_t *eye_ids,
                             size_t n_eyes, void *dev_ct, size_t bytes, void *stream) {
    if (!c || !dev_ct || (n_eyes && (!codes || !masks || !eye_ids))) return fail(ICM_EINVAL, "null argument");
    if (!c->have_keys) return fail(ICM_EINVAL, "icm_keygen has not run");
    size_t need; icm_query_ct_bytes(c, n_eyes, &need);
    if (bytes < need) return fail(ICM_ENOMEM, "query ciphertext buffer too small");
    if (n_eyes * c->p.rho > 0x7FFFFFFFull) return fail(ICM_EINVAL, "too many eyes");
    if (!n_eyes) return ICM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t tb = c->p.code_bits / 8;
    uint8_t *d_t = nullptr;
    CUDA_TRY(cudaMallocAsync((void **)&d_t, 2 * n_eyes * tb + n_eyes * 8 + 16, st));
    uint64_t *d_ids = (uint64_t *)(d_t + ((2 * n_eyes * tb + 15) & ~(size_t)15));
    cudaError_t e = cudaMemcpyAsync(d_t, codes, n_eyes * tb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_t + n_eyes * tb, masks, n_eyes * tb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_ids, eye_ids, n_eyes * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_query_encrypt(c, d_t, d_t + n_eyes * tb, d_ids, (uint32_t)n_eyes, (uint64_t *)dev_ct, st);
    cudaFreeAsync(d_t, st);
    if (e != cudaSuccess) return fail(ICM_ECUDA, std::string("query encrypt: ") + cudaGetErrorString(e));
    return ICM_OK;
}

icm_status icm_query_op_bytes(const icm_ctx *c, size_t n_eyes, icm_form form, size_t *bytes) {
    if (!c || !bytes) return fail(ICM_EINVAL, "null argument");
    const size_t n = (size_t)c->p.n_limbs * n_eyes * c->p.rho * c->K;
    switch (form) {
        case ICM_FORM_U64: *bytes = n * 8; return ICM_OK;
        case ICM_FORM_I8_DIGITS:
        case ICM_FORM_I8_CRT:
        case ICM_FORM_F16_CRT: {
            if (form != ICM_FORM_I8_DIGITS && !c->i8_crt_ok) return fail(ICM_EBOUND, "CRT form unavailable for these primes / K");
            const uint32_t P = form == ICM_FORM_I8_DIGITS ? 8 : c->i8_crt.n_mod;
            *bytes = n * 8 + crt_plane_bytes(form == ICM_FORM_F16_CRT, c->p.n_limbs, P, n_eyes * c->p.rho, i8_kpad(c->K));
            return ICM_OK;
        }
        default: return fail(ICM_EUNSUPPORTED, "form not built");
    }
}

icm_status icm_query_prepare(icm_ctx *c, const void *dev_ct, size_t n_eyes, icm_form form, void *dev_op,
                             size_t bytes, void *stream, icm_query **out) {
    if (!c || !dev_ct || !dev_op || !out) return fail(ICM_EINVAL, "null argument");
    size_t need;
    icm_status s = icm_query_op_bytes(c, n_eyes, form, &need);
    if (s != ICM_OK) return s;
    if (bytes < need) return fail(ICM_ENOMEM, "query operand buffer too small");
    icm_query *q = new (std::nothrow) icm_query();
    if (!q) return fail(ICM_ENOMEM, "host allocation");
    const uint32_t n_cols = (uint32_t)(n_eyes * c->p.rho);
    cudaError_t e = launch_query_extend(c, (const uint64_t *)dev_ct, n_cols, (uint64_t *)dev_op, (cudaStream_t)stream);
    if (e == cudaSuccess && form != ICM_FORM_U64) {
        const I8Consts &k = form == ICM_FORM_I8_DIGITS ? c->i8_digits : c->i8_crt;
        int8_t *planes = (int8_t *)dev_op + (size_t)c->p.n_limbs * n_cols * c->K * 8;
        if (form == ICM_FORM_I8_DIGITS)
            e = launch_planes(form, k, (const uint64_t *)dev_op, planes, n_cols, c->K, i8_kpad(c->K), (cudaStream_t)stream);
        else
            e = launch_crt_planes(form == ICM_FORM_F16_CRT, k, (const uint64_t *)dev_op, planes, n_cols, c->K, i8_kpad(c->K),
                                  (cudaStream_t)stream);
    }
    if (e != cudaSuccess) { delete q; return fail(ICM_ECUDA, std::string("query prepare: ") + cudaGetErrorString(e)); }
    q->ctx = c; q->form = form; q->n_eyes = (uint32_t)n_eyes; q->n_cols = n_cols; q->dev = dev_op; q->bytes = bytes;
    *out = q;
    return ICM_OK;
}

void icm_query_destroy(icm_query *q) { delete q; }

icm_status icm_scores_bytes(const icm_ctx *c, const icm_db *db, size_t n_eyes, int folded, size_t *bytes) {
    if (!c || !db || !bytes) return fail(ICM_EINVAL, "null argument");
    const size_t cols = folded ? n_eyes * ((c->p.rho + c->p.fold_k - 1) / c->p.fold_k) : n_eyes * c->p.rho;
    *bytes = (size_t)c->p.n_limbs * cols * db->lay.M * 8;
    return ICM_OK;
}

icm_status icm_match_workspace_bytes(const icm_ctx *c, const icm_db *db, size_t n_eyes, icm_form form, size_t *bytes) {
    if (!c || !db || !bytes) return fail(ICM_EINVAL, "null argument");
    const bool crt = form == ICM_FORM_F16_CRT || form == ICM_FORM_I8_CRT;
    *bytes = crt ? crt_scratch_bytes(c->p.n_limbs, c->i8_crt.n_mod, (uint64_t)n_eyes * c->p.rho, db->lay.M) : 0;
    return ICM_OK;
}

icm_status icm_match_launches(const icm_ctx *c, const icm_db *db, size_t n_eyes, icm_form form, size_t *n) {
    if (!c || !db || !n) return fail(ICM_EINVAL, "null argument");
    const uint64_t N = (uint64_t)n_eyes * c->p.rho, M = db->lay.M;
    *n = 0;
    if (N == 0 || M == 0) return ICM_OK;
    if (form == ICM_FORM_U64 || form == ICM_FORM_I8_DIGITS) { *n = 1; return ICM_OK; }
    if (form != ICM_FORM_I8_CRT && form != ICM_FORM_F16_CRT) return fail(ICM_EINVAL, "not a match form");
    const uint32_t L = c->p.n_limbs, G = crt_limb_group(L, c->i8_crt.n_mod, N, M);
    const bool tc = form == ICM_FORM_F16_CRT && crt_tc_variant(c->crt_bn) && crt_tc_supported(c->K);
    const uint64_t cols = tc ? 1024 : 512;
    *n = (size_t)((L + G - 1) / G) * ((N + cols - 1) / cols) * 2;
    return ICM_OK;
}

icm_status icm_match(icm_ctx *c, const icm_db *db, const icm_query *q, void *dev_out, size_t bytes, void *dev_ws,
                     size_t ws_bytes, void *stream, icm_scores **out) {
    if (!c || !db || !q || !dev_out || !out) return fail(ICM_EINVAL, "null argument");
    if (db->ctx != c || q->ctx != c) return fail(ICM_EINVAL, "handles from another context");
    size_t need; icm_scores_bytes(c, db, q->n_eyes, 0, &need);
    if (bytes < need) return fail(ICM_ENOMEM, "scores buffer too small");
    size_t wneed; icm_match_workspace_bytes(c, db, q->n_eyes, q->form, &wneed);
    if (wneed && (!dev_ws || ws_bytes < wneed)) return fail(ICM_ENOMEM, "match workspace too small");
    icm_scores *sc = new (std::nothrow) icm_scores();
    if (!sc) return fail(ICM_ENOMEM, "host allocation");
    cudaError_t e = cudaSuccess;
    switch (q->form) {
        case ICM_FORM_U64:
            e = launch_ppmm_u64(c->lt, db->dev, (const uint64_t *)q->dev, (uint64_t *)dev_out, db->lay.M, q->n_cols, c->K,
                                true, (cudaStream_t)stream);
            break;
        case ICM_FORM_I8_DIGITS: {
            const int8_t *planes = (const int8_t *)q->dev + (size_t)c->p.n_limbs * q->n_cols * c->K * 8;
            e = launch_ppmm_i8(q->form, c->i8_digits, db->dev, true, planes, (uint64_t *)dev_out, db->lay.M, q->n_cols,
                               c->K, i8_kpad(c->K), (cudaStream_t)stream);
            break;
        }
        case ICM_FORM_I8_CRT:
        case ICM_FORM_F16_CRT: {
            const void *planes = (const char *)q->dev + (size_t)c->p.n_limbs * q->n_cols * c->K * 8;
            e = launch_ppmm_crt(q->form == ICM_FORM_F16_CRT, c->crt_bn, c->i8_crt, db->dev, true, planes,
                                (uint64_t *)dev_out, db->lay.M, q->n_cols, c->K, i8_kpad(c->K), dev_ws, (cudaStream_t)stream);
            break;
        }
        default: delete sc; return fail(ICM_EUNSUPPORTED, "form not built");
    }
    if (e != cudaSuccess) { delete sc; return fail(ICM_ECUDA, std::string("match: ") + cudaGetErrorString(e)); }
    sc->ctx = c; sc->lay = db->lay; sc->n_eyes = q->n_eyes; sc->n_cols = q->n_cols; sc->folded = 0;
    sc->dev = (uint64_t *)dev_out; sc->bytes = bytes;
    *out = sc;
    return ICM_OK;
}

icm_status icm_fold(icm_ctx *c, const icm_scores *in, void *dev_out, size_t bytes, void *stream, icm_scores **out) {
    if (!c || !in || !dev_out || !out) return fail(ICM_EINVAL, "null argument");
    if (in->ctx != c) return fail(ICM_EINVAL, "handle from another context");
    if (in->folded) return fail(ICM_EINVAL, "scores are already folded");
    const uint32_t groups = (c->p.rho + c->p.fold_k - 1) / c->p.fold_k;
    const uint32_t limbs = in->rescaled ? c->p.n_limbs_q : c->p.n_limbs;
    const size_t need = (size_t)limbs * in->n_eyes * groups * in->lay.M * 8;
    if (bytes < need) return fail(ICM_ENOMEM, "fold buffer too small");
    icm_scores *sc = new (std::nothrow) icm_scores();
    if (!sc) return fail(ICM_ENOMEM, "host allocation");
    cudaError_t e = launch_fold(c, to_dev(in->lay), in->dev, in->n_eyes, limbs, (uint64_t *)dev_out, (cudaStream_t)stream);
    if (e != cudaSuccess) { delete sc; return fail(ICM_ECUDA, std::string("fold: ") + cudaGetErrorString(e)); }
    sc->ctx = c; sc->lay = in->lay; sc->n_eyes = in->n_eyes; sc->n_cols = in->n_eyes * groups; sc->folded = 1;
    sc->rescaled = in->rescaled;
    sc->dev = (uint64_t *)dev_out; sc->bytes = bytes;
    *out = sc;
    return ICM_OK;
}

void icm_scores_destroy(icm_scores *s) { delete s; }

icm_status icm_scores_shape(const icm_scores *s, size_t *n_limbs, size_t *n_cols, size_t *m_rows) {
    if (!s) return fail(ICM_EINVAL, "null argument");
    if (n_limbs) *n_limbs = s->rescaled ? s->ctx->p.n_limbs_q : s->ctx->p.n_limbs;
    if (n_cols) *n_cols = s->n_cols;
    if (m_rows) *m_rows = s->lay.M;
    return ICM_OK;
}

icm_status icm_decrypt_scores(icm_ctx *c, const icm_scores *s, int64_t *dev_num, size_t n, void *stream) {
    if (!c || !s || !dev_num) return fail(ICM_EINVAL, "null argument");
    if (!c->have_keys) return fail(ICM_EINVAL, "icm_keygen has not run");
    if (s->lay.slot_log2) return fail(ICM_EINVAL, "slot-encoded scores decode with icm_decrypt_slots");
    if (n < (size_t)s->n_cols * s->lay.n_real) return fail(ICM_ENOMEM, "numerator buffer too small");
    cudaError_t e = launch_decrypt(c, to_dev(s->lay), s->dev, s->n_cols, s->rescaled != 0, dev_num,
                                   (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(ICM_ECUDA, std::string("decrypt: ") + cudaGetErrorString(e));
    return ICM_OK;
}

icm_status icm_decrypt_scores_max_error(icm_ctx *c, const icm_scores *s, int64_t *dev_num, size_t n, float *dev_max_err,
                                        void *stream) {
    if (!c || !s || !dev_num || !dev_max_err) return fail(ICM_EINVAL, "null argument");
    if (!c->have_keys) return fail(ICM_EINVAL, "icm_keygen has not run");
    if (s->lay.slot_log2) return fail(ICM_EINVAL, "slot-encoded scores decode with icm_decrypt_slots");
    if (n < (size_t)s->n_cols * s->lay.n_real) return fail(ICM_ENOMEM, "numerator buffer too small");
    cudaError_t e = cudaMemsetAsync(dev_max_err, 0, sizeof(float), (cudaStream_t)stream);
    if (e == cudaSuccess)
        e = launch_decrypt(c, to_dev(s->lay), s->dev, s->n_cols, s->rescaled != 0, dev_num, (cudaStream_t)stream,
                           reinterpret_cast<uint32_t *>(dev_max_err));
    if (e != cudaSuccess) return fail(ICM_ECUDA, std::string("decrypt: ") + cudaGetErrorString(e));
    return ICM_OK;
}

icm_status icm_rescale_bytes(const icm_scores *in, size_t *bytes) {
    if (!in || !bytes) return fail(ICM_EINVAL, "null argument");
    *bytes = (size_t)in->ctx->p.n_limbs_q * in->n_cols * in->lay.M * 8;
    return ICM_OK;
}

icm_status icm_rescale(icm_ctx *c, const icm_scores *in, void *dev_out, size_t bytes, void *stream, icm_scores **out) {
    if (!c || !in || !dev_out || !out) return fail(ICM_EINVAL, "null argument");
    if (in->ctx != c) return fail(ICM_EINVAL, "handle from another context");
    if (in->rescaled) return fail(ICM_EINVAL, "scores are already rescaled");
    if (c->p.n_limbs_q >= c->p.n_limbs) return fail(ICM_EINVAL, "no limb of Q' to drop");
    size_t need;
    icm_rescale_bytes(in, &need);
    if (bytes < need) return fail(ICM_ENOMEM, "rescale buffer too small");
    icm_scores *sc = new (std::nothrow) icm_scores();
    if (!sc) return fail(ICM_ENOMEM, "host allocation");
    cudaError_t e = launch_rescale(c, in->dev, (uint64_t)in->n_cols * in->lay.M, (uint64_t *)dev_out,
                                   (cudaStream_t)stream);
    if (e != cudaSuccess) { delete sc; return fail(ICM_ECUDA, std::string("rescale: ") + cudaGetErrorString(e)); }
    *sc = *in;
    sc->rescaled = 1;
    sc->dev = (uint64_t *)dev_out; sc->bytes = bytes;
    *out = sc;
    return ICM_OK;
}

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// icm_match_host runs the eyes in two parts so that the copies of one part overlap the product of
// the other: the query ciphertext of part 2 is copied in while part 1 is prepared and matched, and
// the folded scores of part 1 are copied out while part 2 is matched.  Workspace: the ciphertext
// of both parts, the operand, scores and match workspace of the larger part (reused in turn), and
// the folded scores of both parts.
struct HostParts {
    size_t n1, n2;
    size_t ct1, ct2, op, sc, mw, fo1, fo2;
    size_t off_ct2, off_op, off_sc, off_mw, off_fo1, off_fo2, total;
};
static icm_status host_parts(const icm_ctx *c, const icm_db *db, size_t n_eyes, icm_form form, HostParts &h) {
    h.n1 = (n_eyes + 1) / 2;
    h.n2 = n_eyes - h.n1;
    icm_status s;
    if ((s = icm_query_ct_bytes(c, h.n1, &h.ct1)) != ICM_OK) return s;
    if ((s = icm_query_ct_bytes(c, h.n2, &h.ct2)) != ICM_OK) return s;
    if ((s = icm_query_op_bytes(c, h.n1, form, &h.op)) != ICM_OK) return s;
    if ((s = icm_scores_bytes(c, db, h.n1, 0, &h.sc)) != ICM_OK) return s;
    if ((s = icm_match_workspace_bytes(c, db, h.n1, form, &h.mw)) != ICM_OK) return s;
    if ((s = icm_scores_bytes(c, db, h.n1, 1, &h.fo1)) != ICM_OK) return s;
    if ((s = icm_scores_bytes(c, db, h.n2, 1, &h.fo2)) != ICM_OK) return s;
    h.off_ct2 = align256(h.ct1);
    h.off_op = h.off_ct2 + align256(h.ct2);
    h.off_sc = h.off_op + align256(h.op);
    h.off_mw = h.off_sc + align256(h.sc);
    h.off_fo1 = h.off_mw + align256(h.mw);
    h.off_fo2 = h.off_fo1 + align256(h.fo1);
    h.total = h.off_fo2 + align256(h.fo2);
    return ICM_OK;
}

icm_status icm_match_host_workspace_bytes(const icm_ctx *c, const icm_db *db, size_t n_eyes, icm_form form,
                                          size_t *bytes) {
    if (!c || !db || !bytes) return fail(ICM_EINVAL, "null argument");
    HostParts h;
    icm_status s = host_parts(c, db, n_eyes, form, h);
    if (s != ICM_OK) return s;
    *bytes = h.total;
    return ICM_OK;
}

// prepare, match and fold one part of the eyes (device buffers of the part)
static icm_status host_part(icm_ctx *c, const icm_db *db, const void *d_ct, size_t n, icm_form form, void *d_op,
                            size_t op, void *d_sc, size_t sc, void *d_mw, size_t mw, void *d_fo, size_t fo,
                            void *stream) {
    icm_query *q = nullptr;
    icm_scores *m = nullptr, *f = nullptr;
    icm_status s = icm_query_prepare(c, d_ct, n, form, d_op, op, stream, &q);
    if (s != ICM_OK) return s;
    s = icm_match(c, db, q, d_sc, sc, mw ? d_mw : nullptr, mw, stream, &m);
    if (s == ICM_OK) s = icm_fold(c, m, d_fo, fo, stream, &f);
    icm_query_destroy(q);
    icm_scores_destroy(m);
    icm_scores_destroy(f);
    return s;
}

icm_status icm_match_host(icm_ctx *c, const icm_db *db, const uint64_t *host_ct, size_t n_eyes, icm_form form,
                          uint64_t *host_folded, void *dev_ws, size_t ws_bytes, void *stream) {
    if (!c || !db || !host_ct || !host_folded || !dev_ws) return fail(ICM_EINVAL, "null argument");
    if (n_eyes == 0) return fail(ICM_EINVAL, "no eyes");
    HostParts h;
    icm_status s = host_parts(c, db, n_eyes, form, h);
    if (s != ICM_OK) return s;
    if (ws_bytes < h.total) return fail(ICM_ENOMEM, "workspace too small");
    char *w = (char *)dev_ws;
    cudaStream_t st = (cudaStream_t)stream;
    // wire format [Lq][n rho][K]: part p holds eyes [e0, e0 + n_p) as its own wire-format buffer;
    // folded scores [L][n G][M] (G folded columns per eye): part p's rows of every limb
    const size_t Lq = c->p.n_limbs_q, L = c->p.n_limbs, rho = c->p.rho, K = c->K;
    const size_t G = (rho + c->p.fold_k - 1) / c->p.fold_k, M = db->lay.M;
    const size_t ct_row = rho * K * 8, fo_row = G * M * 8;           // bytes per eye and limb
    auto h2d = [&](void *dst, size_t e0, size_t n, cudaStream_t s2) {
        return cudaMemcpy2DAsync(dst, n * ct_row, reinterpret_cast<const char *>(host_ct) + e0 * ct_row,
                                 n_eyes * ct_row, n * ct_row, Lq, cudaMemcpyHostToDevice, s2);
    };
    auto d2h = [&](const void *src, size_t e0, size_t n, cudaStream_t s2) {
        return cudaMemcpy2DAsync(reinterpret_cast<char *>(host_folded) + e0 * fo_row, n_eyes * fo_row, src,
                                 n * fo_row, n * fo_row, L, cudaMemcpyDeviceToHost, s2);
    };
    if (h.n2 == 0) {                                                 // a single eye: no second part
        CUDA_TRY(h2d(w, 0, h.n1, st));
        s = host_part(c, db, w, h.n1, form, w + h.off_op, h.op, w + h.off_sc, h.sc, w + h.off_mw, h.mw,
                      w + h.off_fo1, h.fo1, stream);
        if (s != ICM_OK) return s;
        CUDA_TRY(d2h(w + h.off_fo1, 0, h.n1, st));
        return ICM_OK;
    }
    cudaStream_t cs = nullptr;
    cudaEvent_t ev_start = nullptr, ev_h2 = nullptr, ev_f1 = nullptr, ev_d1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (cudaEvent_t *ev : {&ev_start, &ev_h2, &ev_f1, &ev_d1})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    // the copy stream starts after the caller's earlier work on `stream` (which may still read
    // this workspace)
    if (e == cudaSuccess) e = cudaEventRecord(ev_start, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_start, 0);
    if (e == cudaSuccess) e = h2d(w, 0, h.n1, st);
    if (e == cudaSuccess) e = h2d(w + h.off_ct2, h.n1, h.n2, cs);
    if (e == cudaSuccess) e = cudaEventRecord(ev_h2, cs);
    if (e == cudaSuccess) {
        s = host_part(c, db, w, h.n1, form, w + h.off_op, h.op, w + h.off_sc, h.sc, w + h.off_mw, h.mw,
                      w + h.off_fo1, h.fo1, stream);
        if (s == ICM_OK) {
            e = cudaEventRecord(ev_f1, st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_f1, 0);
            if (e == cudaSuccess) e = d2h(w + h.off_fo1, 0, h.n1, cs);
            if (e == cudaSuccess) e = cudaEventRecord(ev_d1, cs);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_h2, 0);
            if (e == cudaSuccess)
                s = host_part(c, db, w + h.off_ct2, h.n2, form, w + h.off_op, h.op, w + h.off_sc, h.sc,
                              w + h.off_mw, h.mw, w + h.off_fo2, h.fo2, stream);
            if (e == cudaSuccess && s == ICM_OK) e = d2h(w + h.off_fo2, h.n1, h.n2, st);
            // the caller's stream completes only after both parts' copies
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_d1, 0);
        }
    }
    for (cudaEvent_t ev : {ev_start, ev_h2, ev_f1, ev_d1})
        if (ev) cudaEventDestroy(ev);
    if (cs) cudaStreamDestroy(cs);
    if (s != ICM_OK) return s;
    if (e != cudaSuccess) return fail(ICM_ECUDA, std::string("match_host: ") + cudaGetErrorString(e));
    return ICM_OK;
}

icm_status icm_ppmm_workspace_bytes(icm_form form, uint32_t n_limbs, size_t M, size_t N, size_t K, size_t *bytes) {
    if (!bytes) return fail(ICM_EINVAL, "null argument");
    switch (form) {
        case ICM_FORM_U64: *bytes = 0; return ICM_OK;
        case ICM_FORM_I8_DIGITS:
        case ICM_FORM_I8_CRT:
        case ICM_FORM_F16_CRT: {
            // sized for the worst case of primes just below 2^60
            const int pf = form == ICM_FORM_F16_CRT ? (int)ICM_FORM_I8_CRT : (int)form;
            const uint64_t qworst = (1ull << 60) - 1;
            const uint32_t P = i8_planes(pf, &qworst, 1, K);
            if (!P) return fail(ICM_EBOUND, "CRT form unavailable for this K");
            *bytes = crt_plane_bytes(form == ICM_FORM_F16_CRT, n_limbs, P, N, i8_kpad(K));
            if (form != ICM_FORM_I8_DIGITS) *bytes += 256 + crt_scratch_bytes(n_limbs, P, N, M);
            return ICM_OK;
        }
        case ICM_FORM_I8_P2: *bytes = (size_t)n_limbs * 2 * N * i8_kpad(K); return ICM_OK;
        default: return fail(ICM_EUNSUPPORTED, "form not built");
    }
}

icm_status icm_ppmm(icm_form form, const uint64_t *q, uint32_t n_limbs, const uint64_t *dev_A, const uint64_t *dev_B,
                    uint64_t *dev_C, size_t M, size_t N, size_t K, void *dev_ws, size_t ws_bytes, void *stream) {
    if (!q) return fail(ICM_EINVAL, "null prime list");
    // empty operands may be null: no element of an empty matrix is read or written
    if ((!dev_A && M && K) || (!dev_B && N && K) || (!dev_C && M && N)) return fail(ICM_EINVAL, "null argument");
    if (n_limbs < 1 || n_limbs > ICM_MAX_LIMBS) return fail(ICM_EINVAL, "n_limbs must be 1..8");
    for (uint32_t l = 0; l < n_limbs; ++l)
        if (q[l] < 3 || q[l] >= (1ull << 60) || !(q[l] & 1)) return fail(ICM_EINVAL, "moduli must be odd and below 2^60");
    if ((uint64_t)K >= (1ull << 32)) return fail(ICM_EBOUND, "K too large for exact accumulation");
    std::vector<uint64_t> qv(q, q + n_limbs);
    I8Consts kp2;
    if (form == ICM_FORM_I8_P2) {                       // moduli checked before any device call
        const char *why = "";
        if (!make_i8_consts(form, qv.data(), qv.size(), K, kp2, &why)) return fail(ICM_EINVAL, why);
    }
    const LimbTable lt = make_limb_table(qv);
    if (crt_set_attributes() != cudaSuccess) return fail(ICM_ECUDA, "kernel attributes");
    cudaError_t e;
    switch (form) {
        case ICM_FORM_U64: e = launch_ppmm_u64(lt, dev_A, dev_B, dev_C, M, N, K, false, (cudaStream_t)stream); break;
        case ICM_FORM_I8_DIGITS: {
            I8Consts k;
            const char *why = "";
            if (!make_i8_consts(form, qv.data(), qv.size(), K, k, &why)) return fail(ICM_EBOUND, why);
            const size_t pl = (size_t)n_limbs * 8 * N * i8_kpad(K);
            if (pl && (!dev_ws || ws_bytes < pl)) return fail(ICM_ENOMEM, "workspace too small");
            e = launch_planes(form, k, dev_B, (int8_t *)dev_ws, N, K, i8_kpad(K), (cudaStream_t)stream);
            if (e == cudaSuccess)
                e = launch_ppmm_i8(form, k, dev_A, false, (const int8_t *)dev_ws, dev_C, M, N, K, i8_kpad(K),
                                   (cudaStream_t)stream);
            break;
        }
        case ICM_FORM_I8_P2: {
            const size_t pl = (size_t)n_limbs * 2 * N * i8_kpad(K);
            if (pl && (!dev_ws || ws_bytes < pl)) return fail(ICM_ENOMEM, "workspace too small");
            e = launch_planes(form, kp2, dev_B, (int8_t *)dev_ws, N, K, i8_kpad(K), (cudaStream_t)stream);
            if (e == cudaSuccess)
                e = launch_ppmm_i8(form, kp2, dev_A, false, (const int8_t *)dev_ws, dev_C, M, N, K, i8_kpad(K),
                                   (cudaStream_t)stream);
            break;
        }
        case ICM_FORM_I8_CRT:
        case ICM_FORM_F16_CRT: {
            I8Consts k;
            const char *why = "";
            if (!make_i8_consts(ICM_FORM_I8_CRT, qv.data(), qv.size(), K, k, &why)) return fail(ICM_EBOUND, why);
            const bool f16 = form == ICM_FORM_F16_CRT;
            const size_t pl = crt_plane_bytes(f16, n_limbs, k.n_mod, N, i8_kpad(K));
            const size_t sc = crt_scratch_bytes(n_limbs, k.n_mod, N, M);
            if ((pl || sc) && (!dev_ws || ws_bytes < align256(pl) + sc)) return fail(ICM_ENOMEM, "workspace too small");
            e = launch_crt_planes(f16, k, dev_B, dev_ws, N, K, i8_kpad(K), (cudaStream_t)stream);
            if (e == cudaSuccess)
                e = launch_ppmm_crt(f16, 256, k, dev_A, false, dev_ws, dev_C, M, N, K, i8_kpad(K),
                                    (char *)dev_ws + align256(pl), (cudaStream_t)stream);
            break;
        }
        default: return fail(ICM_EUNSUPPORTED, "form not built");
    }
    if (e != cudaSuccess) return fail(ICM_ECUDA, std::string("ppmm: ") + cudaGetErrorString(e));
    return ICM_OK;
}

icm_status icm_sync(void *stream, uint32_t timeout_ms) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery((cudaStream_t)stream);
        if (e == cudaSuccess) return ICM_OK;
        if (e != cudaErrorNotReady) return fail(ICM_ECUDA, cudaGetErrorString(e));
        const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
        if (ms >= (long long)timeout_ms) return fail(ICM_ETIMEOUT, "stream did not finish in time");
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

}  // extern "C"
