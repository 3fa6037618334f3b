// Fold (Algorithm 2, linear key-free part) and decryption for checking.
//
// Fold: for eye e and group g of fold_k consecutive rotations, ct'_{e,g} = sum_{r in g} X^r ct_{e,r},
// applied to the a-part polynomial and to every b-block polynomial of the MSRLWE result.  The
// shift is the global rotation index r (Algorithm 2 rotates term rk + r' by rk + r'); X^r is the
// negacyclic monomial shift, (X^r p)[i] = p[i - r] for i >= r and -p[N + i - r] for i < r.  Slot i
// of the shifted result then carries database entry i - r, so that a group never stacks two
// scores of the same database entry (Section 4.3).  The kernel is HBM-bound: every input column
// is read once, one output column is written per group.
//
// Decryption (Section 2.2.2, Dec(a, b) = a * sk + b per b-block): D = C_b + s_{db,t} * C_a modulo
// every q_l, then a fixed-point CRT gives D / Q_db modulo 1, and the numerator is the nearest
// integer to D_centred / (Q' Delta).  After rescaling the same holds modulo Q with scale Delta.
//
// Rescaling by Q' (Section 2.2.2, Maintenance: RS divides by a modulus factor and rounds, here
// the factor Q' = q_Lq ... q_{L-1}, so the scores leave at the query modulus Q with scale Delta):
// per coefficient, yh_i = x_i (Q'/q_i)^-1 mod q_i for the limbs of Q', the correction
// v = floor((sum_i F_i + 2^63) / 2^64) from the 64-bit fixed-point fractions
// F_i = floor(yh_i floor(2^128 / q_i) / 2^64) (integer arithmetic only), the centred
// y = sum_i yh_i (Q'/q_i) - v Q' = x mod Q', and x'_j = (x_j - y mod q_j) Q'^-1 mod q_j for the
// limbs of Q.  HBM-bound: reads L words and writes L_q words per coefficient.
#include "icm_internal.h"

#include <algorithm>

namespace {

using icm::LayoutDev;

// Stored row position of coefficient `coef` of block `blk` (blk = -1: the a-part), or -1 if the
// coefficient is not stored (the gap between the real rows and the tail of a partial block).
__device__ __forceinline__ int64_t pos_of(const LayoutDev &L, int blk, uint32_t coef) {
    if (blk < 0) return coef;
    if ((uint32_t)blk < L.n_full) return (int64_t)L.N + (int64_t)blk * L.N + coef;
    const int64_t base = (int64_t)L.N + (int64_t)L.n_full * L.N;
    if (coef < L.rem) return base + coef;
    if (coef >= L.tail_lo) return base + L.rem + (coef - L.tail_lo);
    return -1;
}

// Block and coefficient of stored row x; tail rows of a partial block report tail = true.
__device__ __forceinline__ void coef_of(const LayoutDev &L, uint64_t x, int &blk, uint32_t &coef, bool &tail) {
    tail = false;
    if (x < L.N) { blk = -1; coef = (uint32_t)x; return; }
    const uint64_t b = x - L.N;
    const uint64_t full = (uint64_t)L.n_full * L.N;
    if (b < full) { blk = (int)(b / L.N); coef = (uint32_t)(b % L.N); return; }
    const uint32_t rel = (uint32_t)(b - full);
    blk = (int)L.n_full;
    if (rel < L.rem) { coef = rel; return; }
    coef = L.tail_lo + (rel - L.rem);
    tail = true;
}

struct FoldArgs {
    LayoutDev lay;
    uint32_t rho, k, groups, n_eyes, L;
    uint64_t q[ICM_MAX_LIMBS], r64[ICM_MAX_LIMBS];
    const uint64_t *in;    // [L][n_eyes*rho][M]
    uint64_t *out;         // [L][n_eyes*groups][M]
};

// grid: (ceil(M / 256), n_eyes * groups, L).  Each thread sums at most fold_k (<= 32) terms,
// adding q - v for the wrapped (negated) ones; fold_k * q < 2^64 keeps the sum exact.
__global__ void __launch_bounds__(256) k_fold(FoldArgs a) {
    const uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t oc = blockIdx.y, l = blockIdx.z;
    if (x >= a.lay.M) return;
    const uint32_t e = oc / a.groups, g = oc % a.groups;
    const uint64_t q = a.q[l];
    uint64_t *dst = a.out + ((size_t)l * a.n_eyes * a.groups + oc) * a.lay.M + x;
    int blk; uint32_t coef; bool tail;
    coef_of(a.lay, x, blk, coef, tail);
    if (tail) { *dst = 0; return; }
    const uint32_t r0 = g * a.k, r1 = min(r0 + a.k, a.rho);
    const uint64_t *col = a.in + ((size_t)l * a.n_eyes * a.rho + (size_t)e * a.rho) * a.lay.M;
    uint64_t acc = 0;
#pragma unroll 4
    for (uint32_t r = r0; r < r1; ++r) {
        const bool wrap = coef < r;
        const uint32_t src = wrap ? a.lay.N + coef - r : coef - r;
        const int64_t p = pos_of(a.lay, blk, src);
        const uint64_t v = (p >= 0) ? col[(size_t)r * a.lay.M + p] : 0;
        acc += wrap ? (v ? q - v : 0) : v;
    }
    *dst = reduce64(acc, q, a.r64[l]);
}

struct DecArgs {
    LayoutDev lay;
    uint32_t L, h, n_cols;
    uint64_t q[ICM_MAX_LIMBS], r64[ICM_MAX_LIMBS];
    icm::CrtDecode crt;
    const int32_t *sdb_pos; const int8_t *sdb_sgn;
    const uint64_t *sc;    // [L][n_cols][M]
    int64_t *num;          // [n_cols][n_real]
    uint32_t *err_bits;    // optional: max |x - round(x)| over all outputs, as fp32 bits
};

// grid: (ceil(n_real / 256), n_cols).  One thread per (column, real database row).
__global__ void __launch_bounds__(256) k_decrypt(DecArgs a) {
    const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t j = blockIdx.y;
    if (r >= a.lay.n_real) return;
    const uint32_t N = a.lay.N;
    const uint32_t t = (uint32_t)(r / N), i = (uint32_t)(r % N);
    const int64_t pos = pos_of(a.lay, (int)t, i);
    uint64_t fhi = 0, flo = 0;                      // sum_l y_l floor(2^128 / q_l) mod 2^128
    for (uint32_t l = 0; l < a.L; ++l) {
        const uint64_t q = a.q[l];
        const uint64_t *col = a.sc + ((size_t)l * a.n_cols + j) * a.lay.M;
        uint64_t d = col[pos];
        for (uint32_t c = 0; c < a.h; ++c) {
            const uint32_t p = (uint32_t)a.sdb_pos[t * a.h + c];
            const int s = a.sdb_sgn[t * a.h + c];
            const uint64_t term = (i >= p) ? col[i - p] : col[N + i - p];
            const bool neg = (i >= p) ? (s < 0) : (s > 0);
            d = neg ? sub_mod(d, term, q) : add_mod(d, term, q);
        }
        const uint64_t y = mulmod_shoup(d, a.crt.inv[l], a.crt.invs[l], q);
        // y * (rhi 2^64 + rlo) mod 2^128
        const uint64_t plo = y * a.crt.rlo[l];
        const uint64_t phi = __umul64hi(y, a.crt.rlo[l]) + y * a.crt.rhi[l];
        const uint64_t nlo = flo + plo;
        fhi = fhi + phi + (nlo < flo ? 1 : 0);
        flo = nlo;
    }
    // F / 2^128 is D / Q_db modulo 1; as a signed 128-bit number it is the centred value.
    const double frac = (double)(int64_t)fhi * 0x1p-64 + (double)flo * 0x1p-128;
    const double x = frac * a.crt.q_over_delta;
    const double n = rint(x);
    a.num[(size_t)j * a.lay.n_real + r] = (int64_t)n;
    if (a.err_bits) {
        // distance of the decoded value from the integer it rounds to (numerator units); the
        // bits of non-negative floats order like unsigned integers
        uint32_t e = __float_as_uint((float)fabs(x - n));
        e = __reduce_max_sync(__activemask(), e);
        if ((threadIdx.x & 31) == (__ffs(__activemask()) - 1)) atomicMax(a.err_bits, e);
    }
}

struct RsArgs {
    icm::RescaleConsts k;
    const uint64_t *in;    // [L][n]
    uint64_t *out;         // [Lq][n]
    uint64_t n;
};

// Rescale one coefficient c of [L][n] into [Lq][n].
__device__ __forceinline__ void rescale_one(const icm::RescaleConsts &k, const uint64_t *in, uint64_t *out, uint64_t n,
                                            uint64_t c) {
    const uint32_t L = k.L, Lq = k.Lq;
    uint64_t yh[ICM_MAX_LIMBS];
    uint64_t slo = 0, shi = 0;                                     // sum of the F_i, 128-bit
#pragma unroll
    for (uint32_t i = 0; i < ICM_MAX_LIMBS; ++i) {
        if (i < Lq || i >= L) continue;
        const uint64_t q = k.q[i];
        yh[i] = mulmod_shoup(in[(size_t)i * n + c], k.yinv[i], k.yinvs[i], q);
        // F_i = yh rhi + floor(yh rlo / 2^64): exact, and < 2^64 because yh < q_i
        const uint64_t f = yh[i] * k.rhi[i] + __umul64hi(yh[i], k.rlo[i]);
        slo += f;
        shi += slo < f ? 1 : 0;
    }
    const uint64_t v = shi + ((slo >> 63) & 1);                    // floor((S + 2^63) / 2^64)
    for (uint32_t j = 0; j < Lq; ++j) {
        const uint64_t q = k.q[j];
        uint64_t y = 0;
#pragma unroll
        for (uint32_t i = 0; i < ICM_MAX_LIMBS; ++i)
            if (i >= Lq && i < L) y = add_mod(y, mulmod_shoup(yh[i], k.w[j][i], k.ws[j][i], q), q);
        y = sub_mod(y, mulmod_shoup(v, k.qp[j], k.qps[j], q), q);
        const uint64_t d = sub_mod(in[(size_t)j * n + c], y, q);
        out[(size_t)j * n + c] = mulmod_shoup(d, k.qpinv[j], k.qpinvs[j], q);
    }
}

// Two coefficients per thread (independent chains for latency hiding); consecutive threads read
// consecutive words of a limb.
__global__ void __launch_bounds__(256) k_rescale(const __grid_constant__ RsArgs a) {
    const uint64_t c0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x);
    const uint64_t half = (a.n + 1) / 2;
    if (c0 >= half) return;
    rescale_one(a.k, a.in, a.out, a.n, c0);
    if (c0 + half < a.n) rescale_one(a.k, a.in, a.out, a.n, c0 + half);
}

}  // namespace

namespace icm {

cudaError_t launch_rescale(const icm_ctx *c, const uint64_t *d_in, uint64_t n, uint64_t *d_out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    RsArgs a{c->rs, d_in, d_out, n};
    const uint64_t threads = (n + 1) / 2;
    k_rescale<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}


cudaError_t launch_fold(const icm_ctx *c, const LayoutDev &lay, const uint64_t *d_in, uint32_t n_eyes, uint32_t limbs,
                        uint64_t *d_out, cudaStream_t st) {
    FoldArgs a{};
    a.lay = lay; a.rho = c->p.rho; a.k = c->p.fold_k;
    a.groups = (c->p.rho + c->p.fold_k - 1) / c->p.fold_k;
    a.n_eyes = n_eyes; a.L = limbs;                 // the first `limbs` primes (Q's come first)
    for (uint32_t l = 0; l < a.L; ++l) { a.q[l] = c->q[l]; a.r64[l] = c->lt.r64[l]; }
    a.in = d_in; a.out = d_out;
    if (n_eyes == 0 || lay.M == 0) return cudaSuccess;
    dim3 grid((unsigned)((lay.M + 255) / 256), n_eyes * a.groups, a.L);
    k_fold<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_decrypt(const icm_ctx *c, const LayoutDev &lay, const uint64_t *d_scores, uint32_t n_cols,
                           bool rescaled, int64_t *d_num, cudaStream_t st, uint32_t *d_err_bits) {
    DecArgs a{};
    a.lay = lay; a.L = rescaled ? c->p.n_limbs_q : c->p.n_limbs; a.h = c->p.hamming_weight; a.n_cols = n_cols;
    for (uint32_t l = 0; l < a.L; ++l) { a.q[l] = c->q[l]; a.r64[l] = c->lt.r64[l]; }
    a.crt = rescaled ? c->crt_q : c->crt;
    a.sdb_pos = c->d_sdb_pos; a.sdb_sgn = c->d_sdb_sgn;
    a.sc = d_scores; a.num = d_num; a.err_bits = d_err_bits;
    if (n_cols == 0 || lay.n_real == 0) return cudaSuccess;
    dim3 grid((unsigned)((lay.n_real + 255) / 256), n_cols);
    k_decrypt<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace icm
