// Query operand preparation, the first step of the CCMM (Section 2.3): the query ciphertext
// arrives modulo Q = q_0 (L_q = 1) or q_0 q_1 (L_q = 2); each coefficient is lifted to its
// centred representative x in (-Q/2, Q/2] and reduced modulo every prime q_l of the database
// modulus, so that the products of the CCMM are taken over the integers modulo Q_db.
#include "icm_internal.h"

namespace {

struct ExtArgs {
    uint32_t L, Lq;
    uint64_t n;                              // elements per limb (n_cols * K)
    uint64_t q[ICM_MAX_LIMBS], r64[ICM_MAX_LIMBS];
    uint64_t q0m[ICM_MAX_LIMBS], q0ms[ICM_MAX_LIMBS];   // q_0 mod q_l and Shoup companion
    uint64_t Qm[ICM_MAX_LIMBS];              // Q mod q_l
    uint64_t inv01, inv01s;                  // q_0^-1 mod q_1 and Shoup companion
    const uint64_t *ct;                      // [Lq][n]
    uint64_t *out;                           // [L][n]
};

__global__ void __launch_bounds__(256) k_query_extend(ExtArgs a) {
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < a.n;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r0 = a.ct[idx];
        if (a.Lq == 1) {
            // x = r0 in [0, q_0); centred: x - q_0 when x > (q_0 - 1) / 2
            const bool neg = r0 > (a.q[0] - 1) / 2;
            const uint64_t mag = neg ? a.q[0] - r0 : r0;        // |x|
            for (uint32_t l = 0; l < a.L; ++l) {
                const uint64_t m = reduce64(mag, a.q[l], a.r64[l]);
                a.out[(size_t)l * a.n + idx] = (neg && m) ? a.q[l] - m : m;
            }
        } else {
            // Garner: x = r0 + q_0 d with d = (r1 - r0) q_0^-1 mod q_1, x in [0, Q)
            const uint64_t q1 = a.q[1];
            const uint64_t r1 = a.ct[a.n + idx];
            const uint64_t diff = sub_mod(r1, reduce64(r0, q1, a.r64[1]), q1);
            const uint64_t d = mulmod_shoup(diff, a.inv01, a.inv01s, q1);
            // centred: x > (Q - 1)/2  <=>  d > (q1 - 1)/2, or d == (q1 - 1)/2 and r0 > (q0 - 1)/2
            const uint64_t h1 = (q1 - 1) / 2;
            const bool neg = d > h1 || (d == h1 && r0 > (a.q[0] - 1) / 2);
            for (uint32_t l = 0; l < a.L; ++l) {
                const uint64_t ql = a.q[l];
                uint64_t v = add_mod(reduce64(r0, ql, a.r64[l]), mulmod_shoup(d, a.q0m[l], a.q0ms[l], ql), ql);
                if (neg) v = sub_mod(v, a.Qm[l], ql);
                a.out[(size_t)l * a.n + idx] = v;
            }
        }
    }
}

uint64_t mulmod_host(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)((unsigned __int128)a * b % q); }
uint64_t powmod_host(uint64_t b, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    b %= q;
    while (e) { if (e & 1) r = mulmod_host(r, b, q); b = mulmod_host(b, b, q); e >>= 1; }
    return r;
}

}  // namespace

namespace icm {

cudaError_t launch_query_extend(const icm_ctx *c, const uint64_t *d_ct, uint32_t n_cols, uint64_t *d_op,
                                cudaStream_t st) {
    ExtArgs a{};
    a.L = c->p.n_limbs; a.Lq = c->p.n_limbs_q;
    a.n = (uint64_t)n_cols * c->K;
    for (uint32_t l = 0; l < a.L; ++l) {
        a.q[l] = c->q[l];
        a.r64[l] = c->lt.r64[l];
        a.q0m[l] = c->q[0] % c->q[l];
        a.q0ms[l] = shoup_of(a.q0m[l], c->q[l]);
        uint64_t Qm = 1;
        for (uint32_t j = 0; j < a.Lq; ++j) Qm = mulmod_host(Qm, c->q[j] % c->q[l], c->q[l]);
        a.Qm[l] = Qm;
    }
    if (a.Lq == 2) {
        a.inv01 = powmod_host(c->q[0] % c->q[1], c->q[1] - 2, c->q[1]);
        a.inv01s = shoup_of(a.inv01, c->q[1]);
    }
    a.ct = d_ct; a.out = d_op;
    if (a.n == 0) return cudaSuccess;
    const uint64_t blocks = (a.n + 255) / 256;
    k_query_extend<<<(unsigned)(blocks < 152u * 64u ? blocks : 152u * 64u), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace icm
