// Encryption kernels of libicm (setup path, not timed in the matching step).
//
// Database chunk, MSRLWE-RGSW form (Section 6.2.1: a pair of encryptions of M_db and of
// M_db * S_q under the database secrets, modulus Q_db = Q * Q'):
//   a-part row i, column k:   A[i][k] uniform modulo Q_db (an independent residue per limb)
//   b-row r = t * N_db + i:   B[r][k] = -(s_{db,t} * A[:, k])[i] + Q' * W[r][k] + E[r][k]
//   W[r][k] = c'_r[k] for k < d2 (the masked bit-vector of template r, Section 2.1.3) and
//   W[r][d2 + j] = (M_db S_q)[r][j] for j < N_q (S_q: vertical stack of the negacyclic matrices
//   of the query secrets).  The gadget factor Q' makes Q' * Q = 0 modulo Q_db, which removes
//   the query's wrap-around multiple of Q from the decrypted product.
// Stored rows are written in the balanced-digit form of icm_device.cuh (to_digit_form).
// Query eyes, MSRLWE form modulo Q (Section 2.3):
//   b_{t,j} = -(s_{q,t} * a_j) + Delta * c'_j[t N_q .. (t+1) N_q) + e_{t,j},  a_j uniform mod Q,
//   where column j = eye * rho + r holds rotation r of the eye (Section 2.1.2).
#include "icm_internal.h"

namespace {

using icm::LayoutDev;

// Map a b-region index (0-based, after the a-part rows) to its logical row (t, i).
__device__ __forceinline__ void b_row_of(const LayoutDev &L, uint64_t bidx, uint32_t &t, uint32_t &i) {
    const uint64_t full = (uint64_t)L.n_full * L.N;
    if (bidx < full) {
        t = (uint32_t)(bidx / L.N);
        i = (uint32_t)(bidx % L.N);
    } else {
        const uint32_t rel = (uint32_t)(bidx - full);
        t = L.n_full;
        i = rel < L.rem ? rel : L.tail_lo + (rel - L.rem);
    }
}

__device__ __forceinline__ int template_bit(const uint8_t *tpl, uint32_t b) { return (tpl[b >> 3] >> (b & 7)) & 1; }

struct DbMsgArgs {
    LayoutDev lay;
    uint32_t K, d2, Nq, nqblk, h, code_bits, L, Lq;
    const uint8_t *codes, *masks;      // [n_real][code_bits/8]
    const int32_t *wmsg;               // message rows [n_real][d2] (slot encoding), or null: c' of codes
    const int32_t *sq_pos; const int8_t *sq_sgn;   // [nqblk][h]
    uint64_t qp[ICM_MAX_LIMBS], qps[ICM_MAX_LIMBS], q[ICM_MAX_LIMBS];
    uint64_t *db;                      // [L][M][K]
};

// Pass 1: the message residues Q' * W[r][k] of every stored b-row, for every limb.  The message
// row is the masked bit-vector c' of template r (coefficient encoding) or, for a slot-encoded
// chunk, the given row of rounded slot-encoding coefficients.
__global__ void __launch_bounds__(512) k_db_messages(DbMsgArgs a) {
    extern __shared__ unsigned char smem[];
    int32_t *cp = reinterpret_cast<int32_t *>(smem);                        // [d2]
    int32_t *spos = cp + ((a.d2 + 3) & ~3u);                                // [nqblk*h]
    int8_t *ssgn = reinterpret_cast<int8_t *>(spos + a.nqblk * a.h);

    const uint64_t bidx = blockIdx.x;
    const uint64_t pos = a.lay.N + bidx;
    uint32_t t, i;
    b_row_of(a.lay, bidx, t, i);
    const uint64_t r = (uint64_t)t * a.lay.N + i;
    const bool real = r < a.lay.n_real;
    const uint32_t tb = a.code_bits / 8;
    for (uint32_t k = threadIdx.x; k < a.d2; k += blockDim.x) {
        int v = 0;
        if (real && a.wmsg) {
            v = a.wmsg[r * a.d2 + k];
        } else if (real && k < a.code_bits) {
            const int c = template_bit(a.codes + r * tb, k), m = template_bit(a.masks + r * tb, k);
            v = m - 2 * (c & m);
        }
        cp[k] = v;
    }
    for (uint32_t x = threadIdx.x; x < a.nqblk * a.h; x += blockDim.x) { spos[x] = a.sq_pos[x]; ssgn[x] = a.sq_sgn[x]; }
    __syncthreads();

    for (uint32_t k = threadIdx.x; k < a.K; k += blockDim.x) {
        int32_t W = 0;
        if (real) {
            if (k < a.d2) {
                W = cp[k];
            } else {
                // (M_db S_q)[r][j] = sum_t sum_{k'} c'[t Nq + k'] Neg(s_{q,t})[k'][j]; only k' = (j + p) mod Nq
                // with s_{q,t}[p] != 0 contribute, with sign -1 when j + p wraps past Nq.
                const uint32_t j = k - a.d2;
                for (uint32_t tt = 0; tt < a.nqblk; ++tt) {
                    const int32_t *crow = cp + tt * a.Nq;
                    for (uint32_t c = 0; c < a.h; ++c) {
                        const uint32_t p = (uint32_t)spos[tt * a.h + c];
                        const int s = ssgn[tt * a.h + c];
                        const uint32_t jp = j + p;
                        W += (jp < a.Nq) ? s * crow[jp] : -s * crow[jp - a.Nq];
                    }
                }
            }
        }
        for (uint32_t l = 0; l < a.L; ++l) {
            uint64_t v = 0;
            if (W != 0 && l < a.Lq) {
                const uint64_t m = mulmod_shoup((uint64_t)(W < 0 ? -W : W), a.qp[l], a.qps[l], a.q[l]);
                v = (W < 0 && m) ? a.q[l] - m : m;
            }
            a.db[((size_t)l * a.lay.M + pos) * a.K + k] = v;
        }
    }
}

struct DbEncArgs {
    LayoutDev lay;
    uint32_t K, h, eta, n_blocks;
    uint64_t seed, chunk;
    const int32_t *sdb_pos; const int8_t *sdb_sgn;   // [blocks][h]
    LimbTable lt;
    uint64_t *db;
};

// Pass 2, one block per (column k, limb l): draw the a-part column into shared memory and write
// it, then finish every b-row: B = msg - (s_{db,t} * a)[i] + e (mod q_l).
__global__ void __launch_bounds__(1024) k_db_apart_b(DbEncArgs a) {
    extern __shared__ unsigned char smem[];
    uint64_t *acol = reinterpret_cast<uint64_t *>(smem);                 // [N]
    int32_t *spos = reinterpret_cast<int32_t *>(acol + a.lay.N);         // [n_blocks*h]
    int8_t *ssgn = reinterpret_cast<int8_t *>(spos + a.n_blocks * a.h);

    const uint32_t k = blockIdx.x, l = blockIdx.y, N = a.lay.N;
    const uint64_t q = a.lt.q[l];
    const uint64_t ka = stream_key(a.seed, ICM_KIND_A_DB, a.chunk, l);
    const uint64_t ke = stream_key(a.seed, ICM_KIND_E_DB, a.chunk, 0);
    uint64_t *dbl = a.db + (size_t)l * a.lay.M * a.K;
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
        const uint64_t v = uniform_mod(sm64(ka, (uint64_t)i * a.K + k), q);
        acol[i] = v;
        dbl[(size_t)i * a.K + k] = to_digit_form(v, q);
    }
    for (uint32_t x = threadIdx.x; x < a.n_blocks * a.h; x += blockDim.x) { spos[x] = a.sdb_pos[x]; ssgn[x] = a.sdb_sgn[x]; }
    __syncthreads();

    const uint64_t nb = a.lay.M - N;
    for (uint64_t bidx = threadIdx.x; bidx < nb; bidx += blockDim.x) {
        uint32_t t, i;
        b_row_of(a.lay, bidx, t, i);
        const uint64_t r = (uint64_t)t * N + i;
        uint64_t sa = 0;       // (s_{db,t} * a)[i] mod q
        for (uint32_t c = 0; c < a.h; ++c) {
            const uint32_t p = (uint32_t)spos[t * a.h + c];
            const int s = ssgn[t * a.h + c];
            // X^p * X^(i-p): wraps with a sign flip when i < p
            const uint64_t term = (i >= p) ? acol[i - p] : acol[N + i - p];
            const bool neg = (i >= p) ? (s < 0) : (s > 0);
            sa = neg ? sub_mod(sa, term, q) : add_mod(sa, term, q);
        }
        uint64_t *dst = dbl + (size_t)(N + bidx) * a.K + k;
        const int e = cbd_sample(sm64(ke, r * a.K + k), a.eta);
        uint64_t v = sub_mod(*dst, sa, q);
        v = e >= 0 ? add_mod(v, (uint64_t)e, q) : sub_mod(v, (uint64_t)(-e), q);
        *dst = to_digit_form(v, q);
    }
}

struct QEncArgs {
    uint32_t K, d2, Nq, h, eta, rho, code_bits, Lq, nqblk;
    uint64_t seed;
    const uint8_t *codes, *masks;        // [n_eyes][code_bits/8]
    const uint64_t *eye_ids;
    const int32_t *sq_pos; const int8_t *sq_sgn;
    uint64_t q[ICM_MAX_LIMBS], dl[ICM_MAX_LIMBS];   // primes and Delta mod q_l
    uint32_t n_cols;
    uint64_t *ct;                        // [Lq][n_cols][K]
};

// One block per (query column j, limb l < Lq).
__global__ void __launch_bounds__(1024) k_query_encrypt(QEncArgs a) {
    extern __shared__ unsigned char smem[];
    uint64_t *acol = reinterpret_cast<uint64_t *>(smem);           // [Nq]
    int8_t *cp = reinterpret_cast<int8_t *>(acol + a.Nq);          // [d2]
    const uint32_t j = blockIdx.x, l = blockIdx.y;
    const uint32_t e = j / a.rho, r = j % a.rho;
    const int shift = (int)r - (int)(a.rho - 1) / 2;
    const uint64_t q = a.q[l];
    const uint64_t eid = a.eye_ids[e];
    const uint64_t ka = stream_key(a.seed, ICM_KIND_A_Q, eid, l);
    const uint64_t ke = stream_key(a.seed, ICM_KIND_E_Q, eid, 0);
    uint64_t *col = a.ct + ((size_t)l * a.n_cols + j) * a.K;
    const uint32_t tb = a.code_bits / 8;
    const uint8_t *cd = a.codes + (size_t)e * tb, *mk = a.masks + (size_t)e * tb;
    // rotated masked bit-vector: x_s[row, col, b] = x[row, (col + s) mod 200, b] on 16 x 200 x 4
    for (uint32_t k = threadIdx.x; k < a.d2; k += blockDim.x) {
        int v = 0;
        if (k < a.code_bits) {
            const uint32_t row = k / 800, cc = (k / 4) % 200, b = k % 4;
            const uint32_t src_col = (uint32_t)(((int)cc + shift + 200) % 200);
            const uint32_t src = (row * 200 + src_col) * 4 + b;
            const int c = template_bit(cd, src), m = template_bit(mk, src);
            v = m - 2 * (c & m);
        }
        cp[k] = (int8_t)v;
    }
    for (uint32_t i = threadIdx.x; i < a.Nq; i += blockDim.x) {
        const uint64_t v = uniform_mod(sm64(ka, (uint64_t)r * a.Nq + i), q);
        acol[i] = v;
        col[a.d2 + i] = v;
    }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < a.d2; k += blockDim.x) {
        const uint32_t t = k / a.Nq, i = k % a.Nq;
        uint64_t sa = 0;
        for (uint32_t c = 0; c < a.h; ++c) {
            const uint32_t p = (uint32_t)a.sq_pos[t * a.h + c];
            const int s = a.sq_sgn[t * a.h + c];
            const uint64_t term = (i >= p) ? acol[i - p] : acol[a.Nq + i - p];
            const bool neg = (i >= p) ? (s < 0) : (s > 0);
            sa = neg ? sub_mod(sa, term, q) : add_mod(sa, term, q);
        }
        uint64_t v = sa ? q - sa : 0;                          // -(s * a)
        const int m = cp[k];
        if (m > 0) v = add_mod(v, a.dl[l], q);
        else if (m < 0) v = sub_mod(v, a.dl[l], q);
        const int err = cbd_sample(sm64(ke, (uint64_t)r * a.d2 + k), a.eta);
        v = err >= 0 ? add_mod(v, (uint64_t)err, q) : sub_mod(v, (uint64_t)(-err), q);
        col[k] = v;
    }
}

}  // namespace

namespace icm {

cudaError_t launch_db_messages(const icm_ctx *c, const LayoutDev &lay, const uint8_t *d_codes,
                               const uint8_t *d_masks, uint64_t *d_db, cudaStream_t st, const int32_t *d_wmsg) {
    DbMsgArgs a{};
    a.lay = lay;
    a.K = c->K; a.d2 = c->p.d2; a.Nq = c->N_q; a.nqblk = c->n_qblk; a.h = c->p.hamming_weight;
    a.code_bits = c->p.code_bits; a.L = c->p.n_limbs; a.Lq = c->p.n_limbs_q;
    a.codes = d_codes; a.masks = d_masks; a.wmsg = d_wmsg;
    a.sq_pos = c->d_sq_pos; a.sq_sgn = c->d_sq_sgn;
    for (uint32_t l = 0; l < a.L; ++l) { a.qp[l] = c->qp_mod[l]; a.qps[l] = c->qp_mods[l]; a.q[l] = c->q[l]; }
    a.db = d_db;
    const uint64_t nb = lay.M - lay.N;
    if (nb == 0) return cudaSuccess;
    const size_t smem = (size_t)((a.d2 + 3) & ~3u) * 4 + (size_t)a.nqblk * a.h * 5;
    cudaError_t e = cudaFuncSetAttribute(k_db_messages, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_db_messages<<<(unsigned)nb, 512, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_db_apart_and_b(const icm_ctx *c, const LayoutDev &lay, uint64_t chunk_id, uint64_t *d_db,
                                  cudaStream_t st) {
    DbEncArgs a{};
    a.lay = lay; a.K = c->K; a.h = c->p.hamming_weight; a.eta = c->p.noise_eta;
    a.n_blocks = (uint32_t)((lay.M - lay.N) ? (lay.n_full + (lay.rem ? 1 : 0)) : 0);
    a.seed = c->p.seed; a.chunk = chunk_id;
    a.sdb_pos = c->d_sdb_pos; a.sdb_sgn = c->d_sdb_sgn;
    a.lt = c->lt; a.db = d_db;
    const size_t smem = (size_t)lay.N * 8 + (size_t)a.n_blocks * a.h * 5;
    cudaError_t e = cudaFuncSetAttribute(k_db_apart_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(c->K, c->p.n_limbs);
    k_db_apart_b<<<grid, 1024, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_query_encrypt(const icm_ctx *c, const uint8_t *d_codes, const uint8_t *d_masks,
                                 const uint64_t *d_eye_ids, uint32_t n_eyes, uint64_t *d_ct, cudaStream_t st) {
    QEncArgs a{};
    a.K = c->K; a.d2 = c->p.d2; a.Nq = c->N_q; a.h = c->p.hamming_weight; a.eta = c->p.noise_eta;
    a.rho = c->p.rho; a.code_bits = c->p.code_bits; a.Lq = c->p.n_limbs_q; a.nqblk = c->n_qblk;
    a.seed = c->p.seed; a.codes = d_codes; a.masks = d_masks; a.eye_ids = d_eye_ids;
    a.sq_pos = c->d_sq_pos; a.sq_sgn = c->d_sq_sgn;
    for (uint32_t l = 0; l < a.Lq; ++l) { a.q[l] = c->q[l]; a.dl[l] = c->delta_mod[l]; }
    a.n_cols = n_eyes * c->p.rho;
    a.ct = d_ct;
    if (a.n_cols == 0) return cudaSuccess;
    const size_t smem = (size_t)a.Nq * 8 + a.d2;
    cudaError_t e = cudaFuncSetAttribute(k_query_encrypt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(a.n_cols, a.Lq);
    k_query_encrypt<<<grid, 1024, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace icm
