/*
 * icm_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU restatement of what the encrypted 1:N iris matching hot
 * path computes (arxiv 2601.17561, "Private Iris Recognition with High-Performance FHE").
 * Only tests/, the smoke check and the benchmark's CPU-baseline leg may load this file.  It
 * shares no code, header, table or constant generator with the CUDA library; the two meet only
 * through the packed iris templates that the synthetic-input module hands to both.
 *
 * Integer arithmetic is exact (u64 residues, __int128 accumulation).  Every loop follows the
 * definition it cites, with no blocking, fusion or reordering beyond what that definition
 * states.  OpenMP only splits independent outputs across threads.
 *
 * Randomness (Section 2.2.2 defers key generation and encryption to the original CKKS paper):
 *   counter-based SplitMix64 (Steele, Lea and Flood, OOPSLA 2014; public-domain reference
 *   splitmix64.c by S. Vigna): output i of the stream seeded with s is mix(s + (i+1) * gamma).
 *   Stream keys are derived as key(seed, kind, a, b) = sm(sm(sm(seed, kind), a), b).
 *   Uniform residue mod q from a 64-bit word w: floor(w * q / 2^64) (Lemire's multiply-shift
 *   range reduction, without the rejection step).  Noise: centred binomial with eta = 21 from
 *   one word.  Secret: ternary with exactly h non-zeros at uniform positions.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;
typedef __int128 i128;

#define GAMMA 0x9E3779B97F4A7C15ULL

enum { KIND_SK_DB = 1, KIND_SK_Q = 2, KIND_A_DB = 3, KIND_E_DB = 4, KIND_A_Q = 5, KIND_E_Q = 6 };

/* ---------------------------------------------------------------- generator ---- */

static uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Output i (0-based) of SplitMix64 seeded with `seed`. */
uint64_t orc_sm64(uint64_t seed, uint64_t i) { return sm_mix(seed + (i + 1) * GAMMA); }

uint64_t orc_stream_key(uint64_t seed, uint64_t kind, uint64_t a, uint64_t b) {
    return orc_sm64(orc_sm64(orc_sm64(seed, kind), a), b);
}

uint64_t orc_uniform_mod(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w * q) >> 64); }

static int popc64(uint64_t x) { return __builtin_popcountll(x); }

/* Centred binomial: popcount of eta bits minus popcount of the next eta bits. */
int orc_cbd(uint64_t w, int eta) {
    uint64_t m = (eta >= 64) ? ~0ULL : ((1ULL << eta) - 1);
    return popc64(w & m) - popc64((w >> eta) & m);
}

/* Ternary secret of degree n with exactly h non-zero coefficients: draw positions
 * floor(w * n / 2^64) from the stream in order, skip positions already taken, sign from the
 * lowest bit of the same word (1 -> -1). */
void orc_secret(uint64_t key, int n, int h, int8_t *s) {
    memset(s, 0, (size_t)n);
    int cnt = 0;
    for (uint64_t j = 0; cnt < h; ++j) {
        uint64_t w = orc_sm64(key, j);
        uint64_t pos = (uint64_t)(((u128)w * (uint64_t)n) >> 64);
        if (s[pos] == 0) { s[pos] = (w & 1) ? -1 : 1; ++cnt; }
    }
}

/* ---------------------------------------------------------------- modular helpers ---- */

static uint64_t mod_i128(i128 x, uint64_t q) {
    i128 r = x % (i128)q;
    if (r < 0) r += q;
    return (uint64_t)r;
}

static uint64_t pow2_mod(unsigned e, uint64_t q) {
    uint64_t r = 1 % q;
    for (unsigned i = 0; i < e; ++i) r = (uint64_t)(((u128)r * 2) % q);
    return r;
}

/* Non-zero positions of a sparse ternary secret, in increasing order (sums over them skip
 * only zero terms). */
typedef struct { int h; int *pos; int8_t *sgn; } support;

static support support_of(const int8_t *s, int n) {
    support sp; sp.h = 0;
    for (int p = 0; p < n; ++p) sp.h += (s[p] != 0);
    sp.pos = (int *)malloc(sizeof(int) * (size_t)(sp.h ? sp.h : 1));
    sp.sgn = (int8_t *)malloc((size_t)(sp.h ? sp.h : 1));
    int c = 0;
    for (int p = 0; p < n; ++p) if (s[p]) { sp.pos[c] = p; sp.sgn[c] = s[p]; ++c; }
    return sp;
}
static void support_free(support *sp) { free(sp->pos); free(sp->sgn); }

/* Coefficient i of s * a in Z_q[X]/(X^n + 1) (Section 2.2.1 plaintext ring) for a sparse
 * ternary s: the product of X^p and X^(i-p) wraps with a sign flip when i - p < 0. */
static uint64_t negacyclic_coeff(const support *s, const uint64_t *a, int n, int i, uint64_t q) {
    i128 acc = 0;
    for (int c = 0; c < s->h; ++c) {
        const int p = s->pos[c];
        i128 term = (i >= p) ? (i128)a[i - p] : -(i128)a[n + i - p];
        acc += (s->sgn[c] > 0) ? term : -term;
    }
    return mod_i128(acc, q);
}

/* Full product s * a in Z_q[X]/(X^n + 1), coefficient by coefficient (exposed for tests). */
void orc_negacyclic_mul(const int8_t *s, const uint64_t *a, int n, uint64_t q, uint64_t *out) {
    support sp = support_of(s, n);
    for (int i = 0; i < n; ++i) out[i] = negacyclic_coeff(&sp, a, n, i, q);
    support_free(&sp);
}

/* Product of two polynomials of Z_q[X]/(X^n + 1) (Section 2.2.1 plaintext ring), schoolbook:
 * out[k] = sum_{i + j = k} a_i b_j - sum_{i + j = k + n} a_i b_j  (mod q), inputs in [0, q), q < 2^62.
 * The u128 partial sums are reduced every 16 products (16 * 2^124 = 2^128). */
void orc_negacyclic_mulmod(const uint64_t *a, const uint64_t *b, int n, uint64_t q, uint64_t *out) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n; ++k) {
        u128 pos = 0, neg = 0;
        int cnt = 0;
        for (int i = 0; i <= k; ++i) {
            pos += (u128)a[i] * b[k - i];
            if (++cnt == 16) { pos %= q; cnt = 0; }
        }
        cnt = 0;
        for (int i = k + 1; i < n; ++i) {
            neg += (u128)a[i] * b[n + k - i];
            if (++cnt == 16) { neg %= q; cnt = 0; }
        }
        const uint64_t p = (uint64_t)(pos % q), m = (uint64_t)(neg % q);
        out[k] = p >= m ? p - m : p + q - m;
    }
}

/* ---------------------------------------------------------------- encryption ---- */

/* MSRLWE query encryption under S_q modulo Q = q_0 ... q_{Lq-1} (Section 2.3 shared-a format,
 * Section 2.2.2 Dec(a, b) = a*sk + b): for query column j (eye e = j / rho, rotation
 * r = j % rho) and block t < d2/nq,
 *     b_{t,j} = -(s_{q,t} * a_j) + Delta * c'_j[t*nq : (t+1)*nq] + e_{t,j}   (mod q_l),
 * with a_j uniform mod Q.  Output layout [Lq][d3][d2 + nq]: column j holds b (d2 values) then
 * a (nq values). */
int orc_query_encrypt(int Lq, const uint64_t *q, int nq, int d2, int h, int eta, unsigned log2_delta,
                      uint64_t seed, int n_eyes, int rho, const uint64_t *eye_ids,
                      const int8_t *cprime /* [d3][d2] */, uint64_t *out) {
    if (d2 % nq) return -1;
    const int nblk = d2 / nq, d3 = n_eyes * rho, K = d2 + nq;
    int8_t *sq = (int8_t *)malloc((size_t)nblk * nq);
    support *sqs = (support *)malloc(sizeof(support) * (size_t)nblk);
    for (int t = 0; t < nblk; ++t) {
        orc_secret(orc_stream_key(seed, KIND_SK_Q, (uint64_t)t, 0), nq, h, sq + (size_t)t * nq);
        sqs[t] = support_of(sq + (size_t)t * nq, nq);
    }
    for (int l = 0; l < Lq; ++l) {
        const uint64_t ql = q[l], delta = pow2_mod(log2_delta, ql);
#pragma omp parallel for schedule(dynamic)
        for (int j = 0; j < d3; ++j) {
            const int e = j / rho, r = j % rho;
            uint64_t *col = out + ((size_t)l * d3 + j) * K;
            const uint64_t ka = orc_stream_key(seed, KIND_A_Q, eye_ids[e], (uint64_t)l);
            const uint64_t ke = orc_stream_key(seed, KIND_E_Q, eye_ids[e], 0);
            uint64_t *a = col + d2;
            for (int i = 0; i < nq; ++i) a[i] = orc_uniform_mod(orc_sm64(ka, (uint64_t)r * nq + i), ql);
            for (int t = 0; t < nblk; ++t)
                for (int i = 0; i < nq; ++i) {
                    const int k = t * nq + i;
                    const uint64_t sa = negacyclic_coeff(&sqs[t], a, nq, i, ql);
                    const int m = cprime[(size_t)j * d2 + k];
                    const int err = orc_cbd(orc_sm64(ke, (uint64_t)r * d2 + k), eta);
                    i128 v = -(i128)sa + (i128)m * (i128)delta + err;
                    col[k] = mod_i128(v, ql);
                }
        }
    }
    for (int t = 0; t < nblk; ++t) support_free(&sqs[t]);
    free(sqs); free(sq);
    return 0;
}

/* Basis extension of the query (first step of CCMM, Section 2.3): lift every residue vector
 * mod Q to its centred representative in (-Q/2, Q/2] and reduce it modulo every q_l.  Exact for
 * Q < 2^127 (Lq <= 2 primes below 2^63).  in: [Lq][n], out: [L][n]. */
int orc_query_extend(int L, int Lq, const uint64_t *q, size_t n, const uint64_t *in, uint64_t *out) {
    if (Lq < 1 || Lq > 2) return -1;
    u128 Q = q[0];
    uint64_t inv = 0;
    if (Lq == 2) {
        Q *= q[1];
        /* inverse of q0 modulo q1 by Fermat (q1 prime) */
        uint64_t b = q[0] % q[1], e = q[1] - 2, r = 1;
        while (e) { if (e & 1) r = (uint64_t)(((u128)r * b) % q[1]); b = (uint64_t)(((u128)b * b) % q[1]); e >>= 1; }
        inv = r;
    }
#pragma omp parallel for
    for (size_t i = 0; i < n; ++i) {
        u128 x = in[i];
        if (Lq == 2) {
            uint64_t r0 = in[i], r1 = in[n + i];
            uint64_t d = (uint64_t)(((u128)((r1 + q[1] - r0 % q[1]) % q[1]) * inv) % q[1]);
            x = (u128)r0 + (u128)q[0] * d;
        }
        i128 xc = (x > (Q - 1) / 2) ? (i128)x - (i128)Q : (i128)x;
        for (int l = 0; l < L; ++l) out[(size_t)l * n + i] = mod_i128(xc, q[l]);
    }
    return 0;
}

/* Rows of one database chunk in MSRLWE-RGSW form (Section 6.2.1: encryptions of M_db and of
 * M_db * S_q under S_db, modulus Q_db = Q * Q'; gadget factor Q' so that the query's
 * wrap-around multiple of Q vanishes modulo Q_db).  With K = d2 + nq:
 *   a-part row i < ndb:  [A1 A2][i][k] uniform mod Q_db (independent residues per limb);
 *   b-row r (block t = r / ndb, coefficient i = r % ndb):
 *        B[r][k] = -(s_{db,t} * A[:, k])[i] + Q' * W[r][k] + E[r][k]    (mod q_l)
 *   with W[r][k] = m_r[k] for k < d2 and W[r][d2 + j] = (M_db S_q)[r][j], where m_r is row r
 *   of the database message matrix: the masked bit-vector c'_r of template r (coefficient
 *   encoding, Section 2.1.3) or the rounded slot-encoding coefficients of a block of templates
 *   (Section 2.2.1 Ecd_slot, built by oracle/slots.py).
 * row_ids: values < ndb select a-part rows, ndb + r selects logical b-row r.
 * msg: [n_rows][d2] message rows of the selected b-rows (zero rows for padding and for a-part
 * rows), |m| < 2^21.  out: [L][n_rows][K]. */
int orc_db_rows(int L, int Lq, const uint64_t *q, int ndb, int nq, int d2, int h, int eta,
                uint64_t seed, uint64_t chunk, const int64_t *row_ids, int n_rows,
                const int32_t *msg, uint64_t *out) {
    if (d2 % nq) return -1;
    const int K = d2 + nq, nqb = d2 / nq;
    int max_blk = 0;
    for (int x = 0; x < n_rows; ++x)
        if (row_ids[x] >= ndb) { int t = (int)((row_ids[x] - ndb) / ndb); if (t + 1 > max_blk) max_blk = t + 1; }
    int8_t *sdb = (int8_t *)calloc((size_t)(max_blk ? max_blk : 1) * ndb, 1);
    int8_t *sq = (int8_t *)malloc((size_t)nqb * nq);
    support *sdbs = (support *)malloc(sizeof(support) * (size_t)(max_blk ? max_blk : 1));
    support *sqs = (support *)malloc(sizeof(support) * (size_t)nqb);
    for (int t = 0; t < max_blk; ++t) {
        orc_secret(orc_stream_key(seed, KIND_SK_DB, (uint64_t)t, 0), ndb, h, sdb + (size_t)t * ndb);
        sdbs[t] = support_of(sdb + (size_t)t * ndb, ndb);
    }
    for (int t = 0; t < nqb; ++t) {
        orc_secret(orc_stream_key(seed, KIND_SK_Q, (uint64_t)t, 0), nq, h, sq + (size_t)t * nq);
        sqs[t] = support_of(sq + (size_t)t * nq, nq);
    }

    /* W[x][k] for every selected row: the message matrix [M_db | M_db S_q]. */
    int32_t *W = (int32_t *)calloc((size_t)n_rows * K, sizeof(int32_t));
#pragma omp parallel for schedule(dynamic)
    for (int x = 0; x < n_rows; ++x) {
        if (row_ids[x] < ndb) continue;
        const int32_t *c = msg + (size_t)x * d2;
        int32_t *w = W + (size_t)x * K;
        for (int k = 0; k < d2; ++k) w[k] = c[k];
        /* (M_db S_q)[r][j] = sum_k' c'[t*nq + k'] * Neg(s_{q,t})[k'][j] summed over the blocks t of
         * S_q (vertical stack of Neg(s_{q,t})), where Neg(s)[k'][j] = s[k'-j] if k' >= j else
         * -s[nq+k'-j].  Only k' = (j + p) mod nq with s[p] != 0 give non-zero terms. */
        for (int j = 0; j < nq; ++j) {
            long acc = 0;
            for (int t = 0; t < nqb; ++t)
                for (int cidx = 0; cidx < sqs[t].h; ++cidx) {
                    const int p = sqs[t].pos[cidx];
                    const int kp = (j + p < nq) ? j + p : j + p - nq;
                    const int sv = (kp >= j) ? sqs[t].sgn[cidx] : -sqs[t].sgn[cidx];
                    acc += (long)sv * c[t * nq + kp];
                }
            w[d2 + j] = (int32_t)acc;
        }
    }

    const uint64_t ke = orc_stream_key(seed, KIND_E_DB, chunk, 0);
    for (int l = 0; l < L; ++l) {
        const uint64_t ql = q[l];
        uint64_t qp = 1 % ql;                       /* Q' mod q_l */
        for (int l2 = Lq; l2 < L; ++l2) qp = (uint64_t)(((u128)qp * (q[l2] % ql)) % ql);
        const uint64_t ka = orc_stream_key(seed, KIND_A_DB, chunk, (uint64_t)l);
#pragma omp parallel
        {
            uint64_t *acol = (uint64_t *)malloc((size_t)ndb * sizeof(uint64_t));
#pragma omp for schedule(dynamic, 16)
            for (int k = 0; k < K; ++k) {
                for (int i = 0; i < ndb; ++i) acol[i] = orc_uniform_mod(orc_sm64(ka, (uint64_t)i * K + k), ql);
                for (int x = 0; x < n_rows; ++x) {
                    uint64_t *dst = out + ((size_t)l * n_rows + x) * K + k;
                    if (row_ids[x] < ndb) { *dst = acol[row_ids[x]]; continue; }
                    const int64_t r = row_ids[x] - ndb;
                    const int t = (int)(r / ndb), i = (int)(r % ndb);
                    const uint64_t sa = negacyclic_coeff(&sdbs[t], acol, ndb, i, ql);
                    const int err = orc_cbd(orc_sm64(ke, (uint64_t)r * K + k), eta);
                    i128 v = -(i128)sa + (i128)qp * W[(size_t)x * K + k] + err;
                    *dst = mod_i128(v, ql);
                }
            }
            free(acol);
        }
    }
    for (int t = 0; t < max_blk; ++t) support_free(&sdbs[t]);
    for (int t = 0; t < nqb; ++t) support_free(&sqs[t]);
    free(sdbs); free(sqs);
    free(W); free(sq); free(sdb);
    return 0;
}

/* ---------------------------------------------------------------- CCMM ---- */

/* Plaintext modular matrix product (Section 2.3: CCMM is dominated by plaintext products
 * modulo the ciphertext modulus), per RNS limb:
 *     C[l][j][i] = sum_k A[l][i][k] * B[l][j][k]  mod q_l
 * A: [L][M][K], B: [L][N][K] (both K-contiguous), C: [L][N][M].  Exact: the u128 accumulator is
 * reduced every 64 products (64 * 2^126 < 2^128 for q < 2^63). */
void orc_ppmm(int L, const uint64_t *q, int M, int N, int K, const uint64_t *A, const uint64_t *B, uint64_t *C) {
    for (int l = 0; l < L; ++l) {
        const uint64_t ql = q[l];
#pragma omp parallel for collapse(2) schedule(static)
        for (int j = 0; j < N; ++j)
            for (int i = 0; i < M; ++i) {
                const uint64_t *a = A + ((size_t)l * M + i) * K, *b = B + ((size_t)l * N + j) * K;
                u128 acc = 0;
                for (int k = 0; k < K; ++k) {
                    acc += (u128)a[k] * b[k];
                    if ((k & 63) == 63) acc %= ql;
                }
                C[((size_t)l * N + j) * M + i] = (uint64_t)(acc % ql);
            }
    }
}

/* ---------------------------------------------------------------- decryption ---- */

/* Decryption of the b-rows of one result column (Section 2.2.2: Dec(a, b) = a*sk + b, block by
 * block of the MSRLWE result): for selected logical b-row r (block t, coefficient i)
 *     D[l][x] = Cb[l][x] + (s_{db,t} * Ca[l])[i]   (mod q_l).
 * Ca: [L][ndb] a-part polynomial of the column, Cb: [L][n_rows], D: [L][n_rows]. */
void orc_decrypt_rows(int L, const uint64_t *q, int ndb, int h, uint64_t seed, const int64_t *b_rows, int n_rows,
                      const uint64_t *Ca, const uint64_t *Cb, uint64_t *D) {
    int max_blk = 0;
    for (int x = 0; x < n_rows; ++x) { int t = (int)(b_rows[x] / ndb); if (t + 1 > max_blk) max_blk = t + 1; }
    int8_t *sdb = (int8_t *)calloc((size_t)(max_blk ? max_blk : 1) * ndb, 1);
    support *sdbs = (support *)malloc(sizeof(support) * (size_t)(max_blk ? max_blk : 1));
    for (int t = 0; t < max_blk; ++t) {
        orc_secret(orc_stream_key(seed, KIND_SK_DB, (uint64_t)t, 0), ndb, h, sdb + (size_t)t * ndb);
        sdbs[t] = support_of(sdb + (size_t)t * ndb, ndb);
    }
    for (int l = 0; l < L; ++l)
#pragma omp parallel for
        for (int x = 0; x < n_rows; ++x) {
            const int t = (int)(b_rows[x] / ndb), i = (int)(b_rows[x] % ndb);
            const uint64_t sa = negacyclic_coeff(&sdbs[t], Ca + (size_t)l * ndb, ndb, i, q[l]);
            D[(size_t)l * n_rows + x] = (uint64_t)(((u128)Cb[(size_t)l * n_rows + x] + sa) % q[l]);
        }
    for (int t = 0; t < max_blk; ++t) support_free(&sdbs[t]);
    free(sdbs); free(sdb);
}

/* ---------------------------------------------------------------- cleartext ---- */

/* Fractional Hamming distance ingredients (Section 2.1.1, Eq. (1)) on packed 64-bit words:
 *   num[a][b] = <c_a XOR c_b, m_a AND m_b>,  den[a][b] = ||m_a AND m_b||_1.
 * qc, qm: [na][words], dc, dm: [nb][words]; outputs [na][nb]. */
void orc_hd_counts(int na, int nb, int words, const uint64_t *qc, const uint64_t *qm,
                   const uint64_t *dc, const uint64_t *dm, int32_t *num, int32_t *den) {
#pragma omp parallel for collapse(2) schedule(static)
    for (int a = 0; a < na; ++a)
        for (int b = 0; b < nb; ++b) {
            int n = 0, d = 0;
            for (int w = 0; w < words; ++w) {
                const uint64_t mm = qm[(size_t)a * words + w] & dm[(size_t)b * words + w];
                n += popc64((qc[(size_t)a * words + w] ^ dc[(size_t)b * words + w]) & mm);
                d += popc64(mm);
            }
            num[(size_t)a * nb + b] = n;
            den[(size_t)a * nb + b] = d;
        }
}

int orc_omp_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
