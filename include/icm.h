/*
 * icm.h -- C ABI of the GB300-native encrypted 1:N iris matching library (libicm.so).
 *
 * The library computes the data-parallel core of CKKS-encrypted iris matching from
 * arxiv 2601.17561 ("Private Iris Recognition with High-Performance FHE"): encryption of an
 * iris database in MSRLWE-RGSW form and of query eyes in MSRLWE form, the ciphertext x
 * ciphertext matrix product (CCMM) as modular matrix products over the RNS limbs, the
 * linear (key-free) fold of Algorithm 2, and decryption for checking.
 *
 * Conventions shared by every call
 *  - Pointers named dev_* are CUDA device pointers owned by the caller; host_* / plain pointers
 *    are host memory owned by the caller.  Sizes are in bytes unless named n_* (counts).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls that
 *    take a stream only enqueue work: they return ICM_OK once the work is enqueued, and the
 *    caller synchronises the stream (or calls icm_sync) before reading results.
 *  - Every call returns an icm_status.  On error, out-parameters are left untouched, nothing is
 *    allocated and no work is enqueued; icm_last_error() gives a one-line reason (per thread).
 *    No call aborts, traps or waits without a bound.
 *  - Handles (icm_ctx, icm_db, icm_query, icm_scores) are owned by the library until the
 *    matching *_destroy call.  icm_db / icm_query / icm_scores only describe caller-owned device
 *    buffers; destroying a handle never frees caller memory.  A context must outlive the
 *    handles made from it.  Handles are immutable after creation and may be shared across
 *    streams; icm_ctx_create/icm_keygen are not thread-safe on the same context.
 *
 * Data layouts (u64 residues are canonical, in [0, q_l), unless stated otherwise)
 *  - Templates: `code_bits / 8` bytes per code and per mask, bit b at byte b/8, bit b%8.
 *  - Database chunk: [L][M][K] u64 words, K = d2 + N_q, M = N_db + (stored b-rows).  Each word holds
 *    the residue in balanced-digit form: its bytes (two's complement) are the digits d_t in
 *    [-128, 127] of the centred lift c = sum_t d_t 256^t (c = (word ^ 0x80..80) - 0x80..80).  Row order: the
 *    N_db a-part rows, then the b-rows of every full block, then for a partial last block its
 *    real rows followed by the wrap-around tail coefficients [max(n_t, N_db - rho + 1), N_db)
 *    (encryptions of zero that the fold's negacyclic shift reads).
 *  - Query ciphertext (wire format, modulo Q): [L_q][d3][K] u64, d3 = n_eyes * rho, column
 *    j = eye * rho + rotation holds b (d2 values) then a (N_q values).
 *  - Scores: [L][n_cols][M] u64 (column-major: one result column contiguous, same row order as
 *    the database chunk).  Folded scores: n_cols = n_eyes * ceil(rho / fold_k).
 */
#ifndef ICM_H
#define ICM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ICM_OK = 0,
    ICM_EINVAL = 1,        /* bad argument, size or layout                                     */
    ICM_ENOMEM = 2,        /* host allocation failed, or caller buffer too small              */
    ICM_ECUDA = 3,         /* a CUDA runtime call failed                                      */
    ICM_ETIMEOUT = 4,      /* a bounded wait (host or device) ran out                          */
    ICM_EBOUND = 5,        /* a noise, decoding or accumulator-overflow inequality fails      */
    ICM_EUNSUPPORTED = 6   /* valid request that this build does not implement                */
} icm_status;

/* Arithmetic form of the modular matrix products (Section 6.2.2 reduces them to int8 GEMMs;
 * on sm_103a the forms below are the exact variants this library implements). */
typedef enum {
    ICM_FORM_U64 = 0,        /* u64 residues on CUDA cores, exact 160-bit lazy accumulation   */
    ICM_FORM_I8_DIGITS = 1,  /* 8 signed balanced base-256 digits per residue, int8 tensor-core
                                products per digit pair, int32 accumulation, fused recombination */
    ICM_FORM_I8_CRT = 2,     /* residues split over small pairwise-coprime moduli (<= 256),
                                int8 tensor-core product per modulus, exact CRT back mod q_l  */
    ICM_FORM_F16_CRT = 3,    /* small-modulus residues as exact fp16 integers on fp16 tensor
                                cores, fp32 accumulation reduced modulo m_i before it reaches
                                2^24, residues recombined by CRT in a second pass             */
    ICM_FORM_I8_P2 = 4       /* icm_ppmm only: the paper's own modulus family (Section 6.2.2,
                                Q = prod p^2 over primes 127 <= p <= 253), every modulus q_l = p_l^2
                                with odd p_l <= 253; residues split as x = x0 + p x1 into centred
                                base-p digits, x y = x0 y0 + p (x0 y1 + x1 y0) mod p^2: two int8
                                tensor-core passes (K, then 2K in one accumulator) per modulus */
} icm_form;

typedef struct icm_ctx icm_ctx;
typedef struct icm_db icm_db;
typedef struct icm_query icm_query;
typedef struct icm_scores icm_scores;

/* Parameters (Section 2.3 CCMM shapes; Section 6.2.1 ring degrees N_db = 2^14, N_q = 2^13 and
 * d = 2^14; Table 3 (computing parameters) secret Hamming weight h = 512). */
typedef struct {
    uint32_t log_n_db;        /* ring degree of the database encryption, N_db = 2^log_n_db     */
    uint32_t log_n_q;         /* ring degree of the query encryption,   N_q  = 2^log_n_q       */
    uint32_t n_limbs;         /* L: RNS primes of the database modulus Q_db = q_0 ... q_{L-1}   */
    uint32_t n_limbs_q;       /* L_q: the first L_q primes form the query modulus Q (1 or 2)   */
    uint32_t prime_bits;      /* every prime is below 2^prime_bits (30..60)                     */
    uint32_t code_bits;       /* iris code length, 12800 (16 x 200 x 4 layout)                 */
    uint32_t d2;              /* padded code length, a multiple of N_q                         */
    uint32_t rho;             /* rotations per eye (odd), shifts -(rho-1)/2 .. (rho-1)/2        */
    uint32_t fold_k;          /* fold group size k of Algorithm 2                               */
    uint32_t hamming_weight;  /* h: non-zeros of every sparse ternary secret                    */
    uint32_t log2_delta;      /* query scaling factor Delta = 2^log2_delta                     */
    uint32_t noise_eta;       /* centred-binomial noise parameter (sigma^2 = eta / 2)           */
    uint64_t seed;            /* master seed of every random stream                            */
} icm_params;

/* One-line description of a status code (static storage). */
const char *icm_status_str(icm_status s);
/* Reason for the last error returned on the calling thread ("" if none). */
const char *icm_last_error(void);

/* Create a context: validates the parameters, picks the RNS primes (the n_limbs largest
 * primes below 2^prime_bits that are 1 mod 2^17, decreasing), and checks the noise and exact
 * decoding inequalities of the CCMM result (ICM_EBOUND if they fail).  No device work. */
icm_status icm_ctx_create(const icm_params *p, icm_ctx **out);
void icm_ctx_destroy(icm_ctx *ctx);
/* Copy the primes (n >= n_limbs values) to host memory. */
icm_status icm_ctx_primes(const icm_ctx *ctx, uint64_t *primes, size_t n);
/* The small moduli of the CRT forms (Section 6.2.2's RNS of moduli below 2^8): the largest
 * pairwise-coprime odd integers below 256, as many as make their product exceed
 * 2^3 K ((q_max - 1)/2)^2 (18 for primes below 2^60 at K = 24,576).  *n_moduli receives their
 * count r (the tensor-core products per modular multiply-add), and the first min(cap, r) moduli
 * go to `moduli` (host array, may be NULL with cap 0).  ICM_EBOUND if the CRT forms are
 * unavailable for this context's primes and K. */
icm_status icm_ctx_crt_moduli(const icm_ctx *ctx, int32_t *moduli, size_t cap, size_t *n_moduli);

/* Key generation (Section 2.2.2 refers to the CKKS paper): samples the database secrets
 * s_{db,t} (degree N_db) and query secrets s_{q,t} (degree N_q) as sparse ternary polynomials
 * with exactly h non-zeros from the context seed, and uploads their supports to the current
 * device.  Secrets never leave the library. */
icm_status icm_keygen(icm_ctx *ctx);

/* ---------------------------------------------------------------- database (setup) ---- */

/* Bytes of device memory for a database chunk of n_db templates, and its stored row count M. */
icm_status icm_db_bytes(const icm_ctx *ctx, size_t n_db, size_t *bytes, size_t *m_rows);

/* Encrypt one database chunk (Section 6.2.1: MSRLWE-RGSW pair of encryptions of M_db and of
 * M_db * S_q, modulus Q_db = Q * Q', gadget factor Q').  codes/masks: host, n_db templates.
 * chunk_id selects the chunk's own a-part stream.  dev_buf: caller device memory of at least
 * icm_db_bytes bytes, which must stay alive while the handle is used. */
icm_status icm_db_encrypt(icm_ctx *ctx, const uint8_t *codes, const uint8_t *masks, size_t n_db,
                          uint64_t chunk_id, void *dev_buf, size_t bytes, void *stream, icm_db **out);
void icm_db_destroy(icm_db *db);

/* Slot-encoded database chunk (Section 2.2.1 Ecd_slot, Section 2.3: the CCMM takes a slot-encoded
 * database matrix and its results carry the same encoding).  Templates are placed one per slot,
 * in the slot's real part: block t of the chunk (N_db b-rows) holds templates t N_db/2 ..
 * t N_db/2 + N_db/2 - 1 (missing ones are empty slots), so a chunk of n_db templates has
 * ceil(n_db / (N_db/2)) full blocks.  Entry column k of block t is the rounded polynomial
 * round(2^log2_scale P) (round half to even) with P(zeta^(5^j)) = c'_{t N_db/2 + j}[k], computed by
 * fp64 FFT on the device; the rows are then encrypted exactly as icm_db_encrypt does with those
 * integers as the message matrix.  icm_match, icm_rescale and icm_fold accept the handle as any
 * other; icm_decrypt_scores refuses its scores (use icm_normalize + icm_decrypt_slots).
 * log2_scale 1..24, and Delta 2^log2_scale d2 < Q / 4 and h (d2 / N_q)(2^log2_scale + 1) < 2^31
 * (ICM_EBOUND otherwise).  codes/masks: host, n_db >= 1 templates; dev_buf: icm_db_bytes_slots
 * bytes, 16-byte aligned, alive while the handle is used.  Allocates and frees temporary device
 * memory on `stream` (the message matrix, 4 bytes per entry). */
icm_status icm_db_bytes_slots(const icm_ctx *ctx, size_t n_db, size_t *bytes, size_t *m_rows);
icm_status icm_db_encrypt_slots(icm_ctx *ctx, const uint8_t *codes, const uint8_t *masks, size_t n_db,
                                uint32_t log2_scale, uint64_t chunk_id, void *dev_buf, size_t bytes, void *stream,
                                icm_db **out);

/* ---------------------------------------------------------------- query ---- */

/* Bytes of the query ciphertext modulo Q (wire format) for n_eyes eyes. */
icm_status icm_query_ct_bytes(const icm_ctx *ctx, size_t n_eyes, size_t *bytes);

/* Encrypt query eyes (Section 3.1: rho rotated codes per eye; Section 2.1.3 masked bit-vector;
 * MSRLWE under S_q modulo Q with scaling Delta).  codes/masks: host, n_eyes templates;
 * eye_ids: host, one id per eye keying that eye's encryption randomness (an eye encrypted
 * alone or inside a batch gives the same ciphertext columns).  dev_ct: wire format. */
icm_status icm_query_encrypt(icm_ctx *ctx, const uint8_t *codes, const uint8_t *masks,
                             const uint64_t *eye_ids, size_t n_eyes, void *dev_ct, size_t bytes,
                             void *stream);

/* Bytes of the prepared query operand of a form. */
icm_status icm_query_op_bytes(const icm_ctx *ctx, size_t n_eyes, icm_form form, size_t *bytes);

/* Prepare the query operand (first step of CCMM, Section 2.3): lift the ciphertext modulo Q to
 * its centred representative and reduce it modulo every q_l (basis extension), then lay it out
 * for `form` (digit planes or small-modulus residue planes for the tensor-core forms).
 * dev_ct: wire format (device); dev_op: icm_query_op_bytes bytes. */
icm_status icm_query_prepare(icm_ctx *ctx, const void *dev_ct, size_t n_eyes, icm_form form,
                             void *dev_op, size_t bytes, void *stream, icm_query **out);
void icm_query_destroy(icm_query *q);

/* ---------------------------------------------------------------- CCMM / fold ---- */

/* Bytes of the encrypted scores of one chunk for n_eyes eyes (folded != 0: after the fold). */
icm_status icm_scores_bytes(const icm_ctx *ctx, const icm_db *db, size_t n_eyes, int folded, size_t *bytes);

/* Device workspace bytes that icm_match needs for a form (0 for u64 and the int8 forms; the
 * fp16 CRT form keeps one byte per output residue and modulus). */
icm_status icm_match_workspace_bytes(const icm_ctx *ctx, const icm_db *db, size_t n_eyes, icm_form form, size_t *bytes);

/* Kernel launches that icm_match enqueues for n_eyes eyes in `form` on this chunk with the
 * context's current variant: 1 for the u64 and digit forms; for the CRT forms a product launch
 * and a recombination launch per column round (1,024 columns on the tcgen05 kernel, 512 on
 * mma.sync) and per group of limbs (the groups keep the residue scratch within 6 GiB). */
icm_status icm_match_launches(const icm_ctx *ctx, const icm_db *db, size_t n_eyes, icm_form form, size_t *n);

/* CCMM (Section 2.3): C = [A1 A2; B1 B2] * [B_q; A_q] per limb, i.e. the four plaintext modular
 * products fused into one [M x K] x [K x d3] product per RNS limb, in the query's form.  Output
 * bit-identical across forms.  dev_out: icm_scores_bytes(folded = 0); dev_ws:
 * icm_match_workspace_bytes bytes (may be NULL when that is 0). */
icm_status icm_match(icm_ctx *ctx, const icm_db *db, const icm_query *q, void *dev_out, size_t bytes,
                     void *dev_ws, size_t ws_bytes, void *stream, icm_scores **out);

/* Fold (Algorithm 2, linear key-free part): for eye e and group g of fold_k rotations,
 * ct'_{e,g} = sum_{r in g} X^r * ct_{e,r} on the a-part and every b-block polynomial; the shift
 * is the global rotation index r and X^r is the negacyclic monomial shift (keyed slot rotation
 * and the folding polynomial f are outside this library).  Tail rows of a partial block are
 * written as zero.  dev_out: icm_scores_bytes(folded = 1). */
icm_status icm_fold(icm_ctx *ctx, const icm_scores *in, void *dev_out, size_t bytes, void *stream,
                    icm_scores **out);
void icm_scores_destroy(icm_scores *s);

/* Shape of a scores buffer: limbs, columns, rows. */
icm_status icm_scores_shape(const icm_scores *s, size_t *n_limbs, size_t *n_cols, size_t *m_rows);

/* Decrypt for checking only (Section 2.2.2 Dec = a*sk + b, then rounding by Q' * Delta, or by
 * Delta modulo Q for rescaled scores): for every column and every real database row, the integer
 * numerator <c'_db, c'_q> (unfolded scores) or the folded sum of numerators.  dev_num: int64
 * [n_cols][n_db].  Threshold decryption is outside this library. */
icm_status icm_decrypt_scores(icm_ctx *ctx, const icm_scores *s, int64_t *dev_num, size_t n, void *stream);
/* icm_decrypt_scores, and also the largest distance |x - round(x)| between a decoded value x
 * (decrypted coefficient divided by Q' * Delta, or by Delta at the rescaled level) and the
 * integer it rounds to, over all outputs: dev_max_err is one fp32 in device memory, written on
 * `stream`.  It bounds the pre-rounding error of the decoded numerators (the encryption noise plus
 * the decoder's own 128-bit fixed-point error, below 2^-5 units for 60-bit primes); the decoded
 * numerators are exact while it stays below 1/2. */
icm_status icm_decrypt_scores_max_error(icm_ctx *ctx, const icm_scores *s, int64_t *dev_num, size_t n,
                                        float *dev_max_err, void *stream);

/* Normalisation by the inverse mask overlaps (Algorithm 2: ct <- ct (.) mu with
 * mu = Ecd((1 / ||m_q AND m_db||_1)_j)) of the scores of a slot-encoded chunk after icm_rescale
 * (modulus Q, unfolded): for result column j (eye e = j / rho, rotation r = j % rho) and block t,
 * mu_{j,t} = round(2^log2_scale_mu Ecd(v)) with v_i = 1 / ||rot_r(m_e) AND m_{t N/2 + i}||_1 (0 for
 * an empty overlap or a missing template), and both ciphertext parts of block t are multiplied
 * by it in Z_q[X]/(X^N + 1) for each limb of Q (negacyclic NTTs).  The output holds one full RLWE
 * pair per (column, block): dev_out [L_q][n_cols][n_blocks][2][N_db] u64, part 0 = a-part
 * a_j mu_{j,t}, part 1 = b_{j,t} mu_{j,t}; its slots decode to <c'_q, c'_db> / ||m_q AND m_db||_1
 * = 1 - 2 HD at scale Delta 2^s_db 2^log2_scale_mu (no rescaling follows).  dev_q_masks: device,
 * the n_eyes query masks (code_bits / 8 bytes each, unrotated); dev_db_masks: device, 8-byte
 * aligned, the chunk's n_db template masks.  icm_normalize_bytes gives the sizes of dev_out and of dev_ws (rotated
 * masks, overlaps, mu and NTT scratch).  Errors: ICM_EINVAL (not a rescaled unfolded slot-encoded
 * result, or another context's handle), ICM_ENOMEM (buffers too small), ICM_EBOUND
 * (Delta 2^s_db 2^log2_scale_mu >= Q / 4), ICM_ECUDA. */
icm_status icm_normalize_bytes(const icm_scores *rescaled, size_t *out_bytes, size_t *ws_bytes);
icm_status icm_normalize(icm_ctx *ctx, const icm_scores *rescaled, const uint8_t *dev_q_masks,
                         const uint8_t *dev_db_masks, uint32_t log2_scale_mu, void *dev_out, size_t bytes,
                         void *dev_ws, size_t ws_bytes, void *stream);
/* Decryption and decoding of normalised blocks for checking only (Section 2.2.2 Dec = a sk + b
 * under s_{db,t}; CRT over the limbs of Q to the centred integer; division by Delta 2^s_db
 * 2^log2_scale_mu; Dcd by fp64 FFT): dev_hd [n_cols][n_db] fp64 receives the decoded fractional
 * Hamming distance (1 - s) / 2 of every (column, template) pair.  dev_norm: icm_normalize's output.
 * Allocates and frees temporary device memory on `stream`. */
icm_status icm_decrypt_slots(icm_ctx *ctx, const icm_scores *rescaled, const void *dev_norm, size_t norm_bytes,
                             uint32_t log2_scale_mu, double *dev_hd, size_t n, void *stream);

/* Rescaling by Q' (Section 2.2.2, Maintenance: RS divides a ciphertext by a modulus factor and
 * rounds): scores at modulus Q_db = Q Q' (L limbs) become scores at the query modulus Q (the
 * first L_q limbs) with scale Delta, x' = round(x / Q') mod Q for every coefficient of both
 * ciphertext parts (base conversion from the limbs of Q' with the correction v = round(sum_i y_i /
 * q_i) taken from 64.64-bit fixed-point terms floor(y_i floor(2^128 / q_i) / 2^64): a coefficient
 * within (L - L_q) 2^-64 Q' of a half-integer multiple of Q' may round to either neighbour, inside the
 * rescaling error).  Works on folded or unfolded scores (the fold commutes with it up
 * to that error) and cuts their size L / L_q times.  icm_rescale_bytes gives the size of
 * dev_out (caller-owned, [L_q][n_cols][M] u64).  Errors: ICM_EINVAL (already rescaled, L_q = L,
 * or a handle of another context), ICM_ENOMEM (dev_out too small), ICM_ECUDA. */
icm_status icm_rescale_bytes(const icm_scores *in, size_t *bytes);
icm_status icm_rescale(icm_ctx *ctx, const icm_scores *in, void *dev_out, size_t bytes, void *stream,
                       icm_scores **out);

/* ---------------------------------------------------------------- batching form ---- */

/* Workspace bytes of icm_match_batch (the CRT forms' residue scratch over all chunks). */
icm_status icm_match_batch_workspace_bytes(const icm_ctx *ctx, const icm_db *const *dbs, size_t n_dbs, size_t n_eyes,
                                           icm_form form, size_t *bytes);

/* CCMM of one prepared query batch against 1..16 database chunks (each its own MSRLWE database
 * with its own a-part, uneven sizes allowed; Section 6.2.3 distributes the database the same way
 * over GPUs).  For the CRT forms every limb, chunk, row tile, modulus and column tile of a round of
 * up to 512 columns is one persistent kernel launch; the u64 and digit forms launch per chunk.
 * dev_outs[i]: scores of chunk i (icm_scores_bytes of that chunk); outs[i] receives its handle. */
icm_status icm_match_batch(icm_ctx *ctx, const icm_db *const *dbs, size_t n_dbs, const icm_query *q,
                           void *const *dev_outs, const size_t *out_bytes, void *dev_ws, size_t ws_bytes, void *stream,
                           icm_scores **outs);

/* A captured CUDA graph of one whole batch pass on fixed buffers: query preparation from dev_ct,
 * icm_match_batch over the chunks, and the fold of every chunk into dev_folded[i].  Created by
 * stream capture on `stream` (which must not be the legacy default stream); replayed with
 * icm_plan_launch on any stream.  The buffers must stay valid while the plan is used. */
typedef struct icm_plan icm_plan;
icm_status icm_plan_create(icm_ctx *ctx, const icm_db *const *dbs, size_t n_dbs, size_t n_eyes, icm_form form,
                           const void *dev_ct, void *dev_op, size_t op_bytes, void *const *dev_scores,
                           const size_t *scores_bytes, void *const *dev_folded, const size_t *folded_bytes,
                           void *dev_ws, size_t ws_bytes, void *stream, icm_plan **out);
icm_status icm_plan_launch(icm_plan *plan, void *stream);
void icm_plan_destroy(icm_plan *plan);

/* Kernel variant of the CRT forms' product: 256 = mma.sync with 256-column tiles, 128 = mma.sync
 * with 128-column tiles; for the fp16 form on a database in the storage form, the tcgen05 kernel
 * (tensor-memory accumulators, TMA-fed, one modulus on 512 columns per block and round, every
 * round of up to 1,024 columns in one launch; needs an even K, else variant 256 runs): 1 = rings
 * of 8 raw-database and 4 operand slots; 2 = the same with a wave bound between blocks (a block
 * starts fetching its next tile once every block has fetched its current one; cooperative
 * launch); 3 = 4 raw-database and 8 operand slots.  0 restores the default, variant 2 (which the
 * int8 form and odd K run as 256).  Results are identical; only speed differs. */
icm_status icm_ctx_set_variant(icm_ctx *ctx, int variant);
/* Failure detection of the tcgen05 kernel (no counterpart in the paper).  Every device-side wait
 * of that kernel (barrier phases, the wave bound) gives up after wait_ns nanoseconds of
 * %globaltimer (0 restores the default, 2 s): the kernel then records ICM_ETIMEOUT in the device
 * status word, stops issuing work, waits (bounded) for its own copies and MMAs in flight, frees
 * its tensor memory and returns; its outputs are then invalid.  inject_stall != 0 is for tests
 * only: the kernel's query producer of the first column tile then issues no copies, so the MMA
 * issuer's wait runs out on purpose (no fault, no trap).  Applies to later launches from this
 * context.  Errors: ICM_EINVAL for a null context. */
icm_status icm_ctx_set_device_wait(icm_ctx *ctx, uint64_t wait_ns, int inject_stall);
/* Device status word shared by the library's kernels: ICM_OK, or ICM_ETIMEOUT once a kernel gave
 * up one of its bounded waits (the kernel then stopped early, so its outputs are invalid).  Reads
 * the word (synchronising the device) and clears it when clear != 0. */
icm_status icm_device_status(int clear);

/* Autotuner: times the kernel variants of the CRT product that apply on the caller's batch (one
 * icm_match_batch per variant, CUDA events on `stream`): the tcgen05 variants 1-3 for the fp16
 * form with an even K, else the mma.sync tiles 128 and 256.  Keeps the fastest for the context
 * and reports it (0 for forms with a single variant).  ms_per_choice (optional, n_choices
 * entries) receives the time of each variant in the fixed order 128, 256, 1, 2, 3, with 0 for the
 * variants not timed. */
icm_status icm_autotune(icm_ctx *ctx, const icm_db *const *dbs, size_t n_dbs, const icm_query *q,
                        void *const *dev_outs, const size_t *out_bytes, void *dev_ws, size_t ws_bytes, void *stream,
                        int *best_tile_n, float *ms_per_choice, size_t n_choices);

/* ---------------------------------------------------------------- serving form ---- */

/* A request loop over a resident encrypted database (Section 5: computing servers batch up to 32
 * query eyes).  Query eyes are submitted one at a time with their wire ciphertext; a worker
 * thread batches them (a batch starts when max_eyes eyes wait or the oldest has waited
 * window_us; eyes arriving while batches run join a later one), runs query preparation, the
 * grouped CCMM and the folds, and returns every eye's folded scores.
 * Admission: at most max_pending eyes wait on the host (submit returns ICM_ENOMEM beyond that).
 * A batch starts when one of max_batches batch slots is free and the device workspace, used as a
 * pool, holds the buffers of at least one waiting eye: every batch of n eyes reserves the bytes
 * its buffers take at n eyes for its whole life (first fit) and takes as many waiting eyes (up to
 * max_eyes) as the free memory allows.  Each slot has its own compute and copy streams: one
 * batch's copies, query preparation and folds overlap another's CCMM; the CCMMs of successive
 * batches run one after the other. */
typedef struct icm_server icm_server;
typedef struct {
    uint32_t max_eyes;       /* eyes per batch, 1..32                                          */
    uint32_t window_us;      /* batching window for a partial batch                            */
    icm_form form;           /* arithmetic form of the CCMM                                    */
    uint32_t max_pending;    /* admission bound on waiting eyes (0 = 4096)                     */
    uint32_t max_batches;    /* batch slots (batches in flight), 0..4 (0 = 2)                  */
} icm_server_cfg;

/* Device workspace bytes that hold max_batches full batches (max_eyes eyes each).  A server runs
 * with any workspace of at least one full batch; with less than this, fewer or smaller batches
 * are admitted at a time. */
icm_status icm_server_device_bytes(const icm_ctx *ctx, const icm_db *const *dbs, size_t n_dbs,
                                   const icm_server_cfg *cfg, size_t *bytes);
/* Start a server on 1..16 resident chunks; dev_ws (ws_bytes, at least one full batch, else
 * ICM_ENOMEM) stays owned by the caller and must outlive it. */
icm_status icm_server_create(icm_ctx *ctx, const icm_db *const *dbs, size_t n_dbs, const icm_server_cfg *cfg,
                             void *dev_ws, size_t ws_bytes, icm_server **out);
/* Memory accounting: pool size, bytes of one full batch, the most bytes reserved at once and the
 * most batches in flight at once so far. */
icm_status icm_server_memory(icm_server *s, size_t *pool_bytes, size_t *full_batch_bytes, size_t *peak_bytes,
                             uint32_t *peak_batches);
/* Words (u64) of one eye's ciphertext ([L_q][rho][K], the eye's columns of the wire format) and
 * of one eye's result (for every chunk in order: [L][ceil(rho/fold_k)][M_c] folded scores). */
icm_status icm_server_eye_words(const icm_server *s, size_t *ct_words, size_t *out_words);
/* Queue one eye; host_ct and host_out must stay valid until icm_server_wait returns for the
 * ticket. */
icm_status icm_server_submit(icm_server *s, const uint64_t *host_ct, uint64_t *host_out, uint64_t *ticket);
/* Wait (bounded) for a ticket; on success its result is in host_out and latency_ms (optional)
 * gets the time from submission to completion.  The ticket is released. */
icm_status icm_server_wait(icm_server *s, uint64_t ticket, uint32_t timeout_ms, double *latency_ms);
/* Completed eyes, launched batches, and mean eyes per batch. */
icm_status icm_server_stats(icm_server *s, uint64_t *n_done, uint64_t *n_batches, double *mean_batch);
/* Stop accepting eyes, drain queued and running batches (bounded by timeout_ms), free the server.
 * On ICM_ETIMEOUT the worker keeps draining in the background and the server is not freed. */
icm_status icm_server_destroy(icm_server *s, uint32_t timeout_ms);

/* ---------------------------------------------------------------- host-buffer pipeline ---- */

/* Device workspace bytes of icm_match_host for n_eyes eyes of one chunk in a form. */
icm_status icm_match_host_workspace_bytes(const icm_ctx *ctx, const icm_db *db, size_t n_eyes, icm_form form,
                                          size_t *bytes);

/* One whole matching pass from host memory to host memory, enqueued on `stream`: copy the query
 * ciphertext (wire format, host_ct, icm_query_ct_bytes bytes) to the device, prepare it (basis
 * extension and planes of `form`), CCMM against `db` (Section 2.3), fold (Algorithm 2), and copy
 * the folded scores ([L][n_eyes * ceil(rho / fold_k)][M] u64) to host_folded.  The eyes run in two
 * parts (ceil(n_eyes / 2), then the rest) so that part 2's ciphertext copy overlaps part 1's
 * product and part 1's result copy overlaps part 2's product, on a copy stream the call creates
 * and joins back into `stream` (when `stream` completes, so has all of the call's work).  Host
 * buffers should be page-locked for asynchronous copies; they must stay valid until the stream
 * reaches the end of this work.  dev_ws: icm_match_host_workspace_bytes bytes of caller device
 * memory.  Errors: ICM_EINVAL (null arguments, no eyes), ICM_ENOMEM (workspace too small), and
 * those of icm_query_prepare, icm_match and icm_fold. */
icm_status icm_match_host(icm_ctx *ctx, const icm_db *db, const uint64_t *host_ct, size_t n_eyes, icm_form form,
                          uint64_t *host_folded, void *dev_ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------- plain modular product ---- */

/* Workspace bytes that icm_ppmm needs for a form (0 for ICM_FORM_U64). */
icm_status icm_ppmm_workspace_bytes(icm_form form, uint32_t n_limbs, size_t M, size_t N, size_t K, size_t *bytes);

/* Plaintext modular matrix product (PPMM, Section 2.3) on arbitrary operands:
 * dev_C[l][j][i] = sum_k dev_A[l][i][k] * dev_B[l][j][k] mod q_l, for canonical residues of odd
 * moduli q_l < 2^60 (host array; primes for the u64, digit and CRT forms, squares p_l^2 of odd
 * p_l <= 253 for ICM_FORM_I8_P2, else ICM_EINVAL).  A: [L][M][K], B: [L][N][K], C: [L][N][M] (u64,
 * device). */
icm_status icm_ppmm(icm_form form, const uint64_t *q, uint32_t n_limbs, const uint64_t *dev_A,
                    const uint64_t *dev_B, uint64_t *dev_C, size_t M, size_t N, size_t K,
                    void *dev_ws, size_t ws_bytes, void *stream);

/* Same product as icm_ppmm for the CRT forms (ICM_FORM_I8_CRT, ICM_FORM_F16_CRT), for callers
 * that cannot allocate device memory: it allocates nothing and takes no workspace.  The paper has
 * no counterpart; this serves hosts whose framework owns every device allocation, code running
 * under a fixed device-memory budget, or code enqueued while allocations are not allowed.  The
 * workspace (query residue planes and per-modulus residue scratch) lives in one static device
 * array of 64 MiB that every GPU loading this library holds until the process exits; problems
 * whose workspace exceeds it are rejected with ICM_ENOMEM before any work (checked before the
 * pointers).  The first call in a CUDA context (normally the device's primary context) looks up
 * that context's address of the array (make it before any stream capture); later calls in the
 * same context reuse it, and a context created later (a non-primary context made current, or the
 * primary context re-created after cudaDeviceReset) gets its own lookup on its first call.  All
 * calls share the array: calls that overlap on the GPU race with each other (serialise them, for
 * instance on one stream).  Arguments as icm_ppmm minus the workspace. */
icm_status icm_ppmm_noalloc(icm_form form, const uint64_t *q, uint32_t n_limbs, const uint64_t *dev_A,
                            const uint64_t *dev_B, uint64_t *dev_C, size_t M, size_t N, size_t K, void *stream);

/* ---------------------------------------------------------------- folding-polynomial check ---- */

/* Cleartext check of a folding polynomial (Section 4.1.2 defines a (k, N_f, P_f)-folding
 * polynomial f by two probabilities over negative scores drawn from a law D; Appendix C.2 checks
 * the paper's degree-7 f with 1e12 such experiments; Section 6.1 approximates D by N(0.008, 0.034^2)).
 * Trial t draws 2k - 1 scores from D = N(mu, sigma^2) with Philox4x64-10 (Salmon et al., SC 2011)
 * at counters (t, j, 0, 0), key (seed, 0), and the Box-Muller transform of word pairs (2p, 2p+1)
 * (u1 = (a + 1/2) 2^-64, u2 = b 2^-64; normals 0..k-1 are x_i, normals k..2k-2 are y_i), and forms
 * S_k = sum_i f(x_i) and S_{k-1} = sum_i f(y_i).  Scores, f and sums are computed in fp32. */
typedef struct {
    const double *coef;      /* host, degree + 1 values: f(x) = sum_i coef[i] x^i              */
    uint32_t degree;         /* 0..15                                                           */
    uint32_t k;              /* values per folded sum, 1..32 (the paper's folding capability)   */
    double mu, sigma;        /* the law D = N(mu, sigma^2), sigma > 0                           */
    double nf_lo, nf_hi;     /* N_f                                                             */
    double pf_lo, pf_hi;     /* P_f                                                             */
    double pos_lo, pos_hi;   /* P, the positive-score interval: the library finds min and max of
                                f over it (ends and sign changes of f') in double precision     */
    double hist_lo, hist_hi; /* histogram range of the sums                                     */
    uint32_t n_bins;         /* 0 (no histogram) .. 8192                                        */
    uint32_t accumulate;     /* 0: overwrite dev_counts / dev_hist; else add to them            */
    uint64_t seed;           /* Philox key word 0                                               */
    uint64_t trial0;         /* first trial index (runs over consecutive ranges continue a run)  */
    uint64_t n_trials;       /* trials of this call (0 allowed)                                  */
} icm_fold_mc_args;

/* Run trials trial0 .. trial0 + n_trials - 1 on `stream`.  dev_counts (device, 6 x u64): trials
 * with S_k < nf_lo, S_k > nf_hi, min_P f + S_{k-1} < pf_lo, min_P f + S_{k-1} > pf_hi,
 * max_P f + S_{k-1} < pf_lo, max_P f + S_{k-1} > pf_hi.  dev_hist (device, [2][n_bins + 2] u64,
 * may be NULL when n_bins = 0): histograms of S_k and of S_{k-1}, bin 0 below hist_lo, bins
 * 1..n_bins of width (hist_hi - hist_lo) / n_bins, bin n_bins + 1 at or above hist_hi.  dev_sums
 * (device, optional): n_trials pairs of float (S_k, S_{k-1}).  Device pointers 8-byte aligned.
 * Errors: ICM_EINVAL (bad degree, k, law, interval, histogram, alignment or a trial range that
 * wraps), ICM_ECUDA. */
icm_status icm_fold_mc(const icm_fold_mc_args *args, uint64_t *dev_counts, uint64_t *dev_hist, float *dev_sums,
                       void *stream);
/* Minimum and maximum of f over [lo, hi] as icm_fold_mc takes them for P (host only). */
icm_status icm_fold_poly_range(const double *coef, uint32_t degree, double lo, double hi, double *fmin,
                               double *fmax);

/* ---------------------------------------------------------------- measurement ---- */

/* Peak-rate probe used as a roofline denominator (no counterpart in the paper): runs an
 * issue-bound register-only loop of one instruction class on the current device, timed with
 * CUDA events on `stream` (synchronises it), and returns the rate.  kind 0: IMAD.WIDE operations
 * per second; kind 1: int8 mma.sync multiply-accumulates per second; kind 2: fp16 mma.sync
 * multiply-accumulates per second. */
icm_status icm_probe_peak(int kind, double *ops_per_s, void *stream);

/* ---------------------------------------------------------------- synchronisation ---- */

/* Wait for `stream` with a bound; ICM_ETIMEOUT if it has not finished in timeout_ms. */
icm_status icm_sync(void *stream, uint32_t timeout_ms);

#ifdef __cplusplus
}
#endif

#endif /* ICM_H */
