// Internal host-side declarations of libicm: handle structs, the database row layout and
// kernel launchers.  Not part of the public ABI (include/icm.h).
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/icm.h"
#include "icm_device.cuh"
#include "ppmm_i8.h"

namespace icm {

void set_error(const std::string &msg);

struct SecretSupport {           // sparse ternary polynomial: positions and signs of its non-zeros
    std::vector<int32_t> pos;
    std::vector<int8_t> sgn;
};

struct CrtDecode {               // constants of the fixed-point CRT decoding (decryption check)
    uint64_t inv[ICM_MAX_LIMBS];     // (Q_db / q_l)^-1 mod q_l
    uint64_t invs[ICM_MAX_LIMBS];    // Shoup companions
    uint64_t rhi[ICM_MAX_LIMBS];     // floor(2^128 / q_l), high and low words
    uint64_t rlo[ICM_MAX_LIMBS];
    double q_over_delta;             // Q / Delta
};

// Rescaling by Q' (x' = round(x / Q') mod Q, base conversion from the limbs of Q' to those of Q):
// for the limbs i of Q' (i >= Lq) yinv_i = (Q'/q_i)^-1 mod q_i; for the limbs j of Q (j < Lq)
// w[j][i] = (Q'/q_i) mod q_j, qp_j = Q' mod q_j and qpinv_j = Q'^-1 mod q_j; Shoup companions.
struct RescaleConsts {
    uint32_t L, Lq;
    uint64_t q[ICM_MAX_LIMBS];
    uint64_t yinv[ICM_MAX_LIMBS], yinvs[ICM_MAX_LIMBS];
    uint64_t rhi[ICM_MAX_LIMBS], rlo[ICM_MAX_LIMBS];       // floor(2^128 / q_i), high and low words
    uint64_t w[ICM_MAX_LIMBS][ICM_MAX_LIMBS], ws[ICM_MAX_LIMBS][ICM_MAX_LIMBS];
    uint64_t qp[ICM_MAX_LIMBS], qps[ICM_MAX_LIMBS], qpinv[ICM_MAX_LIMBS], qpinvs[ICM_MAX_LIMBS];
};

}  // namespace icm

namespace icm { struct SlotTables; void free_slot_tables(SlotTables *t); }

struct icm_ctx {
    icm_params p;
    uint32_t N_db, N_q, K, n_qblk;      // ring degrees, K = d2 + N_q, n_qblk = d2 / N_q
    std::vector<uint64_t> q;            // primes
    LimbTable lt;
    icm::CrtDecode crt;                 // decoding at modulus Q_db (L limbs, scale Q' Delta)
    icm::CrtDecode crt_q;               // decoding at modulus Q after rescaling (L_q limbs, scale Delta)
    icm::RescaleConsts rs;
    std::vector<uint64_t> qp_mod;       // Q' mod q_l (gadget factor)
    std::vector<uint64_t> qp_mods;      // Shoup companions
    std::vector<uint64_t> delta_mod;    // Delta mod q_l
    std::vector<uint64_t> delta_mods;
    icm::I8Consts i8_digits, i8_crt;    // constants of the int8 tensor-core forms for (q, K)
    bool i8_crt_ok = false;
    int crt_bn = 2;                     // CRT product variant: tcgen05 wave where it applies, else 256
    bool have_keys = false;
    int device = -1;
    // device copies of the secret supports: s_{db,t} for t < max_db_blocks, s_{q,t} for t < n_qblk
    uint32_t max_db_blocks = 0;
    int32_t *d_sdb_pos = nullptr;  int8_t *d_sdb_sgn = nullptr;   // [max_db_blocks][h]
    int32_t *d_sq_pos = nullptr;   int8_t *d_sq_sgn = nullptr;    // [n_qblk][h]
    icm::SlotTables *slot_tab = nullptr;   // slot-encoding and NTT tables (built on first use)
    ~icm_ctx();
};

// Row layout of one database chunk (see include/icm.h): a-part rows, full blocks, then the
// partial block's real rows followed by its wrap-around tail coefficients.
struct DbLayout {
    uint32_t N;            // N_db
    uint64_t n_real;       // real templates
    uint32_t n_full;       // full b-blocks
    uint32_t rem;          // real rows of the partial block (0 if none)
    uint32_t tail_lo;      // first tail coefficient of the partial block
    uint64_t M;            // stored rows
    uint64_t n_tpl = 0;    // templates (a slot-encoded chunk holds N/2 per block)
    uint32_t slot_log2 = 0;  // log2 of the database slot-encoding scale; 0: coefficient encoding
    uint32_t n_blocks() const { return n_full + (rem ? 1u : 0u); }
};
namespace icm { DbLayout make_layout(uint64_t n_real, uint32_t N, uint32_t rho); }

struct icm_db {
    const icm_ctx *ctx;
    DbLayout lay;
    uint64_t chunk_id;
    uint64_t *dev;          // [L][M][K]
    size_t bytes;
};

struct icm_query {
    const icm_ctx *ctx;
    icm_form form;
    uint32_t n_eyes, n_cols;   // n_cols = d3 = n_eyes * rho
    void *dev;                 // prepared operand
    size_t bytes;
};

struct icm_scores {
    const icm_ctx *ctx;
    DbLayout lay;
    uint32_t n_eyes, n_cols;
    int folded;
    int rescaled;              // 1: rescaled by Q' (modulus Q, L_q limbs, scale Delta)
    uint64_t *dev;             // [limbs][n_cols][M], limbs = L, or L_q when rescaled
    size_t bytes;
};

namespace icm {

// Device-side view of the layout for kernels.
struct LayoutDev {
    uint32_t N, n_full, rem, tail_lo;
    uint64_t n_real, M;
};
inline LayoutDev to_dev(const DbLayout &l) { return {l.N, l.n_full, l.rem, l.tail_lo, l.n_real, l.M}; }

// ---- launchers (return cudaGetLastError of the launch)
cudaError_t launch_db_messages(const icm_ctx *c, const LayoutDev &lay, const uint8_t *d_codes,
                               const uint8_t *d_masks, uint64_t *d_db, cudaStream_t st,
                               const int32_t *d_wmsg = nullptr);
cudaError_t launch_db_apart_and_b(const icm_ctx *c, const LayoutDev &lay, uint64_t chunk_id, uint64_t *d_db,
                                  cudaStream_t st);
cudaError_t launch_query_encrypt(const icm_ctx *c, const uint8_t *d_codes, const uint8_t *d_masks,
                                 const uint64_t *d_eye_ids, uint32_t n_eyes, uint64_t *d_ct, cudaStream_t st);
cudaError_t launch_query_extend(const icm_ctx *c, const uint64_t *d_ct, uint32_t n_cols, uint64_t *d_op,
                                cudaStream_t st);
cudaError_t launch_ppmm_u64(const LimbTable &lt, const uint64_t *A, const uint64_t *B, uint64_t *C,
                            uint64_t M, uint64_t N, uint64_t K, bool a_digits, cudaStream_t st);
cudaError_t launch_fold(const icm_ctx *c, const LayoutDev &lay, const uint64_t *d_in, uint32_t n_eyes, uint32_t limbs,
                        uint64_t *d_out, cudaStream_t st);
cudaError_t launch_decrypt(const icm_ctx *c, const LayoutDev &lay, const uint64_t *d_scores, uint32_t n_cols,
                           bool rescaled, int64_t *d_num, cudaStream_t st, uint32_t *d_err_bits = nullptr);
// Rescaling by Q' of n coefficients per limb: [L][n] at modulus Q_db -> [L_q][n] at modulus Q.
cudaError_t launch_rescale(const icm_ctx *c, const uint64_t *d_in, uint64_t n, uint64_t *d_out, cudaStream_t st);

LimbTable make_limb_table(const std::vector<uint64_t> &q);
uint64_t shoup_of(uint64_t w, uint64_t q);

}  // namespace icm
