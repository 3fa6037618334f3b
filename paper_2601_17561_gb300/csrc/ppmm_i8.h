// Constants of the int8 tensor-core forms (digit pairs and small-modulus CRT), passed to kernels
// by value.
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>
#include "icm_device.cuh"

#define ICM_MAX_MODULI 24

namespace icm {

struct I8Consts {
    uint32_t n_limbs, n_mod;
    uint64_t q[ICM_MAX_LIMBS], r64[ICM_MAX_LIMBS];
    // digit form: 2^(8 s) mod q_l for shifts s = 0..14, with Shoup companions
    uint64_t pw8[ICM_MAX_LIMBS][15], pw8s[ICM_MAX_LIMBS][15];
    // CRT form: moduli, packed centred constants 256^t mod m (t = 0..3 and 4..7), 1/m,
    // y_i = (M/m_i)^-1 mod m_i and round(2^19 y_i / m_i), (M/m_i) mod q_l, y_i (M/m_i) mod q_l,
    // M mod q_l with Shoup companions
    int32_t mod[ICM_MAX_MODULI], wlo[ICM_MAX_MODULI], whi[ICM_MAX_MODULI], yinv[ICM_MAX_MODULI];
    float inv_m[ICM_MAX_MODULI];
    uint32_t r19[ICM_MAX_MODULI];
    // integer residue conversion of the tcgen05 path: dp4a bias c = m ceil(2^17 / m) + h with
    // h = floor(m / 2), division magic ceil(2^32 / m), and the f16x2 bits of -(1024 + h)
    int32_t cbias[ICM_MAX_MODULI];
    uint32_t magic[ICM_MAX_MODULI], hneg2[ICM_MAX_MODULI];
    uint64_t W[ICM_MAX_LIMBS][ICM_MAX_MODULI], Ws[ICM_MAX_LIMBS][ICM_MAX_MODULI], Wy[ICM_MAX_LIMBS][ICM_MAX_MODULI];
    uint64_t Mq[ICM_MAX_LIMBS], Mqs[ICM_MAX_LIMBS];
    // p^2 form: q_l = pd_l^2, digit base pd_l and 1 / pd_l (pw8[l][0..1] hold 1 and pd_l)
    int32_t pd[ICM_MAX_LIMBS];
    float inv_p[ICM_MAX_LIMBS];
    // launch settings of the tcgen05 kernel: bound of every device-side wait in ns (0: 2 s), and
    // the test-only stall of the query producer (its waits then run out on purpose)
    uint64_t tc_wait_ns;
    uint32_t tc_inject_stall;
};

// Builds the constants for primes q and contraction depth K; returns false (with a reason in
// `why`) if the int32 overflow invariant or the CRT range cannot be met.
bool make_i8_consts(int form, const uint64_t *q, size_t nq, uint64_t K, I8Consts &out, const char **why);
// Planes per residue: 8 digit planes, 2 base-p digit planes (p^2 form) or n_mod residue planes.
uint32_t i8_planes(int form, const uint64_t *q, size_t nq, uint64_t K);
inline uint64_t i8_kpad(uint64_t K) { return (K + 31) / 32 * 32; }

cudaError_t launch_planes(int form, const I8Consts &k, const uint64_t *op, int8_t *planes, uint64_t N, uint64_t K,
                          uint64_t Kp, cudaStream_t st);
#define ICM_MAX_CHUNKS 16
// Database chunks of one grouped launch.
struct ChunkTab {
    uint32_t n;
    const uint64_t *A[ICM_MAX_CHUNKS];     // [L][M_c][K]
    uint64_t *C[ICM_MAX_CHUNKS];           // [L][N][M_c]
    uint64_t M[ICM_MAX_CHUNKS];
    uint64_t row0[ICM_MAX_CHUNKS + 1];     // prefix sums of M_c
    uint32_t mt0[ICM_MAX_CHUNKS + 1];      // prefix sums of 128-row tiles
    int a_digits;                          // A in the balanced-digit storage form (else canonical)
};
bool make_chunk_tab(const uint64_t *const *A, uint64_t *const *C, const uint64_t *M, uint32_t n, ChunkTab &t);
cudaError_t launch_ppmm_crt_grouped(bool f16, int bn, const I8Consts &k, const ChunkTab &tab, const void *Bp, uint64_t N,
                                    uint64_t K, uint64_t Kp, void *scratch, cudaStream_t st);
cudaError_t crt_set_attributes();
// Kernel variants of the CRT product: the column tile of the mma.sync kernel (128, 256), or the
// tcgen05 kernel for the fp16 form on the balanced-digit database (one launch per 1,024 columns):
// 1 = rings of 8 raw-database and 4 operand slots, 2 = the same with the wave bound between blocks
// (cooperative launch), 3 = 4 raw-database and 8 operand slots.
#define ICM_CRT_TCGEN05 1
#define ICM_CRT_TCGEN05_LAST 3
inline bool crt_tc_variant(int v) { return v >= ICM_CRT_TCGEN05 && v <= ICM_CRT_TCGEN05_LAST; }
cudaError_t launch_crt_combine(const I8Consts &k, const ChunkTab &tab, const void *scratch, uint64_t N, uint64_t n0,
                               uint64_t nch, cudaStream_t st);
cudaError_t crt_tc_set_attributes();
bool crt_tc_supported(uint64_t K);
cudaError_t launch_ppmm_crt_tc(const I8Consts &k, const ChunkTab &tab, const void *Bp, uint64_t N, uint64_t K, uint64_t Kp,
                               void *scratch, int variant, cudaStream_t st);
uint32_t device_status(bool clear);
// Residue planes of the query operand in the CRT forms.
//  int8: [L][r][N][Kp], K contiguous.
//  fp16: per (limb, modulus) the columns are grouped in tiles of 256 (N padded with zero columns)
//  and K in slabs of 16; every (column tile, slab) pair is one contiguous 8 KB block holding the
//  256 x 16 operand in the tensor cores' K-major layout without swizzle: the core matrices
//  (8 columns x 8 consecutive k, 16 bytes per column) of k 0-7 for column groups 0..31, then those
//  of k 8-15.  One bulk copy moves a block into shared memory as it is; blocks of consecutive
//  slabs of a column tile are adjacent.
constexpr uint64_t CRT_F16_TN = 256;
__host__ __device__ inline uint64_t crt_f16_ncols(uint64_t N) { return (N + CRT_F16_TN - 1) / CRT_F16_TN * CRT_F16_TN; }
inline uint64_t crt_plane_bytes(bool f16, uint32_t n_limbs, uint32_t n_mod, uint64_t N, uint64_t Kp) {
    return f16 ? (uint64_t)n_limbs * n_mod * crt_f16_ncols(N) * Kp * 2 : (uint64_t)n_limbs * n_mod * N * Kp;
}
// fp16 element offset of (column j, k) within one (limb, modulus) plane of Kp columns of K
__host__ __device__ __forceinline__ uint64_t crt_f16_off(uint64_t j, uint64_t k, uint64_t Kp) {
    return ((j >> 8) * (Kp >> 4) + (k >> 4)) * 4096 + ((((k >> 3) & 1) * 32 + ((j & 255) >> 3)) * 8 + (j & 7)) * 8 +
           (k & 7);
}
// small-modulus CRT forms (int8 or fp16 operands): query residue planes, two-phase product.
// The limbs are processed in groups whose residue bytes stay within CRT_SCRATCH_CAP (at least one
// limb per group).  Scratch: the residue bytes [G][r][min(N, 1024)][M] of one group of G limbs
// and one column round of the largest kernel (rounded up to 256 bytes), then CRT_PROGRESS_BYTES
// for the tcgen05 kernel's wave counter and give-up word.
constexpr uint64_t CRT_PROGRESS_BYTES = 4096;
constexpr uint64_t CRT_SCRATCH_CAP = 6ull << 30;
inline uint32_t crt_limb_group(uint32_t n_limbs, uint32_t n_mod, uint64_t N, uint64_t M) {
    const uint64_t per = (uint64_t)n_mod * (N < 1024 ? N : 1024) * M;
    const uint64_t g = per ? CRT_SCRATCH_CAP / per : n_limbs;
    return g < 1 ? 1u : (g > n_limbs ? n_limbs : (uint32_t)g);
}
inline uint64_t crt_scratch_main_bytes(uint32_t n_limbs, uint32_t n_mod, uint64_t N, uint64_t M) {
    const uint64_t per = (uint64_t)n_mod * (N < 1024 ? N : 1024) * M;
    return (crt_limb_group(n_limbs, n_mod, N, M) * per + 255) / 256 * 256;
}
uint64_t crt_scratch_bytes(uint32_t n_limbs, uint32_t n_mod, uint64_t N, uint64_t M);
cudaError_t launch_crt_planes(bool f16, const I8Consts &k, const uint64_t *op, void *planes, uint64_t N, uint64_t K,
                              uint64_t Kp, cudaStream_t st);
cudaError_t launch_ppmm_crt(bool f16, int bn, const I8Consts &k, const uint64_t *A, bool a_digits, const void *Bp,
                            uint64_t *C, uint64_t M, uint64_t N, uint64_t K, uint64_t Kp, void *scratch, cudaStream_t st);
cudaError_t launch_ppmm_i8(int form, const I8Consts &k, const uint64_t *A, bool a_digits, const int8_t *Bp, uint64_t *C,
                           uint64_t M, uint64_t N, uint64_t K, uint64_t Kp, cudaStream_t st);

}  // namespace icm
