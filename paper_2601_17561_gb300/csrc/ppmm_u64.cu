// Plaintext modular matrix product on CUDA cores, u64 form (Section 2.3: the CCMM is dominated
// by plaintext products modulo the ciphertext modulus; here one product per RNS limb):
//     C[l][j][i] = sum_k A[l][i][k] B[l][j][k]  mod q_l,   q_l < 2^60.
//
// Exact lazy accumulation: every residue splits into two 30-bit limbs, a = a0 + a1 2^30.  The four
// 60-bit limb products of a MAC go into three 64-bit accumulators by shift (S0 = sum a0 b0,
// S1 = sum a0 b1 + a1 b0, S2 = sum a1 b1), one IMAD.WIDE each; S1 gains two products below 2^60
// per column, so after 8 columns every accumulator is below 2^64.  Every 8 columns the value
// S0 + S1 2^30 + S2 2^60 (< 2^125) is added into a 160-bit accumulator (a u128 and a carry word)
// with integer adds and shifts, which issue on the ALU pipe while the IMAD.WIDE stream keeps the
// FMA pipe busy.  The epilogue reduces the 160-bit sum modulo q_l with Shoup multiplications by
// 2^64 mod q_l and 2^128 mod q_l.
//
// A arrives either canonical or in the balanced-digit storage form of the database (mapped back to
// canonical when the slab is stored to shared memory, after the load latency).
//
// Tiling: a 64 x 32 output tile per 256-thread block, 4 x 2 outputs per thread (each output holds
// eleven 32-bit registers of accumulator), K in steps of 16.  Global loads are coalesced along K
// (both operands are K-contiguous); the tile is split into limbs once on its way into shared
// memory (stored k-major, rows padded to 2 mod 32 words so that the stores are conflict-free; a
// thread reads its rows or columns with 8-byte loads); the next K-slab is loaded into registers
// while the current one is multiplied.
#include "icm_internal.h"

namespace {

constexpr int BM = 64, BN = 32, BK = 16, NT = 256, FL = 8, TM = 4, TN = 2;
// shared row lengths (words): 2 mod 32 makes the slab stores conflict-free (a warp stores 16 k x 2 rows)
constexpr int AW = BM + 2, BW = BN + 2;

struct PpmmArgs {
    const uint64_t *A, *B;
    uint64_t *C;
    uint64_t M, N, K;
    LimbTable lt;
    int a_digits;            // A stored in the balanced-digit form
};

using u128 = unsigned __int128;

__global__ void __launch_bounds__(NT, 1) k_ppmm_u64(PpmmArgs p) {
    __shared__ __align__(16) uint32_t As[2][BK][AW];
    __shared__ __align__(16) uint32_t Bs[2][BK][BW];
    const uint32_t l = blockIdx.z;
    const uint64_t m0 = (uint64_t)blockIdx.x * BM, n0 = (uint64_t)blockIdx.y * BN;
    const uint64_t M = p.M, N = p.N, K = p.K;
    const uint64_t *Al = p.A + (size_t)l * M * K;
    const uint64_t *Bl = p.B + (size_t)l * N * K;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const uint64_t q = p.lt.q[l], r64 = p.lt.r64[l];

    uint64_t s[TM][TN][3];
    u128 R[TM][TN];
    uint32_t Rh[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            s[i][j][0] = s[i][j][1] = s[i][j][2] = 0;
            R[i][j] = 0;
            Rh[i][j] = 0;
        }

    // slab loads: A is BM x BK (4 words per thread), B is BN x BK (2 words per thread)
    uint64_t ra[BM * BK / NT], rb[BN * BK / NT];
    auto gload = [&](uint64_t k0) {
#pragma unroll
        for (int e = 0; e < BM * BK / NT; ++e) {
            const int idx = tid + e * NT, r = idx >> 4, kk = idx & 15;
            const uint64_t k = k0 + kk;
            ra[e] = (m0 + r < M && k < K) ? __ldg(Al + (m0 + r) * K + k) : 0ull;
        }
#pragma unroll
        for (int e = 0; e < BN * BK / NT; ++e) {
            const int idx = tid + e * NT, r = idx >> 4, kk = idx & 15;
            const uint64_t k = k0 + kk;
            rb[e] = (n0 + r < N && k < K) ? __ldg(Bl + (n0 + r) * K + k) : 0ull;
        }
    };
    auto sstore = [&]() {
#pragma unroll
        for (int e = 0; e < BM * BK / NT; ++e) {
            const int idx = tid + e * NT, r = idx >> 4, kk = idx & 15;
            // digit-form words are mapped back here, after the load latency has passed
            const uint64_t a = p.a_digits ? from_digit_form(ra[e], q) : ra[e];
            As[0][kk][r] = (uint32_t)(a & 0x3FFFFFFF);
            As[1][kk][r] = (uint32_t)(a >> 30);
        }
#pragma unroll
        for (int e = 0; e < BN * BK / NT; ++e) {
            const int idx = tid + e * NT, r = idx >> 4, kk = idx & 15;
            Bs[0][kk][r] = (uint32_t)(rb[e] & 0x3FFFFFFF);
            Bs[1][kk][r] = (uint32_t)(rb[e] >> 30);
        }
    };
    // fold the three shift accumulators into the 160-bit sum
    auto flush = [&]() {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const u128 v = (u128)s[i][j][0] + ((u128)s[i][j][1] << 30) + ((u128)s[i][j][2] << 60);
                const u128 nr = R[i][j] + v;
                Rh[i][j] += (nr < R[i][j]) ? 1u : 0u;
                R[i][j] = nr;
                s[i][j][0] = s[i][j][1] = s[i][j][2] = 0;
            }
    };

    const uint64_t nk = (K + BK - 1) / BK;
    gload(0);
    sstore();
    __syncthreads();
    for (uint64_t kt = 0; kt < nk; ++kt) {
        if (kt + 1 < nk) gload((kt + 1) * BK);
#pragma unroll
        for (int half = 0; half < BK / FL; ++half) {
#pragma unroll
            for (int k8 = 0; k8 < FL; ++k8) {
                const int kk = half * FL + k8;
                const uint2 a0l = *reinterpret_cast<const uint2 *>(&As[0][kk][ty * TM]);
                const uint2 a0h = *reinterpret_cast<const uint2 *>(&As[0][kk][ty * TM + 2]);
                const uint2 a1l = *reinterpret_cast<const uint2 *>(&As[1][kk][ty * TM]);
                const uint2 a1h = *reinterpret_cast<const uint2 *>(&As[1][kk][ty * TM + 2]);
                const uint2 b0 = *reinterpret_cast<const uint2 *>(&Bs[0][kk][tx * TN]);
                const uint2 b1 = *reinterpret_cast<const uint2 *>(&Bs[1][kk][tx * TN]);
                const uint32_t av[2][TM] = {{a0l.x, a0l.y, a0h.x, a0h.y}, {a1l.x, a1l.y, a1h.x, a1h.y}};
                const uint32_t bv[2][TN] = {{b0.x, b0.y}, {b1.x, b1.y}};
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) {
                        s[i][j][0] += (uint64_t)av[0][i] * bv[0][j];
                        s[i][j][1] += (uint64_t)av[0][i] * bv[1][j];
                        s[i][j][1] += (uint64_t)av[1][i] * bv[0][j];
                        s[i][j][2] += (uint64_t)av[1][i] * bv[1][j];
                    }
            }
            flush();
        }
        __syncthreads();
        if (kt + 1 < nk) {
            sstore();
            __syncthreads();
        }
    }

    // epilogue: (Rh 2^128 + R) mod q
    uint64_t *Cl = p.C + (size_t)l * N * M;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
        const uint64_t col = n0 + tx * TN + j;
        if (col >= N) continue;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const uint64_t row = m0 + ty * TM + i;
            if (row >= M) continue;
            const uint64_t r0 = (uint64_t)R[i][j], r1 = (uint64_t)(R[i][j] >> 64);
            uint64_t v = reduce64(r0, q, r64);
            v = add_mod(v, mulmod_shoup(reduce64(r1, q, r64), p.lt.pw64[l], p.lt.pw64s[l], q), q);
            v = add_mod(v, mulmod_shoup(Rh[i][j], p.lt.pw128[l], p.lt.pw128s[l], q), q);
            Cl[col * M + row] = v;
        }
    }
}

}  // namespace

namespace icm {

cudaError_t launch_ppmm_u64(const LimbTable &lt, const uint64_t *A, const uint64_t *B, uint64_t *C,
                            uint64_t M, uint64_t N, uint64_t K, bool a_digits, cudaStream_t st) {
    if (M == 0 || N == 0) return cudaSuccess;
    PpmmArgs p{A, B, C, M, N, K, lt, a_digits ? 1 : 0};
    dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), lt.n);
    k_ppmm_u64<<<grid, NT, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace icm
