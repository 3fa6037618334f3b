// Plaintext modular matrix product on CUDA cores, u64 form (Section 2.3: the CCMM is dominated
// by plaintext products modulo the ciphertext modulus; here one product per RNS limb):
//     C[l][j][i] = sum_k A[l][i][k] B[l][j][k]  mod q_l,   q_l < 2^60.
//
// Exact lazy accumulation: every residue splits into three 20-bit limbs, a = a0 + a1 2^20 + a2 2^40.
// The nine 40-bit limb products of a MAC are summed by shift s = i + j into five 64-bit
// accumulators U_s (each IMAD.WIDE adds a < 2^40 product), so no reduction happens inside the
// K loop: U_2 gains three products per k, 3 K 2^40 < 2^64 for K < 2^22.  The epilogue reduces
// sum_s U_s 2^(20 s) modulo q_l with Shoup multiplications by the constants 2^(20 s) mod q_l.
//
// A arrives either canonical or in the balanced-digit storage form of the database (mapped back to
// canonical on load).
//
// Tiling: a 64 x 64 output tile per 256-thread block, 4 x 4 outputs per thread, K in steps of
// 16.  Global loads are coalesced along K (both operands are K-contiguous); the tile is split
// into limbs once on its way into shared memory (stored k-major so that a thread reads its four
// rows or columns with one 16-byte load per limb); the next K-slab is loaded into registers
// while the current one is multiplied.
#include "icm_internal.h"

namespace {

constexpr int BM = 64, BN = 64, BK = 16, PAD = 8, NT = 256;

struct PpmmArgs {
    const uint64_t *A, *B;
    uint64_t *C;
    uint64_t M, N, K;
    LimbTable lt;
    int a_digits;            // A stored in the balanced-digit form
};

__global__ void __launch_bounds__(NT, 1) k_ppmm_u64(PpmmArgs p) {
    __shared__ __align__(16) uint32_t As[3][BK][BM + PAD];
    __shared__ __align__(16) uint32_t Bs[3][BK][BN + PAD];
    const uint32_t l = blockIdx.z;
    const uint64_t m0 = (uint64_t)blockIdx.x * BM, n0 = (uint64_t)blockIdx.y * BN;
    const uint64_t M = p.M, N = p.N, K = p.K;
    const uint64_t *Al = p.A + (size_t)l * M * K;
    const uint64_t *Bl = p.B + (size_t)l * N * K;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const uint64_t q = p.lt.q[l], r64 = p.lt.r64[l];

    uint64_t acc[4][4][5];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int s = 0; s < 5; ++s) acc[i][j][s] = 0;

    uint64_t ra[4], rb[4];
    auto gload = [&](uint64_t k0) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = tid + e * NT, r = idx >> 4, kk = idx & 15;
            const uint64_t k = k0 + kk;
            ra[e] = (m0 + r < M && k < K) ? (p.a_digits ? from_digit_form(__ldg(Al + (m0 + r) * K + k), q)
                                                        : __ldg(Al + (m0 + r) * K + k)) : 0ull;
            rb[e] = (n0 + r < N && k < K) ? __ldg(Bl + (n0 + r) * K + k) : 0ull;
        }
    };
    auto sstore = [&]() {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = tid + e * NT, r = idx >> 4, kk = idx & 15;
            const uint64_t a = ra[e], b = rb[e];
            As[0][kk][r] = (uint32_t)(a & 0xFFFFF);
            As[1][kk][r] = (uint32_t)((a >> 20) & 0xFFFFF);
            As[2][kk][r] = (uint32_t)(a >> 40);
            Bs[0][kk][r] = (uint32_t)(b & 0xFFFFF);
            Bs[1][kk][r] = (uint32_t)((b >> 20) & 0xFFFFF);
            Bs[2][kk][r] = (uint32_t)(b >> 40);
        }
    };

    const uint64_t nk = (K + BK - 1) / BK;
    gload(0);
    sstore();
    __syncthreads();
    for (uint64_t kt = 0; kt < nk; ++kt) {
        if (kt + 1 < nk) gload((kt + 1) * BK);
#pragma unroll 2
        for (int kk = 0; kk < BK; ++kk) {
            uint4 a0 = *reinterpret_cast<const uint4 *>(&As[0][kk][ty * 4]);
            uint4 a1 = *reinterpret_cast<const uint4 *>(&As[1][kk][ty * 4]);
            uint4 a2 = *reinterpret_cast<const uint4 *>(&As[2][kk][ty * 4]);
            uint4 b0 = *reinterpret_cast<const uint4 *>(&Bs[0][kk][tx * 4]);
            uint4 b1 = *reinterpret_cast<const uint4 *>(&Bs[1][kk][tx * 4]);
            uint4 b2 = *reinterpret_cast<const uint4 *>(&Bs[2][kk][tx * 4]);
            const uint32_t av[3][4] = {{a0.x, a0.y, a0.z, a0.w}, {a1.x, a1.y, a1.z, a1.w}, {a2.x, a2.y, a2.z, a2.w}};
            const uint32_t bv[3][4] = {{b0.x, b0.y, b0.z, b0.w}, {b1.x, b1.y, b1.z, b1.w}, {b2.x, b2.y, b2.z, b2.w}};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j][0] += (uint64_t)av[0][i] * bv[0][j];
                    acc[i][j][1] += (uint64_t)av[0][i] * bv[1][j];
                    acc[i][j][1] += (uint64_t)av[1][i] * bv[0][j];
                    acc[i][j][2] += (uint64_t)av[0][i] * bv[2][j];
                    acc[i][j][2] += (uint64_t)av[1][i] * bv[1][j];
                    acc[i][j][2] += (uint64_t)av[2][i] * bv[0][j];
                    acc[i][j][3] += (uint64_t)av[1][i] * bv[2][j];
                    acc[i][j][3] += (uint64_t)av[2][i] * bv[1][j];
                    acc[i][j][4] += (uint64_t)av[2][i] * bv[2][j];
                }
        }
        __syncthreads();
        if (kt + 1 < nk) {
            sstore();
            __syncthreads();
        }
    }

    // epilogue: sum_s U_s 2^(20 s) mod q
    uint64_t *Cl = p.C + (size_t)l * N * M;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint64_t col = n0 + tx * 4 + j;
        if (col >= N) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint64_t row = m0 + ty * 4 + i;
            if (row >= M) continue;
            uint64_t v = 0;
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                const uint64_t u = reduce64(acc[i][j][s], q, r64);
                v = add_mod(v, mulmod_shoup(u, p.lt.pw20[l][s], p.lt.pw20s[l][s], q), q);
            }
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
