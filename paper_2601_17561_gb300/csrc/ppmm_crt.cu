// Plaintext modular matrix product over a small-modulus RNS on tensor cores (Section 6.2.2: the
// modular products are reduced to int8 GEMMs through an RNS of small moduli below 2^8).  Used by
// the forms ICM_FORM_I8_CRT (int8 operands, mma.sync m16n8k32 s8 -> s32) and ICM_FORM_F16_CRT
// (the same residues held exactly as fp16, mma.sync m16n8k16 f16 -> f32; GB300 issues fp16 tensor
// products at about four times its int8 rate).
//
// For r pairwise-coprime odd moduli m_i < 256 with product M > 2^3 K ((q-1)/2)^2:
//  phase 1 (one block per limb, modulus, 128-row tile and column tile): c_i = C mod m_i with
//    C = sum_k a[k] b[k] over the centred residues a = A mod m_i, b = B mod m_i (|x| <= 127) of
//    the centred lifts of A and B.  int8: int32 accumulation is exact (K 2^14 < 2^31).  fp16:
//    products <= 127^2 are exact in fp32 and the fp32 sum stays an exact integer below 2^24, so it
//    is reduced modulo m_i every 1024 columns of K (1024 * 127^2 + 1.5 * 255 < 2^24; a reduction
//    leaves |x| <= 1.5 m_i because the rounded quotient may be off by one).  c_i goes to a byte
//    scratch.
//  phase 2 (one thread per output): C mod q = sum_i c_i (y_i M/m_i mod q) - kappa (M mod q) with
//    y_i = (M/m_i)^-1 mod m_i and kappa = round(sum_i c_i y_i / m_i) (|C| / M <= 2^-3 and the
//    fixed-point sum is within 2^-7 of the exact one, so the rounding decides kappa exactly).
//
// Phase 1 tiling: 128 x BN tile per 256-thread block (2 x 4 warps, 64 x BN/4 each), K in slabs of
// 32 values.  The database residues are formed on the fly from the canonical u64 (centred lift,
// balanced base-256 digits, two dp4a against the centred constants 256^t mod m_i, one rounding
// step) and stored to shared memory; the next slab is loaded into registers while the current
// one is multiplied.  The query planes stream in with cp.async.  Fragments come from ldmatrix on
// rows padded by 16 bytes (conflict-free).  Blocks of one (limb, row tile) are consecutive in
// launch order (column tiles, then moduli, vary fastest) so a database slab is read from HBM
// about once and re-served from L2.  Columns are processed in chunks of 512 (the scratch holds
// L r min(N, 1024) M bytes, the largest column round of any CRT kernel).
#include "icm_internal.h"
#include "ppmm_i8.h"

#include <algorithm>
#include <cuda_fp16.h>

namespace {

constexpr int BM = 128, KS = 32, NT = 256, FLUSH = 1024;
constexpr uint64_t NCHUNK = 512;            // columns per phase-1/phase-2 round

struct P1Args {
    icm::ChunkTab tab;       // database chunks: A_c [L][M_c][K], scratch row offsets, row-tile offsets
    const void *Bp;          // residue planes: int8 [L][r][N][Kp], or fp16 tiled (crt_f16_off)
    uint8_t *R;              // [L][r][nch][sum M_c] scratch
    uint64_t N, K, Kp, n0, nch;
    uint32_t n_ntile;
    uint64_t n_tiles;        // L * (row tiles of all chunks) * r * n_ntile
    icm::I8Consts k;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool pred) {
    const int n = pred ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(n));
}

template <bool F16>
struct Acc;
template <>
struct Acc<true> { using T = float; };
template <>
struct Acc<false> { using T = int; };

__device__ __forceinline__ void mma(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ void mma(int (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Centred residue (|r| <= m/2) modulo m of a residue given by its balanced digits z (the storage
// form of the database): lift(x) = sum_t d_t 256^t, so two dp4a against the centred constants
// w_t = 256^t mod m give a representative s with |s| <= 2^17, then one rounding step.
__device__ __forceinline__ int crt_residue_z(uint64_t z, int m, int wlo, int whi, float inv_m) {
    int s = __dp4a((int)(uint32_t)z, wlo, 0);
    s = __dp4a((int)(uint32_t)(z >> 32), whi, s);
    return s - m * __float2int_rn((float)s * inv_m);
}
__device__ __forceinline__ int crt_residue(uint64_t x, uint64_t q, int m, int wlo, int whi, float inv_m) {
    return crt_residue_z(to_digit_form(x, q), m, wlo, whi, inv_m);
}

// 4 residues -> packed operand bits (int8: one word, fp16: two words)
template <bool F16>
__device__ __forceinline__ void pack4(const int (&v)[4], uint32_t (&w)[2]) {
    if (F16) {
        __half2 h01 = __halves2half2(__int2half_rn(v[0]), __int2half_rn(v[1]));
        __half2 h23 = __halves2half2(__int2half_rn(v[2]), __int2half_rn(v[3]));
        w[0] = *reinterpret_cast<uint32_t *>(&h01);
        w[1] = *reinterpret_cast<uint32_t *>(&h23);
    } else {
        w[0] = (uint32_t)(v[0] & 0xFF) | ((uint32_t)(v[1] & 0xFF) << 8) | ((uint32_t)(v[2] & 0xFF) << 16) |
               ((uint32_t)(v[3] & 0xFF) << 24);
        w[1] = 0;
    }
}

template <bool F16, int BN>
__global__ void __launch_bounds__(NT, 1) k_crt_p1(P1Args p) {
    constexpr int ESZ = F16 ? 2 : 1;              // operand bytes
    constexpr int ROWB = KS * ESZ;                // bytes of one row of a slab
    constexpr int LDB = ROWB + 16;                // padded row stride (bytes)
    constexpr int STEPS = ROWB / 32;              // mma k-steps per slab (32 operand bytes each)
    constexpr int WN = BN / 4;                    // warp tile columns
    constexpr int NT8 = WN / 8;
    using AccT = typename Acc<F16>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *sA = smem;                                   // [2][BM][LDB]
    unsigned char *sB = smem + 2 * BM * LDB;                    // [2][BN][LDB]
    const uint32_t r = p.k.n_mod;
    const uint32_t mt_total = p.tab.mt0[p.tab.n];
    const uint64_t N = p.N, K = p.K, Kp = p.Kp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;

    // persistent loop: tiles ordered (limb, row tile, modulus, column tile), column tile fastest,
    // so that the blocks running at the same time share database slabs through L2
    for (uint64_t tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x) {
    uint64_t tt = tile;
    const uint32_t nt = (uint32_t)(tt % p.n_ntile); tt /= p.n_ntile;
    const uint32_t mi = (uint32_t)(tt % r); tt /= r;
    const uint32_t mtg = (uint32_t)(tt % mt_total);
    const uint32_t l = (uint32_t)(tt / mt_total);
    uint32_t c = 0;
    while (c + 1 < p.tab.n && mtg >= p.tab.mt0[c + 1]) ++c;
    const uint64_t M = p.tab.M[c];
    const uint64_t m0 = (uint64_t)(mtg - p.tab.mt0[c]) * BM, nb = (uint64_t)nt * BN;   // nb: column within the chunk
    const int m = p.k.mod[mi], wlo = p.k.wlo[mi], whi = p.k.whi[mi];
    const float inv_m = p.k.inv_m[mi];
    const uint64_t q = p.k.q[l];
    const uint64_t *Al = p.tab.A[c] + (size_t)l * M * K;
    // int8 planes [L][r][N][Kp] from the round's first column; fp16 planes in 256-column tiles
    const unsigned char *Bl = reinterpret_cast<const unsigned char *>(p.Bp) +
                              (F16 ? ((size_t)l * r + mi) * icm::crt_f16_ncols(N) * Kp * ESZ
                                   : (((size_t)l * r + mi) * N + p.n0) * Kp * ESZ);

    AccT acc[4][NT8][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < NT8; ++b)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) acc[a][b][cc] = 0;

    uint64_t ra[4][4];                            // prefetched slab: 4 groups of 4 consecutive k
    auto load_a = [&](uint64_t k0) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = tid + e * NT, row = idx >> 3, g = idx & 7;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint64_t k = k0 + g * 4 + j;
                ra[e][j] = (m0 + row < M && k < K) ? __ldg(Al + (m0 + row) * K + k) : 0ull;
            }
        }
    };
    auto store_a = [&](int st) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = tid + e * NT, row = idx >> 3, g = idx & 7;
            int v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                v[j] = p.tab.a_digits ? crt_residue_z(ra[e][j], m, wlo, whi, inv_m) : crt_residue(ra[e][j], q, m, wlo, whi, inv_m);
            uint32_t w[2];
            pack4<F16>(v, w);
            unsigned char *dst = sA + (size_t)st * BM * LDB + row * LDB + g * 4 * ESZ;
            if (F16) *reinterpret_cast<uint2 *>(dst) = make_uint2(w[0], w[1]);
            else *reinterpret_cast<uint32_t *>(dst) = w[0];
        }
    };
    constexpr int CH = ROWB / 16;                 // 16-byte chunks per column per slab
    auto load_b = [&](int st, uint64_t k0) {
#pragma unroll
        for (int e = 0; e < (BN * CH) / NT; ++e) {
            const int idx = tid + e * NT, col = idx / CH, ch = idx % CH;
            const bool ok = p.n0 + nb + col < N && nb + col < p.nch;
            const uint64_t off = F16 ? icm::crt_f16_off(p.n0 + nb + col, k0 + ch * 8, Kp) * 2
                                     : ((nb + col) * Kp + k0) * ESZ + ch * 16;
            const unsigned char *src = Bl + (ok ? off : 0);
            cp_async16(smem_u32(sB + (size_t)st * BN * LDB + col * LDB + ch * 16), src, ok);
        }
        asm volatile("cp.async.commit_group;");
    };

    const uint64_t nk = (K + KS - 1) / KS;
    if (nk > 0) {
        load_a(0);
        load_b(0, 0);
        store_a(0);
        asm volatile("cp.async.wait_group 0;");
        __syncthreads();
    }
    for (uint64_t kt = 0; kt < nk; ++kt) {
        const int st = (int)(kt & 1);
        const bool more = kt + 1 < nk;
        if (more) { load_a((kt + 1) * KS); load_b(st ^ 1, (kt + 1) * KS); }
        const unsigned char *a_s = sA + (size_t)st * BM * LDB, *b_s = sB + (size_t)st * BN * LDB;
#pragma unroll
        for (int ks = 0; ks < STEPS; ++ks) {
            uint32_t af[4][4], bf[NT8][2];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int row = wm * 64 + a * 16 + (lane & 15);
                ldsm_x4(af[a][0], af[a][1], af[a][2], af[a][3], smem_u32(a_s + row * LDB + ks * 32 + (lane >> 4) * 16));
            }
#pragma unroll
            for (int b = 0; b < NT8; b += 2) {
                const int ncol = wn * WN + b * 8 + (lane & 7) + ((lane >> 4) << 3);
                ldsm_x4(bf[b][0], bf[b][1], bf[b + 1][0], bf[b + 1][1],
                        smem_u32(b_s + ncol * LDB + ks * 32 + ((lane >> 3) & 1) * 16));
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < NT8; ++b) mma(acc[a][b], af[a], bf[b]);
        }
        if (F16 && ((kt + 1) * KS) % FLUSH == 0) {
            const float fm = (float)m;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < NT8; ++b)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) {
                        float &x = reinterpret_cast<float &>(acc[a][b][cc]);
                        x = fmaf(-fm, rintf(x * inv_m), x);
                    }
        }
        if (more) store_a(st ^ 1);
        asm volatile("cp.async.wait_group 0;");
        __syncthreads();
    }

    // c_i in [0, m) to the scratch, column-major within the column chunk, rows of all chunks
    const int g = lane >> 2, tq = lane & 3;
    const uint64_t Mall = p.tab.row0[p.tab.n];
    uint8_t *Rl = p.R + ((size_t)l * r + mi) * p.nch * Mall + p.tab.row0[c];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < NT8; ++b)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const uint64_t row = m0 + wm * 64 + a * 16 + g + (cc >> 1) * 8;
                const uint64_t col = nb + wn * WN + b * 8 + tq * 2 + (cc & 1);
                if (row >= M || col >= p.nch || p.n0 + col >= N) continue;
                int v;
                if (F16) v = __float2int_rn(reinterpret_cast<const float &>(acc[a][b][cc])) % m;
                else v = reinterpret_cast<const int &>(acc[a][b][cc]) % m;
                v = v < 0 ? v + m : v;
                Rl[col * Mall + row] = (uint8_t)v;
            }
    __syncthreads();          // shared buffers are reused by the next tile
    }
}

struct P2Args {
    icm::ChunkTab tab;       // outputs C_c [L][N][M_c]
    const uint8_t *R;        // [L][r][nch][sum M_c]
    uint64_t N, n0, nch;
    icm::I8Consts k;
};

// Phase 2: with y_i = (M/m_i)^-1 mod m_i, sum_i c_i y_i (M/m_i) = C + kappa M for an integer kappa
// (each term's residue modulo m_i is c_i, and modulo every other m_j it is 0), so
// C mod q = sum_i c_i Wy_i - kappa (M mod q) with the constants Wy_i = y_i (M/m_i) mod q, and
// kappa = round(sum_i c_i y_i / m_i) in fixed point: T = sum_i c_i R_i with
// R_i = round(2^19 y_i / m_i) < 2^19 is 2^19 (kappa + C / M) within r 2^7 (c_i < 2^8), and
// |C| / M <= 1/8, so kappa = (T + 2^18) >> 19 exactly (T < r 2^27 fits 32 bits).  Each thread
// takes V consecutive rows of one column (V = 4: one 4-byte load per modulus plane, when the row
// count keeps those words aligned).
template <int V>
__global__ void __launch_bounds__(256) k_crt_combine(P2Args p) {
    const uint32_t l = blockIdx.y;
    const uint64_t Mall = p.tab.row0[p.tab.n];
    const uint64_t cnt = p.nch * Mall;
    const uint32_t r = p.k.n_mod;
    const uint64_t q = p.k.q[l];
    const uint64_t idx = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * V;     // (column, row) within the round
    if (idx >= cnt) return;
    const uint64_t col = idx / Mall, grow0 = idx % Mall;
    const uint8_t *Rl = p.R + (size_t)l * r * cnt + idx;
    // sum_i c_i Wy_i over the 32-bit halves of Wy_i (c_i < 2^8, Wy_i < 2^60: each half-sum stays
    // below r 2^40), reduced once at the end
    uint64_t Alo[V], Ahi[V];
    uint32_t T[V];
#pragma unroll
    for (int e = 0; e < V; ++e) { Alo[e] = 0; Ahi[e] = 0; T[e] = 0; }
    for (uint32_t i = 0; i < r; ++i) {
        const uint32_t w = V == 4 ? *reinterpret_cast<const uint32_t *>(Rl + (size_t)i * cnt) : Rl[(size_t)i * cnt];
        const uint32_t ri = p.k.r19[i];
        const uint32_t wlo = (uint32_t)p.k.Wy[l][i], whi = (uint32_t)(p.k.Wy[l][i] >> 32);
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const uint32_t c = (w >> (8 * e)) & 0xFF;
            Alo[e] += (uint64_t)c * wlo;
            Ahi[e] += (uint64_t)c * whi;
            T[e] += c * ri;
        }
    }
    const uint64_t r64 = p.k.r64[l], p32 = p.k.pw8[l][4], p32s = p.k.pw8s[l][4];       // 2^32 mod q
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const uint64_t grow = grow0 + e;
        uint32_t c = 0;
        while (c + 1 < p.tab.n && grow >= p.tab.row0[c + 1]) ++c;
        const uint64_t row = grow - p.tab.row0[c], M = p.tab.M[c];
        const uint64_t S = add_mod(reduce64(Alo[e], q, r64), mulmod_shoup(reduce64(Ahi[e], q, r64), p32, p32s, q), q);
        const uint64_t kappa = (T[e] + (1u << 18)) >> 19;
        p.tab.C[c][((size_t)l * p.N + p.n0 + col) * M + row] = sub_mod(S, mulmod_shoup(kappa, p.k.Mq[l], p.k.Mqs[l], q), q);
    }
}

// int8 residue planes of the query operand: [L][r][N][Kp], zero padded.
__global__ void __launch_bounds__(256) k_crt_planes_i8(const uint64_t *op, int8_t *planes, uint64_t N, uint64_t K,
                                                       uint64_t Kp, icm::I8Consts k) {
    const uint32_t l = blockIdx.y;
    const uint32_t r = k.n_mod;
    const uint64_t q = k.q[l];
    const uint64_t total = N * Kp;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t j = idx / Kp, kk = idx % Kp;
        const uint64_t v = kk < K ? op[((size_t)l * N + j) * K + kk] : 0;
        for (uint32_t i = 0; i < r; ++i)
            planes[((size_t)l * r + i) * total + idx] = (int8_t)crt_residue(v, q, k.mod[i], k.wlo[i], k.whi[i], k.inv_m[i]);
    }
}

// fp16 residue planes in the tiled layout of crt_f16_off (zero padded in K and in the columns
// of the last 256-column tile).  One thread per (column, 8 consecutive k): it reads 64 bytes of
// the operand and writes one 16-byte core-matrix row per modulus; consecutive threads take
// consecutive columns, so their stores fill contiguous memory.
__global__ void __launch_bounds__(256) k_crt_planes_f16(const uint64_t *op, __half *planes, uint64_t N, uint64_t K,
                                                        uint64_t Kp, icm::I8Consts k) {
    const uint32_t l = blockIdx.y;
    const uint32_t r = k.n_mod;
    const uint64_t q = k.q[l];
    const uint64_t Np = icm::crt_f16_ncols(N), total = Np * (Kp / 8);
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t j = idx % Np, k0 = (idx / Np) * 8;
        uint64_t v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = (j < N && k0 + e < K) ? op[((size_t)l * N + j) * K + k0 + e] : 0;
        const uint64_t o = icm::crt_f16_off(j, k0, Kp);
        for (uint32_t i = 0; i < r; ++i) {
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                __half2 h = __halves2half2(__int2half_rn(crt_residue(v[2 * e], q, k.mod[i], k.wlo[i], k.whi[i], k.inv_m[i])),
                                           __int2half_rn(crt_residue(v[2 * e + 1], q, k.mod[i], k.wlo[i], k.whi[i], k.inv_m[i])));
                w[e] = *reinterpret_cast<uint32_t *>(&h);
            }
            *reinterpret_cast<uint4 *>(planes + ((size_t)l * r + i) * Np * Kp + o) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

template <bool F16, int BN>
constexpr size_t p1_smem() { return (size_t)2 * (BM + BN) * (KS * (F16 ? 2 : 1) + 16); }

template <bool F16, int BN>
cudaError_t set_p1_attr() {
    return cudaFuncSetAttribute(k_crt_p1<F16, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p1_smem<F16, BN>());
}

template <bool F16, int BN>
cudaError_t run_p1(const P1Args &a, cudaStream_t st) {
    const size_t smem = p1_smem<F16, BN>();
    cudaError_t e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t grid = std::min<uint64_t>(a.n_tiles, (uint64_t)sms);     // one resident block per SM
    if (grid == 0) return cudaSuccess;
    k_crt_p1<F16, BN><<<(unsigned)grid, NT, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

namespace icm {

cudaError_t crt_set_attributes() {
    cudaError_t e = crt_tc_set_attributes();
    if (e == cudaSuccess) e = set_p1_attr<true, 128>();
    if (e == cudaSuccess) e = set_p1_attr<true, 256>();
    if (e == cudaSuccess) e = set_p1_attr<false, 128>();
    if (e == cudaSuccess) e = set_p1_attr<false, 256>();
    return e;
}

uint64_t crt_scratch_bytes(uint32_t n_limbs, uint32_t n_mod, uint64_t N, uint64_t M) {
    static_assert(NCHUNK <= 1024, "crt_scratch_main_bytes holds column rounds of up to 1,024");
    return crt_scratch_main_bytes(n_limbs, n_mod, N, M) + CRT_PROGRESS_BYTES;
}

bool make_chunk_tab(const uint64_t *const *A, uint64_t *const *C, const uint64_t *M, uint32_t n, ChunkTab &t) {
    if (n == 0 || n > ICM_MAX_CHUNKS) return false;
    t = ChunkTab{};
    t.n = n;
    t.a_digits = 1;
    t.row0[0] = 0;
    t.mt0[0] = 0;
    for (uint32_t c = 0; c < n; ++c) {
        t.A[c] = A[c];
        t.C[c] = C[c];
        t.M[c] = M[c];
        t.row0[c + 1] = t.row0[c] + M[c];
        t.mt0[c + 1] = t.mt0[c] + (uint32_t)((M[c] + BM - 1) / BM);
    }
    return true;
}

cudaError_t launch_crt_planes(bool f16, const I8Consts &k, const uint64_t *op, void *planes, uint64_t N, uint64_t K,
                              uint64_t Kp, cudaStream_t st) {
    if (N == 0 || Kp == 0) return cudaSuccess;
    if (Kp % 16 || (f16 && reinterpret_cast<uintptr_t>(planes) % 16)) return cudaErrorInvalidValue;
    const uint64_t total = f16 ? crt_f16_ncols(N) * (Kp / 8) : N * Kp;
    const unsigned blocks = (unsigned)std::min<uint64_t>((total + 255) / 256, 152u * 32u);
    if (f16) k_crt_planes_f16<<<dim3(blocks, k.n_limbs), 256, 0, st>>>(op, reinterpret_cast<__half *>(planes), N, K, Kp, k);
    else k_crt_planes_i8<<<dim3(blocks, k.n_limbs), 256, 0, st>>>(op, reinterpret_cast<int8_t *>(planes), N, K, Kp, k);
    return cudaGetLastError();
}

// The constants of limbs [l0, l0 + n) as a context of n limbs.
static I8Consts limb_slice(const I8Consts &k, uint32_t l0, uint32_t n) {
    I8Consts s = k;
    s.n_limbs = n;
    for (uint32_t l = 0; l < n; ++l) {
        const uint32_t f = l0 + l;
        s.q[l] = k.q[f]; s.r64[l] = k.r64[f];
        for (int t = 0; t < 15; ++t) { s.pw8[l][t] = k.pw8[f][t]; s.pw8s[l][t] = k.pw8s[f][t]; }
        for (uint32_t i = 0; i < ICM_MAX_MODULI; ++i) {
            s.W[l][i] = k.W[f][i]; s.Ws[l][i] = k.Ws[f][i]; s.Wy[l][i] = k.Wy[f][i];
        }
        s.Mq[l] = k.Mq[f]; s.Mqs[l] = k.Mqs[f];
        s.pd[l] = k.pd[f]; s.inv_p[l] = k.inv_p[f];
    }
    return s;
}

cudaError_t launch_ppmm_crt_grouped(bool f16, int bn, const I8Consts &k, const ChunkTab &tab, const void *Bp, uint64_t N,
                                    uint64_t K, uint64_t Kp, void *scratch, cudaStream_t st) {
    const uint64_t Mall = tab.row0[tab.n];
    if (Mall == 0 || N == 0) return cudaSuccess;
    // limbs in groups that fit the residue scratch: each group is the same product on a slice of
    // the database words, query planes and outputs
    const uint32_t G = crt_limb_group(k.n_limbs, k.n_mod, N, Mall);
    if (G < k.n_limbs) {
        const uint64_t plane_limb = crt_plane_bytes(f16, 1, k.n_mod, N, Kp);
        for (uint32_t l0 = 0; l0 < k.n_limbs; l0 += G) {
            const uint32_t n = std::min(G, k.n_limbs - l0);
            ChunkTab t = tab;
            for (uint32_t c = 0; c < tab.n; ++c) {
                t.A[c] = tab.A[c] + (uint64_t)l0 * tab.M[c] * K;
                t.C[c] = tab.C[c] + (uint64_t)l0 * N * tab.M[c];
            }
            const I8Consts s = limb_slice(k, l0, n);
            cudaError_t e = launch_ppmm_crt_grouped(f16, bn, s, t, static_cast<const char *>(Bp) + l0 * plane_limb, N,
                                                    K, Kp, scratch, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (f16 && crt_tc_variant(bn) && tab.a_digits && crt_tc_supported(K))
        return launch_ppmm_crt_tc(k, tab, Bp, N, K, Kp, scratch, bn, st);
    if (bn != 128) bn = 256;
    for (uint64_t n0 = 0; n0 < N; n0 += NCHUNK) {
        const uint64_t nch = std::min<uint64_t>(NCHUNK, N - n0);
        P1Args a{};
        a.tab = tab; a.Bp = Bp; a.R = reinterpret_cast<uint8_t *>(scratch);
        a.N = N; a.K = K; a.Kp = Kp; a.n0 = n0; a.nch = nch;
        a.n_ntile = (uint32_t)((nch + bn - 1) / bn);
        a.n_tiles = (uint64_t)k.n_limbs * tab.mt0[tab.n] * k.n_mod * a.n_ntile;
        a.k = k;
        cudaError_t e;
        if (f16) e = bn == 128 ? run_p1<true, 128>(a, st) : run_p1<true, 256>(a, st);
        else e = bn == 128 ? run_p1<false, 128>(a, st) : run_p1<false, 256>(a, st);
        if (e != cudaSuccess) return e;
        e = launch_crt_combine(k, tab, scratch, N, n0, nch, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_crt_combine(const I8Consts &k, const ChunkTab &tab, const void *scratch, uint64_t N, uint64_t n0,
                               uint64_t nch, cudaStream_t st) {
    const uint64_t Mall = tab.row0[tab.n];
    P2Args b{tab, reinterpret_cast<const uint8_t *>(scratch), N, n0, nch, k};
    if ((Mall & 3) == 0) {
        const uint64_t threads = nch * Mall / 4;
        k_crt_combine<4><<<dim3((unsigned)((threads + 255) / 256), k.n_limbs), 256, 0, st>>>(b);
    } else {
        k_crt_combine<1><<<dim3((unsigned)((nch * Mall + 255) / 256), k.n_limbs), 256, 0, st>>>(b);
    }
    return cudaGetLastError();
}

cudaError_t launch_ppmm_crt(bool f16, int bn, const I8Consts &k, const uint64_t *A, bool a_digits, const void *Bp,
                            uint64_t *C, uint64_t M, uint64_t N, uint64_t K, uint64_t Kp, void *scratch, cudaStream_t st) {
    ChunkTab tab;
    make_chunk_tab(&A, &C, &M, 1, tab);
    tab.a_digits = a_digits ? 1 : 0;
    return launch_ppmm_crt_grouped(f16, bn, k, tab, Bp, N, K, Kp, scratch, st);
}

}  // namespace icm
