// Plaintext modular matrix product on int8 tensor cores (Section 6.2.2 reduces the modular
// products to int8 x int8 -> int32 GEMMs).  sm_103a has no tcgen05 int8 MMA kind, so these
// kernels issue the warp-level mma.sync.m16n8k32.s32.s8.s8.s32.  Two exact forms:
//
// Digit form.  The centred lift x in (-q/2, q/2] of a residue has a unique expansion in signed
// balanced base-256 digits, x = sum_t d_t 256^t with d_t in [-128, 127]: the bytes of
// x + 0x8080808080808080 are d_t + 128.  Then sum_k A[i][k] B[j][k] = sum_s T_s 256^s with
// T_s = sum_{t+u=s} sum_k d^A_t[i][k] d^B_u[j][k], one int8 GEMM per digit pair (64 per limb), the
// pairs of one shift s sharing an int32 accumulator.  Overflow invariant: a shift with p pairs
// sums at most p * Kc products of magnitude <= 2^14 per chunk of Kc columns, and
// p * Kc * 2^14 <= 2^31 - 1 is kept by splitting K into chunks; after every chunk the accumulator
// is folded into the modular result R += (T mod q) (2^(8 s) mod q).
//
// CRT form (small-modulus RNS, as in the paper's own RNS of small moduli below 2^8): for r
// pairwise-coprime odd moduli m_i < 256 whose product M exceeds 2 K ((q-1)/2)^2 by 2^2, one int8 GEMM
// per modulus on the centred residues of x mod m_i gives c_i = C mod m_i exactly (K (2^7)^2 < 2^31),
// and C mod q = sum_i c_i (y_i (M/m_i) mod q) - kappa (M mod q) with y_i = (M/m_i)^-1 mod m_i and
// kappa = round(sum_i c_i y_i / m_i): sum_i c_i y_i (M/m_i) = C + kappa M, and
// sum_i c_i y_i / m_i = kappa + C / M with |C / M| <= 2^-3, evaluated in fixed point with
// constants round(2^19 y_i / m_i), off by at most r 2^7 / 2^19 < 2^-7 (c_i < 2^8, r <= 24), so
// the rounding decides kappa exactly.
// Residues of the database operand are formed on the fly from its digits with two dp4a.
//
// Base-p digit form (the paper's own modulus family, Section 6.2.2: Q = prod p^2): for q = p^2
// with odd p <= 253 the centred lift x in (-q/2, q/2] splits as x = x0 + p x1 with x0 the centred
// residue of x mod p (|x0| <= (p-1)/2) and |x1| <= 126, and
// x y = x0 y0 + p (x0 y1 + x1 y0) (mod p^2).  k_ppmm_p2 sweeps K once: every slab's database
// words are split into both digit planes in shared memory, and three int8 products per fragment
// feed two int32 accumulators, T_0 = sum x0 y0 and T_1 = sum (x0 y1 + x1 y0) (the paper's
// K-concatenation of the two cross products); every chunk of 65,504 columns (2 Kc 2^14 < 2^31)
// folds (T_0 + p T_1) mod p^2 into the result.
//
// Tiling (k_ppmm_digits, k_ppmm_p2): 128 x 64 output tile per 256-thread block (8 warps, 32 x 32
// each, 2 x 4 m16n8 tiles), K in slabs of 32; the next slab's words are loaded into registers while
// the current one is multiplied.  Operands are converted into shared memory directly in mma
// fragment order (one 16-byte load per A fragment, one 8-byte load per B fragment,
// conflict-free).  The query operand comes pre-split into int8 planes [L][P][N][Kp] (Kp: K rounded
// up to 32, zero padded).  This file builds the CRT form's constants and query planes; its
// products run in ppmm_crt.cu (k_crt_p1) and ppmm_crt_tc.cu (k_crt_tc).
#include "icm_internal.h"
#include "ppmm_i8.h"

#include <algorithm>
#include <cmath>

namespace {

constexpr int BM = 128, BN = 64, BK = 32, NT = 256;
constexpr int MT = BM / 16, NTL = BN / 8;     // m16 and n8 tiles per block

struct I8Args {
    const uint64_t *A;      // [L][M][K] residues, canonical or balanced-digit form (a_digits)
    const int8_t *Bp;       // [L][P][N][Kp] planes
    uint64_t *C;            // [L][N][M]
    uint64_t M, N, K, Kp;
    icm::I8Consts k;
    int a_digits;
};

__device__ __forceinline__ void mma_s8(int (&c)[4], const uint4 &a, const uint2 &b) {
    asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
                 : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y));
}

// Balanced digits of the centred lift of 4 residues (same row, 4 consecutive k): out[t] packs
// digit t of the 4 values (k ascending in bytes 0..3).
__device__ __forceinline__ void digits4(const uint64_t (&x)[4], uint64_t q, bool in_digits, uint32_t (&out)[8]) {
    uint32_t lo[4], hi[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const uint64_t z = in_digits ? x[e] : to_digit_form(x[e], q);   // bytes = signed digits d_t
        lo[e] = (uint32_t)z;
        hi[e] = (uint32_t)(z >> 32);
    }
    // gather byte t of the four words
    const uint32_t a01 = __byte_perm(lo[0], lo[1], 0x5140), a23 = __byte_perm(lo[2], lo[3], 0x5140);
    const uint32_t b01 = __byte_perm(lo[0], lo[1], 0x7362), b23 = __byte_perm(lo[2], lo[3], 0x7362);
    const uint32_t c01 = __byte_perm(hi[0], hi[1], 0x5140), c23 = __byte_perm(hi[2], hi[3], 0x5140);
    const uint32_t d01 = __byte_perm(hi[0], hi[1], 0x7362), d23 = __byte_perm(hi[2], hi[3], 0x7362);
    out[0] = __byte_perm(a01, a23, 0x5410); out[1] = __byte_perm(a01, a23, 0x7632);
    out[2] = __byte_perm(b01, b23, 0x5410); out[3] = __byte_perm(b01, b23, 0x7632);
    out[4] = __byte_perm(c01, c23, 0x5410); out[5] = __byte_perm(c01, c23, 0x7632);
    out[6] = __byte_perm(d01, d23, 0x5410); out[7] = __byte_perm(d01, d23, 0x7632);
}

// Centred residue (|r| <= 127, m odd) of x mod m from the 8 digits of x: x = sum_t d_t 256^t, so
// x = sum_t d_t w_t (mod m) with centred constants w_t = 256^t mod m; two dp4a give the sum.
__device__ __forceinline__ int residue_from_digits(uint32_t dlo, uint32_t dhi, int wlo, int whi, int m, float inv_m) {
    int s = __dp4a((int)dlo, wlo, 0);
    s = __dp4a((int)dhi, whi, s);
    int r = s - m * __float2int_rn((float)s * inv_m);
    const int h = (m - 1) >> 1;
    r = r > h ? r - m : (r < -h ? r + m : r);
    return r;
}

// Centred base-p digits (x0, x1) of the centred lift of a residue v of q = p^2 (odd p <= 253):
// x1 = round(x / p) (|x| < 2^15, so the fp32 quotient is exact to far below 1/(2p) and x / p is
// never a half-integer for odd p), x0 = x - p x1.
__device__ __forceinline__ void pdigits(uint64_t v, uint64_t q, int pb, float ip, int &x0, int &x1) {
    const int x = (int)(v > (q >> 1) ? (int64_t)v - (int64_t)q : (int64_t)v);
    x1 = __float2int_rn((float)x * ip);
    x0 = x - x1 * pb;
    const int h = (pb - 1) >> 1;
    if (x0 > h) { x0 -= pb; ++x1; } else if (x0 < -h) { x0 += pb; --x1; }
}

// Base-p digits of 4 residues (same row, 4 consecutive k): out[t] packs digit t of the 4 values.
__device__ __forceinline__ void pdigits4(const uint64_t (&x)[4], uint64_t q, int pb, float ip, uint32_t (&out)[2]) {
    out[0] = out[1] = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        int d0, d1;
        pdigits(x[e], q, pb, ip, d0, d1);
        out[0] |= (uint32_t)(d0 & 0xFF) << (8 * e);
        out[1] |= (uint32_t)(d1 & 0xFF) << (8 * e);
    }
}

// Digit form: one pass per shift s = 0..14 over the pairs t + u = s.  The next slab's database
// words and query plane words are loaded into registers while the current slab is multiplied; the
// modular results R (32 u64 per thread, updated once per K-chunk) live in shared memory to leave
// the registers to the prefetch.  Dynamic shared memory: sA 32 KB, sB 16 KB, sR 64 KB.
constexpr size_t DIG_SMEM = 8 * MT * 32 * 4 * 4 + 8 * NTL * 32 * 2 * 4 + 32 * NT * 8;

__global__ void __launch_bounds__(NT, 1) k_ppmm_digits(I8Args p) {
    extern __shared__ __align__(16) uint8_t dsm[];
    uint32_t (*sA)[MT][32][4] = reinterpret_cast<uint32_t (*)[MT][32][4]>(dsm);
    uint32_t (*sB)[NTL][32][2] = reinterpret_cast<uint32_t (*)[NTL][32][2]>(dsm + 8 * MT * 32 * 4 * 4);
    uint64_t *sR = reinterpret_cast<uint64_t *>(dsm + 8 * MT * 32 * 4 * 4 + 8 * NTL * 32 * 2 * 4);   // [32][NT]
    const uint32_t l = blockIdx.z;
    const uint64_t m0 = (uint64_t)blockIdx.x * BM, n0 = (uint64_t)blockIdx.y * BN;
    const uint64_t M = p.M, N = p.N, K = p.K, Kp = p.Kp;
    const uint64_t *Al = p.A + (size_t)l * M * K;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 3, wn = warp >> 2;
    const uint64_t q = p.k.q[l], r64 = p.k.r64[l];
    const int8_t *Bl = p.Bp + (size_t)l * 8 * N * Kp;
    for (int i = 0; i < 32; ++i) sR[i * NT + tid] = 0;

    uint64_t xr[4][4];
    uint32_t br[8][2];
    for (int pass = 0; pass < 15; ++pass) {
        const int t_lo = max(0, pass - 7), t_hi = min(7, pass);
        // K-chunk keeping np * Kc * 2^14 <= 2^31 - 1 for the np pairs of this shift
        const uint64_t kc = (uint64_t)((2147483647u / (16384u * (uint32_t)(t_hi - t_lo + 1))) / BK * BK);
        auto load = [&](uint64_t k0) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int idx = tid + e * NT, r = idx >> 3, g = idx & 7;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint64_t k = k0 + g * 4 + j;
                    xr[e][j] = (m0 + r < M && k < K) ? __ldg(Al + (m0 + r) * K + k) : 0ull;
                }
            }
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                if (t < t_lo || t > t_hi) continue;
                const int8_t *Bu = Bl + (size_t)(pass - t) * N * Kp;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int idx = tid + e * NT, cidx = idx >> 3, g = idx & 7;
                    br[t][e] = n0 + cidx < N ? __ldg(reinterpret_cast<const uint32_t *>(Bu + (n0 + cidx) * Kp + k0 + g * 4))
                                             : 0u;
                }
            }
        };
        int acc[2][4][4];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][b][c] = 0;
        if (K > 0) load(0);
        for (uint64_t k0 = 0; k0 < K; k0 += BK) {
            __syncthreads();
            // ---- A: 128 rows x 32 k into the digit planes of this shift; B: the matching planes
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int idx = tid + e * NT, r = idx >> 3, g = idx & 7;
                const int mt = r >> 4, rr = r & 15;
                const int reg = (rr >> 3) + ((g >> 2) << 1), ln = ((rr & 7) << 2) + (g & 3);
                uint32_t d[8];
                digits4(xr[e], q, p.a_digits != 0, d);
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (t >= t_lo && t <= t_hi) sA[t][mt][ln][reg] = d[t];
            }
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                if (t < t_lo || t > t_hi) continue;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int idx = tid + e * NT, cidx = idx >> 3, g = idx & 7;
                    sB[t][cidx >> 3][((cidx & 7) << 2) + (g & 3)][g >> 2] = br[t][e];
                }
            }
            __syncthreads();
            if (k0 + BK < K) load(k0 + BK);
            // ---- MMA: all pairs of this shift
            for (int t = t_lo; t <= t_hi; ++t) {
                uint4 af[2];
                uint2 bf[4];
#pragma unroll
                for (int a = 0; a < 2; ++a) af[a] = *reinterpret_cast<const uint4 *>(&sA[t][wm * 2 + a][lane][0]);
#pragma unroll
                for (int b = 0; b < 4; ++b) bf[b] = *reinterpret_cast<const uint2 *>(&sB[t][wn * 4 + b][lane][0]);
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) mma_s8(acc[a][b], af[a], bf[b]);
            }
            // ---- end of a K-chunk: R += (T_s mod q) (2^(8 s) mod q)
            if ((k0 + BK) % kc == 0 || k0 + BK >= K) {
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b)
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const uint64_t v = reduce_s64((int64_t)acc[a][b][c], q, r64);
                            uint64_t &R = sR[((a * 4 + b) * 4 + c) * NT + tid];
                            R = add_mod(R, mulmod_shoup(v, p.k.pw8[l][pass], p.k.pw8s[l][pass], q), q);
                            acc[a][b][c] = 0;
                        }
            }
        }
    }
    // ---- store (column-major output)
    const int g = lane >> 2, tq = lane & 3;
    uint64_t *Cl = p.C + (size_t)l * N * M;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint64_t row = m0 + (uint64_t)(wm * 2 + a) * 16 + g + (c >> 1) * 8;
                const uint64_t col = n0 + (uint64_t)(wn * 4 + b) * 8 + tq * 2 + (c & 1);
                if (row < M && col < N) Cl[col * M + row] = sR[((a * 4 + b) * 4 + c) * NT + tid];
            }
}

// p^2 form, one sweep over K (see the file comment).  Same 128 x 64 tile and fragment layout as
// k_ppmm_digits; blockIdx.x enumerates (row tile, column tile) with column tiles fastest so that the
// blocks in flight share one row tile of the database operand in L2.
__global__ void __launch_bounds__(NT, 1) k_ppmm_p2(I8Args p) {
    __shared__ __align__(16) uint32_t sA[2][MT][32][4];
    __shared__ __align__(16) uint32_t sB[2][NTL][32][2];
    const uint32_t l = blockIdx.z;
    const uint64_t M = p.M, N = p.N, K = p.K, Kp = p.Kp;
    const uint64_t n_tiles = (N + BN - 1) / BN;
    const uint64_t m0 = (uint64_t)blockIdx.x / n_tiles * BM, n0 = (uint64_t)blockIdx.x % n_tiles * BN;
    const uint64_t *Al = p.A + (size_t)l * M * K;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 3, wn = warp >> 2;
    const uint64_t q = p.k.q[l], r64 = p.k.r64[l];
    const int pb = p.k.pd[l];
    const float ip = p.k.inv_p[l];
    const int8_t *Bl = p.Bp + (size_t)l * 2 * N * Kp;
    constexpr uint64_t KC = (2147483647u / (16384u * 2u)) / BK * BK;   // 65,504

    uint32_t R[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) R[a][b][c] = 0;

    // the next slab's words are loaded into registers while the current one is multiplied
    uint64_t xr[4][4];
    uint32_t br[2][2];
    auto load = [&](uint64_t k0) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = tid + e * NT, r = idx >> 3, g = idx & 7;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint64_t k = k0 + g * 4 + j;
                xr[e][j] = (m0 + r < M && k < K) ? __ldg(Al + (m0 + r) * K + k) : 0ull;
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int idx = tid + e * NT, cidx = idx >> 3, g = idx & 7;
                br[u][e] = n0 + cidx < N
                    ? __ldg(reinterpret_cast<const uint32_t *>(Bl + (size_t)u * N * Kp + (n0 + cidx) * Kp + k0 + g * 4))
                    : 0u;
            }
    };
    int acc0[2][4][4], acc1[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) { acc0[a][b][c] = 0; acc1[a][b][c] = 0; }
    if (K > 0) load(0);
    for (uint64_t k0 = 0; k0 < K; k0 += BK) {
        __syncthreads();
        // ---- A: 128 rows x 32 k split into both digit planes; B: both planes, 64 columns x 32 k
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = tid + e * NT, r = idx >> 3, g = idx & 7;
            const int mt = r >> 4, rr = r & 15;
            const int reg = (rr >> 3) + ((g >> 2) << 1), ln = ((rr & 7) << 2) + (g & 3);
            uint32_t d[2];
            pdigits4(xr[e], q, pb, ip, d);
            sA[0][mt][ln][reg] = d[0];
            sA[1][mt][ln][reg] = d[1];
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int idx = tid + e * NT, cidx = idx >> 3, g = idx & 7;
                sB[u][cidx >> 3][((cidx & 7) << 2) + (g & 3)][g >> 2] = br[u][e];
            }
        __syncthreads();
        if (k0 + BK < K) load(k0 + BK);
        // ---- MMA: x0 y0 into acc0, x0 y1 and x1 y0 into acc1
        uint4 a0[2], a1[2];
        uint2 b0[4], b1[4];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            a0[a] = *reinterpret_cast<const uint4 *>(&sA[0][wm * 2 + a][lane][0]);
            a1[a] = *reinterpret_cast<const uint4 *>(&sA[1][wm * 2 + a][lane][0]);
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            b0[b] = *reinterpret_cast<const uint2 *>(&sB[0][wn * 4 + b][lane][0]);
            b1[b] = *reinterpret_cast<const uint2 *>(&sB[1][wn * 4 + b][lane][0]);
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                mma_s8(acc0[a][b], a0[a], b0[b]);
                mma_s8(acc1[a][b], a0[a], b1[b]);
                mma_s8(acc1[a][b], a1[a], b0[b]);
            }
        // ---- end of a chunk of KC columns (or of K): R += (T_0 + p T_1) mod p^2, exact in int64
        if ((k0 + BK) % KC == 0 || k0 + BK >= K) {
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int64_t t = (int64_t)acc0[a][b][c] + (int64_t)pb * (int64_t)acc1[a][b][c];
                        R[a][b][c] = (uint32_t)add_mod(R[a][b][c], reduce_s64(t, q, r64), q);
                        acc0[a][b][c] = 0;
                        acc1[a][b][c] = 0;
                    }
        }
    }
    // ---- store (column-major output)
    const int g = lane >> 2, tq = lane & 3;
    uint64_t *Cl = p.C + (size_t)l * N * M;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint64_t row = m0 + (uint64_t)(wm * 2 + a) * 16 + g + (c >> 1) * 8;
                const uint64_t col = n0 + (uint64_t)(wn * 4 + b) * 8 + tq * 2 + (c & 1);
                if (row < M && col < N) Cl[col * M + row] = R[a][b][c];
            }
}

// Query planes: for each residue of the extended operand [L][N][K], digit planes (8) or
// centred residue planes (n_mod) in [L][P][N][Kp], zero padded to Kp.
template <int FORM>
__global__ void __launch_bounds__(256) k_planes(const uint64_t *op, int8_t *planes, uint64_t N, uint64_t K,
                                                uint64_t Kp, icm::I8Consts k) {
    const uint32_t l = blockIdx.y;
    const int P = FORM == 0 ? 8 : (FORM == 2 ? 2 : (int)k.n_mod);
    const uint64_t q = k.q[l];
    const uint64_t total = N * Kp;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t j = idx / Kp, kk = idx % Kp;
        const uint64_t v = kk < K ? op[((size_t)l * N + j) * K + kk] : 0;
        const uint64_t c = (v > (q >> 1)) ? v - q : v;
        const uint64_t y = c + 0x8080808080808080ull;
        int8_t *dst = planes + (size_t)l * P * N * Kp + idx;
        if (FORM == 0) {
#pragma unroll
            for (int t = 0; t < 8; ++t) dst[(size_t)t * N * Kp] = (int8_t)(((y >> (8 * t)) & 0xFF) ^ 0x80);
        } else if (FORM == 2) {
            int d0, d1;
            pdigits(v, q, k.pd[l], k.inv_p[l], d0, d1);
            dst[0] = (int8_t)d0;
            dst[(size_t)N * Kp] = (int8_t)d1;
        } else {
            const uint32_t dlo = (uint32_t)y ^ 0x80808080u, dhi = (uint32_t)(y >> 32) ^ 0x80808080u;
            for (int i = 0; i < P; ++i)
                dst[(size_t)i * N * Kp] = (int8_t)residue_from_digits(dlo, dhi, k.wlo[i], k.whi[i], k.mod[i], k.inv_m[i]);
        }
    }
}

}  // namespace

namespace icm {

cudaError_t launch_planes(int form, const I8Consts &k, const uint64_t *op, int8_t *planes, uint64_t N, uint64_t K,
                          uint64_t Kp, cudaStream_t st) {
    if (N == 0 || Kp == 0) return cudaSuccess;
    const uint64_t total = N * Kp;
    const unsigned blocks = (unsigned)std::min<uint64_t>((total + 255) / 256, 152u * 32u);
    dim3 grid(blocks, k.n_limbs);
    if (form == ICM_FORM_I8_P2) k_planes<2><<<grid, 256, 0, st>>>(op, planes, N, K, Kp, k);
    else k_planes<0><<<grid, 256, 0, st>>>(op, planes, N, K, Kp, k);
    return cudaGetLastError();
}

cudaError_t launch_ppmm_i8(int form, const I8Consts &k, const uint64_t *A, bool a_digits, const int8_t *Bp, uint64_t *C,
                           uint64_t M, uint64_t N, uint64_t K, uint64_t Kp, cudaStream_t st) {
    if (M == 0 || N == 0) return cudaSuccess;
    I8Args a{A, Bp, C, M, N, K, Kp, k, a_digits ? 1 : 0};
    if (form == ICM_FORM_I8_P2) {
        const uint64_t tiles = ((N + BN - 1) / BN) * ((M + BM - 1) / BM);
        if (tiles > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
        dim3 grid((unsigned)tiles, 1, k.n_limbs);
        k_ppmm_p2<<<grid, NT, 0, st>>>(a);
    } else {
        const cudaError_t attr =                         // per device: set at every launch
            cudaFuncSetAttribute(k_ppmm_digits, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DIG_SMEM);
        if (attr != cudaSuccess) return attr;
        dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), k.n_limbs);
        k_ppmm_digits<<<grid, NT, DIG_SMEM, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace icm

namespace icm {

namespace {
using u128 = unsigned __int128;
uint64_t mulmod_h(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)((u128)a * b % q); }
uint64_t powmod_h(uint64_t b, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    b %= q;
    while (e) { if (e & 1) r = mulmod_h(r, b, q); b = mulmod_h(b, b, q); e >>= 1; }
    return r;
}
uint64_t gcd_h(uint64_t a, uint64_t b) { while (b) { uint64_t t = a % b; a = b; b = t; } return a; }
// Inverse of a modulo m (gcd 1) by the extended Euclidean algorithm.
int64_t inv_h(int64_t a, int64_t m) {
    int64_t g = m, x = 0, x1 = 1, a1 = a % m;
    while (a1) { int64_t qq = g / a1, t = g - qq * a1; g = a1; a1 = t; t = x - qq * x1; x = x1; x1 = t; }
    return ((x % m) + m) % m;
}
uint64_t shoup_h(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }

// Greedy: the largest pairwise-coprime odd integers below 256, as many as the range needs.  Odd
// moduli keep every centred residue within [-127, 127], so a product is at most 127^2 = 16,129
// and 1024 products plus a reduced residue (|x| <= 1.5 m) stay below 2^24, the bound under which
// the fp16 forms' fp32 sums are exact (leaving out 256 costs no modulus for 50- and 60-bit primes).
// Fills mods and returns their count (0 if no set within ICM_MAX_MODULI covers the range); no
// allocation.
uint32_t crt_moduli(const uint64_t *q, size_t nq, uint64_t K, int (&mods)[ICM_MAX_MODULI]) {
    uint64_t qmax = 0;
    for (size_t i = 0; i < nq; ++i) qmax = q[i] > qmax ? q[i] : qmax;
    // |C| <= K ((qmax-1)/2)^2; need log2 M >= 1 + log2|C| + 2 (kappa margin: |C| / M <= 2^-3)
    const double need = 1.0 + std::log2((double)(K ? K : 1)) + 2.0 * std::log2((double)((qmax - 1) / 2 + 1)) + 2.0;
    uint32_t n = 0;
    double have = 0;
    for (int v = 255; v >= 3 && have < need && n < ICM_MAX_MODULI; v -= 2) {
        bool ok = true;
        for (uint32_t i = 0; i < n; ++i) if (gcd_h((uint64_t)v, (uint64_t)mods[i]) != 1) { ok = false; break; }
        if (ok) { mods[n++] = v; have += std::log2((double)v); }
    }
    return have < need ? 0 : n;
}
}  // namespace

uint32_t i8_planes(int form, const uint64_t *q, size_t nq, uint64_t K) {
    int mods[ICM_MAX_MODULI];
    return form == ICM_FORM_I8_DIGITS ? 8u : form == ICM_FORM_I8_P2 ? 2u : crt_moduli(q, nq, K, mods);
}

bool make_i8_consts(int form, const uint64_t *q, size_t nq, uint64_t K, I8Consts &k, const char **why) {
    k = I8Consts{};
    k.n_limbs = (uint32_t)nq;
    for (size_t l = 0; l < nq; ++l) {
        if (q[l] >= (1ull << 60)) { *why = "int8 forms need primes below 2^60 (8 balanced digits)"; return false; }
        k.q[l] = q[l];
        k.r64[l] = (uint64_t)(((u128)1 << 64) / q[l]);
        for (int s = 0; s < 15; ++s) { k.pw8[l][s] = powmod_h(2, 8ull * s, q[l]); k.pw8s[l][s] = shoup_h(k.pw8[l][s], q[l]); }
    }
    if (form == ICM_FORM_I8_P2) {
        // q = p^2 with odd 3 <= p <= 253: digits fit int8; weights 1 and p of the two passes
        for (size_t l = 0; l < nq; ++l) {
            const uint64_t pb = (uint64_t)std::llround(std::sqrt((double)q[l]));
            if (pb * pb != q[l] || pb < 3 || pb > 253 || !(pb & 1)) {
                *why = "the p^2 form needs moduli p^2 with odd 3 <= p <= 253";
                return false;
            }
            k.pd[l] = (int32_t)pb;
            k.inv_p[l] = 1.0f / (float)pb;
            k.pw8[l][0] = 1; k.pw8s[l][0] = shoup_h(1, q[l]);
            k.pw8[l][1] = pb; k.pw8s[l][1] = shoup_h(pb, q[l]);
        }
        k.n_mod = 0;
        return true;
    }
    if (form == ICM_FORM_I8_DIGITS) {
        // chunking keeps p * Kc * 2^14 <= 2^31 - 1 for every shift (p <= 8); nothing else to check
        k.n_mod = 0;
        return true;
    }
    // CRT form: every int32 accumulator sums K products of magnitude <= 2^14
    if (K * 16384ull > 2147483647ull) { *why = "K too deep for int32 accumulation of the CRT form (K <= 131071)"; return false; }
    int mods[ICM_MAX_MODULI];
    const uint32_t nm = crt_moduli(q, nq, K, mods);
    if (nm == 0) { *why = "no set of small moduli covers the product range"; return false; }
    k.n_mod = nm;
    for (uint32_t i = 0; i < nm; ++i) {
        const int m = mods[i];
        int w[8];
        for (int t = 0; t < 8; ++t) {
            int v = (int)powmod_h(256, (uint64_t)t, (uint64_t)m);
            if (v > (m - 1) / 2) v -= m;                   // centred
            w[t] = v;
        }
        k.mod[i] = m;
        k.wlo[i] = (int32_t)((uint32_t)(uint8_t)w[0] | ((uint32_t)(uint8_t)w[1] << 8) | ((uint32_t)(uint8_t)w[2] << 16) | ((uint32_t)(uint8_t)w[3] << 24));
        k.whi[i] = (int32_t)((uint32_t)(uint8_t)w[4] | ((uint32_t)(uint8_t)w[5] << 8) | ((uint32_t)(uint8_t)w[6] << 16) | ((uint32_t)(uint8_t)w[7] << 24));
        k.inv_m[i] = 1.0f / (float)m;
        const int h = m / 2;
        k.cbias[i] = m * ((131072 + m - 1) / m) + h;
        k.magic[i] = (uint32_t)(((1ull << 32) + (uint64_t)m - 1) / (uint64_t)m);
        const uint32_t hb = 0xE400u | (uint32_t)h;           // fp16 bits of -(1024 + h)
        k.hneg2[i] = hb | (hb << 16);
        // (M / m_i) mod m_i and its inverse
        uint64_t hat = 1;
        for (uint32_t j = 0; j < nm; ++j) if (j != i) hat = hat * (uint64_t)mods[j] % (uint64_t)m;
        k.yinv[i] = (int32_t)inv_h((int64_t)hat, m);
        k.r19[i] = (uint32_t)((((uint64_t)k.yinv[i] << 19) + (uint64_t)m / 2) / (uint64_t)m);
        for (size_t l = 0; l < nq; ++l) {
            uint64_t W = 1 % q[l];
            for (uint32_t j = 0; j < nm; ++j) if (j != i) W = mulmod_h(W, (uint64_t)mods[j], q[l]);
            k.W[l][i] = W;
            k.Ws[l][i] = shoup_h(W, q[l]);
            k.Wy[l][i] = mulmod_h((uint64_t)k.yinv[i], W, q[l]);
        }
    }
    for (size_t l = 0; l < nq; ++l) {
        uint64_t Mq = 1 % q[l];
        for (uint32_t j = 0; j < nm; ++j) Mq = mulmod_h(Mq, (uint64_t)mods[j], q[l]);
        k.Mq[l] = Mq;
        k.Mqs[l] = shoup_h(Mq, q[l]);
    }
    return true;
}

}  // namespace icm
