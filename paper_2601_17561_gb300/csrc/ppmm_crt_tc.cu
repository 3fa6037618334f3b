// Phase 1 of the fp16 small-modulus CRT product on the tcgen05 tensor cores (Blackwell 5th-gen
// MMA with accumulators in tensor memory).  Same arithmetic as k_crt_p1<fp16> (ppmm_crt.cu):
// for one (limb, database chunk, 128-row tile, modulus m_i, 256-column tile) it computes
// c_i = (sum_k a[k] b[k]) mod m_i over centred residues held exactly in fp16, accumulating in fp32
// TMEM and reducing the accumulator modulo m_i every 512 columns of K so that it stays an exact
// integer below 2^24; c_i goes to the byte scratch that phase 2 (k_crt_combine) recombines.
//
// Block: 8 converter warps + 1 MMA warp.  A 4-stage ring in shared memory holds, per K-slab of 32,
//   A: 128 x 32 fp16 residues of the database rows (converted from the balanced-digit storage
//      words by the converter warps: two dp4a and one rounding step per residue),
//   B: 256 x 32 fp16 residue planes of the query (copied with cp.async),
// both in the K-major canonical layout without swizzle (8-row x 16-byte core matrices; LBO = byte
// step between core matrices along K, SBO = step between 8-row groups).  One elected thread of the
// MMA warp issues two tcgen05.mma (M = 128, N = 256, K = 16) per slab into a 256-column fp32 TMEM
// accumulator and commits to the stage's "empty" mbarrier.  Every 16 slabs, and at the end of a
// tile, it commits to "acc_full"; the converter warps (two per TMEM lane quarter, 128 columns
// each) then reduce the accumulator in place (tcgen05.ld / st) or write the final residues, and
// arrive on "acc_free".  The converters run S - 1 slabs ahead of the reductions, so the ring is
// full when the MMA thread resumes.
//
// Every wait is bounded by %globaltimer (2 s); on expiry the block records ICM_DEV_TIMEOUT in the
// device status word, stops issuing work, waits (bounded) for its own MMAs and frees its TMEM.
#include "icm_internal.h"
#include "ppmm_i8.h"

#include <algorithm>
#include <cuda_fp16.h>

namespace {

constexpr int BM = 128, BN = 256, KS = 32, S = 5, FLUSH_SLABS = 16;
constexpr int D = 2;                             // raw database slabs prefetched ahead (cp.async)
constexpr int RS = D + 1;                        // raw slab stages
constexpr int LAG = S - D;                       // accumulator reductions trail production by LAG slabs
constexpr int NCONV = 256;                       // converter threads (8 warps)
constexpr int NT = NCONV + 32;                   // + MMA warp
constexpr int A_STAGE = BM * KS * 2;             // 8 KB
constexpr int B_STAGE = BN * KS * 2;             // 16 KB
constexpr int RAW_STAGE = BM * KS * 8;           // 32 KB of balanced-digit words
constexpr uint32_t TMEM_COLS = 256;
constexpr uint64_t WAIT_NS = 2000000000ull;      // bound of every wait
// Shared memory: ring, mbarriers, TMEM address, abort flag.  The block opts in to the full
// 227 KB so that descriptor offsets stay inside its allocation under any stride reading.
constexpr int SMEM_RING = S * (A_STAGE + B_STAGE) + RS * RAW_STAGE;
constexpr int SMEM_BYTES = 227 * 1024;
constexpr uint64_t NCHUNK = 512;

struct TcArgs {
    icm::ChunkTab tab;
    const void *Bp;          // [L][r][N][Kp] fp16 planes
    uint8_t *R;              // [L][r][nch][sum M_c]
    uint64_t N, K, Kp, n0, nch;
    uint32_t n_ntile;
    uint64_t n_tiles;
    icm::I8Consts k;
};

// Device status word: ICM_DEV_TIMEOUT once any block gave up a bounded wait (read and cleared by
// icm_device_status).
__device__ uint32_t g_status;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" :: "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// Bounded wait; false on timeout or when another thread has aborted the block.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = gtime();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtime() - t0 > WAIT_NS) {
            *abort_flag = 1;
            atomicExch(&g_status, (uint32_t)ICM_DEV_TIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major canonical layout without swizzle: descriptor fields (bits): start address >> 4 [0,14),
// leading byte offset >> 4 [16,30), stride byte offset >> 4 [32,46), version 1 [46,48),
// base offset 0, layout type 0 (no swizzle) [61,64).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor, kind::f16: D = f32 [4,6), A = B = f16 [7,10) [10,13), both K-major,
// N >> 3 [17,23), M >> 4 [24,29).
constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(d_tmem), "l"(a), "l"(b), "r"(IDESC), "r"(accumulate) : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(bar)) : "memory");
}

#define LD32_REGS                                                                                   \
    "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25," \
    "%26,%27,%28,%29,%30,%31}"
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 " LD32_REGS ", [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
#define ST32_REGS                                                                                   \
    "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26," \
    "%27,%28,%29,%30,%31,%32}"
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], " ST32_REGS ";"
                 :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
                    "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
                    "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
                    "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
                 : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool pred) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(pred ? 16 : 0) : "memory");
}

// centred residue of a balanced-digit storage word modulo m (|r| <= m/2), as fp16 bits
__device__ __forceinline__ uint32_t res_half(uint64_t z, int m, int wlo, int whi, float inv_m) {
    int s = __dp4a((int)(uint32_t)z, wlo, 0);
    s = __dp4a((int)(uint32_t)(z >> 32), whi, s);
    const int r = s - m * __float2int_rn((float)s * inv_m);
    return (uint32_t)__half_as_ushort(__int2half_rn(r));
}

struct __align__(8) Bars {
    uint64_t full[S], empty[S], acc_full, acc_free, done;
    uint32_t tmem;
    int abort_flag;
};

__global__ void __launch_bounds__(NT, 1) k_crt_tc(TcArgs p) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem;                          // [S][A_STAGE]
    unsigned char *sB = smem + S * A_STAGE;            // [S][B_STAGE]
    unsigned char *sR = smem + S * (A_STAGE + B_STAGE); // [RS][RAW_STAGE]: raw slabs, per-thread chunks
    Bars *bars = reinterpret_cast<Bars *>(smem + SMEM_RING);
    volatile int *abort_flag = &bars->abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) { mbar_init(&bars->full[s], NCONV); mbar_init(&bars->empty[s], 1); }
        mbar_init(&bars->acc_full, 1);
        mbar_init(&bars->acc_free, NCONV);
        mbar_init(&bars->done, 1);
        bars->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&bars->tmem)), "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bars->tmem;

    const uint32_t r = p.k.n_mod;
    const uint32_t mt_total = p.tab.mt0[p.tab.n];
    const uint64_t N = p.N, K = p.K, Kp = p.Kp;
    const uint64_t nk = (K + KS - 1) / KS;
    const uint64_t Mall = p.tab.row0[p.tab.n];

    if (warp < NCONV / 32) {
        // ------------------------------------------------------------------ converter warps
        uint64_t g = 0;                 // global slab counter (ring position)
        uint32_t acc_uses = 0;          // acc_full completions consumed
        const uint32_t qtr = warp & 3, half = warp >> 2;                 // TMEM lane quarter, column half
        const uint32_t trow = qtr * 32 + lane;                           // accumulator row of this thread
        // every loop decision below is warp-uniform (__all_sync), because drain() issues
        // warp-collective TMEM instructions
        auto go = [&]() { return __all_sync(0xffffffffu, *abort_flag == 0); };
        for (uint64_t tile = blockIdx.x; tile < p.n_tiles && go(); tile += gridDim.x) {
            uint64_t tt = tile;
            const uint32_t nt = (uint32_t)(tt % p.n_ntile); tt /= p.n_ntile;
            const uint32_t mi = (uint32_t)(tt % r); tt /= r;
            const uint32_t mtg = (uint32_t)(tt % mt_total);
            const uint32_t l = (uint32_t)(tt / mt_total);
            uint32_t c = 0;
            while (c + 1 < p.tab.n && mtg >= p.tab.mt0[c + 1]) ++c;
            const uint64_t M = p.tab.M[c];
            const uint64_t m0 = (uint64_t)(mtg - p.tab.mt0[c]) * BM, nb = (uint64_t)nt * BN;
            const int m = p.k.mod[mi], wlo = p.k.wlo[mi], whi = p.k.whi[mi];
            const float inv_m = p.k.inv_m[mi], fm = (float)m;
            const uint64_t *Al = p.tab.A[c] + (size_t)l * M * K;
            const unsigned char *Bl = reinterpret_cast<const unsigned char *>(p.Bp) + (((size_t)l * r + mi) * N + p.n0) * Kp * 2;

            // the reduction (or final write) of the accumulator after slab f
            auto drain = [&](bool final) {
                // warp-uniform decision: the TMEM loads and stores below are warp-collective
                const bool ok = __all_sync(0xffffffffu, mbar_wait(&bars->acc_full, acc_uses & 1, abort_flag));
                if (!ok) {
                    *abort_flag = 1;
                    return;
                }
                ++acc_uses;
                tc_fence_after();
                for (int rnd = 0; rnd < 4; ++rnd) {
                    const uint32_t col0 = half * 128 + rnd * 32;
                    const uint32_t taddr = tmem + ((qtr * 32) << 16) + col0;
                    uint32_t v[32];
                    tmem_ld32(taddr, v);
                    if (!final) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            float x = __uint_as_float(v[j]);
                            x = fmaf(-fm, rintf(x * inv_m), x);
                            v[j] = __float_as_uint(x);
                        }
                        tmem_st32(taddr, v);
                    } else {
                        const uint64_t row = m0 + trow;
                        uint8_t *Rl = p.R + ((size_t)l * r + mi) * p.nch * Mall + p.tab.row0[c];
#pragma unroll 4
                        for (int j = 0; j < 32; ++j) {
                            const uint64_t col = nb + col0 + j;
                            if (row < M && col < p.nch && p.n0 + col < N) {
                                int val = __float2int_rn(__uint_as_float(v[j])) % m;
                                val = val < 0 ? val + m : val;
                                Rl[col * Mall + row] = (uint8_t)val;
                            }
                        }
                    }
                }
                if (!final) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                tc_fence_before();
                mbar_arrive(&bars->acc_free);
            };
            auto is_flush = [&](uint64_t f) { return ((f + 1) % FLUSH_SLABS) == 0 && f + 1 < nk; };

            // loads of slab kk (ring position gg): the raw database words of this thread's two
            // chunks into its raw stage, and the query planes of the slab into the ring stage
            auto issue = [&](uint64_t kk, uint64_t gg) -> bool {
                const uint32_t s = (uint32_t)(gg % S), u = (uint32_t)(gg / S);
                if (u > 0 && !__all_sync(0xffffffffu, mbar_wait(&bars->empty[s], (u - 1) & 1, abort_flag))) {
                    *abort_flag = 1;
                    return false;
                }
                const uint64_t k0 = kk * KS;
                unsigned char *r_s = sR + (gg % RS) * RAW_STAGE, *b_s = sB + s * B_STAGE;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int id = tid + e * NCONV, row = id >> 2, j = id & 3;
                    const uint64_t grow = m0 + row, kk8 = k0 + 8 * j;
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const bool ok = grow < M && kk8 + 2 * h < K;        // K is even: whole pair in range
                        const uint64_t *src = ok ? Al + grow * K + kk8 + 2 * h : Al;
                        cp_async16(smem_u32(r_s + id * 64 + h * 16), src, ok);
                    }
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int id = tid + e * NCONV, n = id >> 2, j = id & 3;
                    const bool ok = nb + n < p.nch && p.n0 + nb + n < N;
                    const unsigned char *src = Bl + (ok ? ((nb + n) * Kp + k0 + 8 * j) * 2 : 0);
                    cp_async16(smem_u32(b_s + (j * 32 + (n >> 3)) * 128 + (n & 7) * 16), src, ok);
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
                return true;
            };

            bool alive = true;
            for (uint64_t d = 0; d < (uint64_t)D && d < nk && alive; ++d) alive = issue(d, g + d);
            for (uint64_t kt = 0; kt < nk && alive; ++kt) {
                const uint64_t gg = g + kt;
                const uint32_t s = (uint32_t)(gg % S);
                if (kt + D < nk && !issue(kt + D, gg + D)) break;
                // slab kt's copies have landed once at most min(D, nk - 1 - kt) later groups are pending
                const uint64_t later = (nk - 1 - kt) < (uint64_t)D ? (nk - 1 - kt) : (uint64_t)D;
                if (later >= 2) asm volatile("cp.async.wait_group 2;" ::: "memory");
                else if (later == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
                else asm volatile("cp.async.wait_group 0;" ::: "memory");
                // convert this thread's raw chunks into fp16 residues in the ring stage
                const unsigned char *r_s = sR + (gg % RS) * RAW_STAGE;
                unsigned char *a_s = sA + s * A_STAGE;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int id = tid + e * NCONV, row = id >> 2, j = id & 3;
                    uint32_t w[4];
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const ulonglong2 zz = *reinterpret_cast<const ulonglong2 *>(r_s + id * 64 + h * 16);
                        w[h] = res_half(zz.x, m, wlo, whi, inv_m) | (res_half(zz.y, m, wlo, whi, inv_m) << 16);
                    }
                    *reinterpret_cast<uint4 *>(a_s + (j * 16 + (row >> 3)) * 128 + (row & 7) * 16) = make_uint4(w[0], w[1], w[2], w[3]);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&bars->full[s]);
                // reductions trail production by LAG slabs (the ring can run LAG slabs past a
                // reduction point before a load would wait on the blocked MMA thread)
                if (kt >= (uint64_t)LAG && is_flush(kt - LAG)) drain(false);
                alive = go();
            }
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            // remaining reductions, then the final residues of the tile
            for (uint64_t f = (nk >= (uint64_t)LAG ? nk - LAG : 0); f < nk && go(); ++f)
                if (is_flush(f)) drain(false);
            if (go()) drain(true);
            g += nk;
        }
    } else if (lane == 0) {
        // ------------------------------------------------------------------ MMA warp (one thread)
        uint64_t g = 0;
        uint32_t acc_commits = 0;
        bool wait_free = false;
        for (uint64_t tile = blockIdx.x; tile < p.n_tiles && !*abort_flag; tile += gridDim.x) {
            for (uint64_t kt = 0; kt < nk && !*abort_flag; ++kt, ++g) {
                const uint32_t s = (uint32_t)(g % S);
                const uint32_t u = (uint32_t)(g / S);
                if (wait_free) {
                    if (!mbar_wait(&bars->acc_free, (acc_commits - 1) & 1, abort_flag)) break;
                    wait_free = false;
                }
                if (!mbar_wait(&bars->full[s], u & 1, abort_flag)) break;
                tc_fence_after();
                const uint32_t a0 = smem_u32(sA + s * A_STAGE), b0 = smem_u32(sB + s * B_STAGE);
#pragma unroll
                for (int ks = 0; ks < 2; ++ks)
                    umma(tmem, sdesc(a0 + ks * 2 * 2048, 2048, 128), sdesc(b0 + ks * 2 * 4096, 4096, 128),
                         (kt > 0 || ks > 0) ? 1u : 0u);
                umma_commit(&bars->empty[s]);
                if ((((kt + 1) % FLUSH_SLABS) == 0 && kt + 1 < nk) || kt + 1 == nk) {
                    umma_commit(&bars->acc_full);
                    ++acc_commits;
                    wait_free = true;
                }
            }
        }
        // make sure every MMA issued by this thread has completed before TMEM is freed
        umma_commit(&bars->done);
        mbar_wait(&bars->done, 0, abort_flag);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace

namespace icm {

cudaError_t crt_tc_set_attributes() {
    return cudaFuncSetAttribute(k_crt_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
}

// The tcgen05 path needs an even K (16-byte loads of pairs of residues); the caller falls back to
// the mma.sync kernel otherwise.
bool crt_tc_supported(uint64_t K) { return K > 0 && K % 2 == 0; }

uint32_t device_status(bool clear) {
    uint32_t v = 0;
    if (cudaMemcpyFromSymbol(&v, g_status, sizeof(v)) != cudaSuccess) return 0xFFFFFFFFu;
    if (clear && v) {
        const uint32_t z = 0;
        cudaMemcpyToSymbol(g_status, &z, sizeof(z));
    }
    return v;
}

cudaError_t launch_ppmm_crt_tc(const I8Consts &k, const ChunkTab &tab, const void *Bp, uint64_t N, uint64_t K, uint64_t Kp,
                               void *scratch, cudaStream_t st) {
    const uint64_t Mall = tab.row0[tab.n];
    if (Mall == 0 || N == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (uint64_t n0 = 0; n0 < N; n0 += NCHUNK) {
        const uint64_t nch = std::min<uint64_t>(NCHUNK, N - n0);
        TcArgs a{};
        a.tab = tab; a.Bp = Bp; a.R = reinterpret_cast<uint8_t *>(scratch);
        a.N = N; a.K = K; a.Kp = Kp; a.n0 = n0; a.nch = nch;
        a.n_ntile = (uint32_t)((nch + BN - 1) / BN);
        a.n_tiles = (uint64_t)k.n_limbs * tab.mt0[tab.n] * k.n_mod * a.n_ntile;
        a.k = k;
        const uint64_t grid = std::min<uint64_t>(a.n_tiles, (uint64_t)sms);
        if (grid == 0) continue;
        k_crt_tc<<<(unsigned)grid, NT, SMEM_BYTES, st>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = launch_crt_combine(k, tab, scratch, N, n0, nch, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace icm
