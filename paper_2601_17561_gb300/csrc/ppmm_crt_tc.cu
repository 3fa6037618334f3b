// Phase 1 of the fp16 small-modulus CRT product on the tcgen05 tensor cores (Blackwell 5th-gen
// MMA with accumulators in tensor memory).  Same arithmetic as k_crt_p1<fp16> (ppmm_crt.cu):
// for one (limb, database chunk, 128-row tile, modulus m_i, column round of up to 512) it computes
// c_i = (sum_k a[k] b[k]) mod m_i over residues held exactly in fp16 (|r| <= 127), accumulating
// in fp32 TMEM (two 256-column accumulators, one per column tile) and reducing each accumulator
// modulo m_i at least every 1024 columns of K so that it stays an exact integer below 2^24 (odd
// moduli: 1024 * 127^2 + 128 < 2^24); c_i goes to the byte scratch that phase 2 (k_crt_combine)
// recombines.  One launch covers every column round of up to 1,024 query columns (the rounds are
// the slowest index of its persistent tile sequence), so a batch of up to 33 eyes is one launch
// and one combine.
//
// Pipeline of one persistent block (one per SM), K in slabs of 16, the stages decoupled by rings
// of shared-memory slots with "full" / "empty" mbarriers:
//  * raw producer (1 thread): one TMA load per slab of the 128 x 16 balanced-digit storage words
//    of the database rows (128-byte swizzle: the 16-byte chunk c of row r sits at chunk
//    c ^ (r mod 8)) into a ring of RS raw slots;
//  * converters (8 warps in NCG groups): the group of slab g (g mod NCG) converts it, each warp
//    128 / (8 / NCG) rows: 8 consecutive storage words of a row become 8 fp16 residues (two dp4a
//    and a multiply-high division per residue, an f16x2 add per pair) in registers, then, once the
//    operand slot is free, 16-byte stores into the MMA's K-major core-matrix layout (no swizzle);
//  * query producers (1 thread per 256-column tile): per slab one bulk copy of the pre-tiled 8 KB
//    fp16 plane block into the operand slot's B half of its tile;
//  * MMA issuers (1 thread per column tile): per slab one wait, one tcgen05.mma (M 128, N 256,
//    K 16) into the tile's accumulator and one commit.  An operand slot (A residues + both tiles'
//    B planes) has a "full" and an "empty" barrier per column tile, so each issuer waits once and
//    commits once per slab;
//  * epilogue (4 warps, one per TMEM lane quarter): reduces an accumulator in place
//    (tcgen05.ld / st) at its reduction points or writes the final residues.  The two tiles'
//    reduction points are staggered by half an interval (tile 1 at slabs 31, 95, ..., tile 0 at
//    63, 127, ...), so the tensor cores keep working on one tile while the other is reduced.
// In a round with a single column tile (the last round of a batch whose width is not a multiple
// of 512 may have one), the tile-1 producer arrives without a copy and the tile-1 issuer commits
// without an MMA, so the barrier counts stay those of the launch.
// Ring depths (measured at the paper shape on GB300): 8 raw slots (2 per converter group) and 4
// operand slots fill the 227 KB of shared memory; 4 raw slots (one per group) left the raw loads'
// latency exposed (~30% slower).
// Option SYNC (cooperative launch): the blocks start fetching the operands of their w-th tile
// only once every block has issued all fetches of its (w-1)-th tile.  The persistent tiles run in
// waves of one tile per SM (8 to 9 row tiles x 18 moduli at the paper shape); keeping the waves
// together keeps the database slabs (shared by the moduli of a row tile) and the query planes
// (shared by the row tiles of a modulus) in L2 between their readers instead of letting the
// blocks drift apart over ~2,000 tiles.
//
// Every wait is bounded by %globaltimer (a launch argument, default 2 s); on expiry the block
// records ICM_DEV_TIMEOUT in the device status word, stops issuing work, waits (bounded) for its
// own MMAs and copies in flight, and frees its TMEM.  A test-only launch flag makes the query
// producer of column tile 0 skip its copies, so that the MMA issuer's wait runs out.
#include "icm_internal.h"
#include "ppmm_i8.h"

#include <algorithm>
#include <cuda.h>
#include <cuda_fp16.h>
#include <mutex>

namespace {

constexpr int BM = 128, BN = 256, KS = 16;
constexpr int A_STAGE = BM * KS * 2;              // 4 KB
constexpr int B_STAGE = BN * KS * 2;              // 8 KB per column tile
constexpr int RAW_STAGE = BM * KS * 8;            // 16 KB
constexpr uint32_t TMEM_COLS = 512;               // two 256-column fp32 accumulators
constexpr int FLUSH = 64;                         // slabs (1024 columns of K) between reductions
constexpr int STAGGER = FLUSH / 2;                // offset of the second accumulator's reductions
constexpr int NCV = 8;                            // converter warps
constexpr int NEP = 8;                            // epilogue warps: NEP / 4 per TMEM lane quarter
constexpr int EP_COLS = BN / (NEP / 4);           // accumulator columns of one epilogue warp
// warps: converters, epilogue, raw database producer, query-plane producers of column tiles 0 and
// 1, MMA issuers of column tiles 0 and 1
constexpr int W_EPI = NCV, W_RAW = NCV + NEP, W_QRY = W_RAW + 1, W_MMA = W_QRY + 2;
constexpr int NTHREADS = (W_MMA + 2) * 32;        // 21 warps
constexpr uint64_t ROUND = 2 * BN;                // columns of one round (one block's accumulators)
constexpr uint64_t LAUNCH_COLS = 1024;            // columns of one launch (its rounds): the scratch width

// Shared memory of a ring configuration: raw slots first (1024-byte aligned for the 128-byte
// swizzle), then the B slots (column tile 0, then 1) and the A slots of the S operand slots, then
// the mbarriers.
template <int RS, int S>
struct Ring {
    static constexpr int OFF_B = RS * RAW_STAGE;
    static constexpr int OFF_A = OFF_B + 2 * S * B_STAGE;
    static constexpr int BARS = OFF_A + S * A_STAGE;
    static constexpr int SMEM = BARS + 1024 + 1024;   // barriers + slack to align the base to 1024
    static_assert(SMEM <= 227 * 1024, "shared memory budget");
    static_assert(OFF_B % 1024 == 0 && OFF_A % 1024 == 0, "stage alignment");
};

struct TcMod {
    int32_t m, wlo, whi, cbias;
    uint32_t magic, hneg2;
    float inv_m;
};

struct TcArgs {
    CUtensorMap tmA[ICM_MAX_CHUNKS];  // per chunk: [L][M_c][K] u64, box 16 x 128, 128-byte swizzle
    const unsigned char *Bt;          // fp16 planes, tiled (crt_f16_off): one 8 KB block per (tile, slab)
    uint64_t Kp, plane;               // padded K; bytes of one (limb, modulus) plane
    icm::ChunkTab tab;
    uint8_t *R;                       // [L][r][nch][sum M_c]
    uint64_t N, K, n0, nch;           // query columns; this launch's first column and its width
    uint32_t n_mod, n_limbs;
    uint32_t two;                     // some round of the launch has a second column tile (nch > 256)
    uint64_t n_tiles;                 // rounds x L x row tiles x moduli
    uint32_t *sync;                   // [0]: fetch arrivals (wave bound), [1]: a block gave up; zeroed per launch
    uint64_t wait_ns;                 // bound of every wait
    uint32_t inject_stall;            // test only: the query producer of tile 0 never copies
    TcMod md[ICM_MAX_MODULI];
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
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// Relaxed probe for the MMA issuers' operand waits: after a wait with the default acquire
// semantics, the next tcgen05.mma of the waiting thread is held until that thread's previous MMA
// has completed (one MMA per MMA latency instead of back to back; measured on GB300: 490 instead
// of 256 cycles for two M128 N256 K16 MMAs).  The operands need no acquire here: the converters
// publish their residues with fence.proxy.async before a release arrive, the query planes land
// through TMA completion, and the MMA is an async-proxy read ordered after the wait by
// tcgen05.fence::after_thread_sync.
__device__ __forceinline__ bool mbar_try_rlx(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.relaxed.cta.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ void give_up(volatile int *abort_flag, uint32_t *sync) {
    *abort_flag = 1;
    atomicExch(&g_status, (uint32_t)ICM_DEV_TIMEOUT);
    atomicExch(&sync[1], 1u);
}
// Bounded wait; false on timeout or when another thread of the block has given up.  RLX: relaxed
// probe (the MMA issuers' operand waits), else acquire.
template <bool RLX = false>
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, uint32_t *sync,
                                          uint64_t wait_ns) {
    if (RLX ? mbar_try_rlx(bar, parity) : mbar_try(bar, parity)) return true;
    const uint64_t t0 = gtime();
    for (;;) {
        if (RLX ? mbar_try_rlx(bar, parity) : mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtime() - t0 > wait_ns) {
            give_up(abort_flag, sync);
            return false;
        }
    }
}
// Bounded wait that ignores the abort flag (drains this block's own copies and MMAs before it
// frees TMEM and exits); gives up at the %globaltimer deadline shared by a whole drain.
__device__ __forceinline__ void mbar_wait_until(uint64_t *bar, uint32_t parity, uint64_t deadline) {
    while (!mbar_try(bar, parity))
        if (gtime() > deadline) {
            atomicExch(&g_status, (uint32_t)ICM_DEV_TIMEOUT);
            return;
        }
}

// TMA tile load into this block's shared memory, completing on an mbarrier.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, uint64_t *bar) {
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                 :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
                 : "memory");
}
// Bulk copy of `bytes` contiguous bytes (16-byte aligned) into this block's shared memory.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared memory matrix descriptor: start address >> 4 [0,14), leading byte offset >> 4 [16,30),
// stride byte offset >> 4 [32,46), version 1 [46,48), base offset 0, swizzle mode [61,64)
// (0: none).  K-major without swizzle: 8-row x 16-byte core matrices, the leading offset steps
// from k 0-7 to k 8-15, the stride offset from one group of 8 rows to the next.
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
// 32 columns of 32-bit TMEM words per thread (lane quarter of the warp), without the wait
__device__ __forceinline__ void tmem_ld32_nw(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 " LD32_REGS ", [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
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

// 16 columns of 32-bit TMEM words per thread (lane quarter of the warp), without the wait
__device__ __forceinline__ void tmem_ld16_nw(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
                    "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
                 : "memory");
}

// Residues modulo m of two balanced-digit storage words, as f16x2 bits, in integer arithmetic:
// v = sum_t d_t (256^t mod m) + c lies in [0, 2^19) (|sum| <= 2^17, c = m ceil(2^17 / m) + h),
// x = v - m floor(v / m) in [0, m) with the quotient from one multiply-high by ceil(2^32 / m)
// (exact because v (ceil(2^32/m) m - 2^32) < 2^32), so x - h = sum mod m with |x - h| <= 128.
// The f16 bits of 1024 + x are 0x6400 + x, and one f16x2 add of -(1024 + h) leaves x - h exactly.
__device__ __forceinline__ uint32_t res_pair(uint64_t z0, uint64_t z1, int wlo, int whi, int cb, uint32_t magic,
                                             uint32_t m, uint32_t hneg2) {
    const uint32_t v0 = (uint32_t)__dp4a((int)(uint32_t)(z0 >> 32), whi, __dp4a((int)(uint32_t)z0, wlo, cb));
    const uint32_t v1 = (uint32_t)__dp4a((int)(uint32_t)(z1 >> 32), whi, __dp4a((int)(uint32_t)z1, wlo, cb));
    const uint32_t x0 = v0 - __umulhi(v0, magic) * m, x1 = v1 - __umulhi(v1, magic) * m;
    const uint32_t bits = __byte_perm(x0, x1, 0x5410) + 0x64006400u;
    uint32_t out;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(out) : "r"(bits), "r"(hneg2));
    return out;
}

template <int RS, int S>
struct __align__(8) Bars {
    // raw slots; operand slots (A residues + the two column tiles' B planes): "full" and "empty" per
    // column tile, so each MMA issuer waits once and commits once per slab
    uint64_t rawfull[RS], rawempty[RS], full[2][S], empty[2][S];
    uint64_t accfull[2], accfree[2], done[2];
    uint32_t tmem;
    int abort_flag;
};

struct TileCoord {
    uint32_t l, c, mi;                // limb, chunk, modulus
    uint64_t m0, M;
    uint64_t col_base;                // first column of the tile's round (within the launch)
    uint32_t two;                     // the round has a second 256-column tile
};
// tile -> (round, limb, row tile, modulus), the modulus fastest and the round slowest
__device__ __forceinline__ TileCoord tile_coord(const TcArgs &p, uint64_t tile) {
    TileCoord t;
    uint64_t tt = tile;
    t.mi = (uint32_t)(tt % p.n_mod); tt /= p.n_mod;
    const uint32_t mt_total = p.tab.mt0[p.tab.n];
    const uint32_t mtg = (uint32_t)(tt % mt_total); tt /= mt_total;
    t.l = (uint32_t)(tt % p.n_limbs);
    t.col_base = (tt / p.n_limbs) * ROUND;
    uint32_t c = 0;
    while (c + 1 < p.tab.n && mtg >= p.tab.mt0[c + 1]) ++c;
    t.c = c;
    t.M = p.tab.M[c];
    t.m0 = (uint64_t)(mtg - p.tab.mt0[c]) * BM;
    t.two = p.nch > t.col_base + BN ? 1u : 0u;
    return t;
}
// Reduction points of accumulator j (column tile j) within a tile of nk slabs: after slab kt when
// (kt + 1 + STAGGER j) is a multiple of FLUSH, and the final write after the last slab.
__device__ __forceinline__ bool acc_event(uint32_t j, uint64_t kt, uint64_t nk) {
    return kt + 1 == nk || (kt + 1 + STAGGER * j) % FLUSH == 0;
}

// Wave bound (SYNC): wait until every block has issued all fetches of its (w-1)-th tile.  Each
// block's fetching threads (raw producer, the active query producers) add one to sync[0] per tile.
__device__ __forceinline__ bool wave_wait(const TcArgs &p, uint32_t w, volatile int *abort_flag) {
    if (w == 0) return true;
    const uint32_t need = (2u + p.two) * gridDim.x * w;
    const uint64_t t0 = gtime();
    for (;;) {
        if (*(volatile uint32_t *)&p.sync[0] >= need) return true;
        if (*abort_flag || *(volatile uint32_t *)&p.sync[1]) return false;
        if (gtime() - t0 > p.wait_ns) {
            give_up(abort_flag, p.sync);
            return false;
        }
        __nanosleep(200);
    }
}

template <int NCG, bool SYNC, int RS, int S>
__global__ void __launch_bounds__(NTHREADS, 1) k_crt_tc(const __grid_constant__ TcArgs p) {
    using RG = Ring<RS, S>;
    using BR = Bars<RS, S>;
    static_assert(sizeof(BR) <= 1024, "barrier block");
    // converter groups: a raw slot and an operand slot always belong to the same group (a warp
    // waits for the next parity of a barrier only after consuming its previous phase)
    constexpr int WPG = NCV / NCG, ROWS_W = BM / WPG, ITEMS = ROWS_W / 16;
    static_assert(NCV % NCG == 0 && ROWS_W % 16 == 0 && RS % NCG == 0 && S % NCG == 0, "converter groups");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the swizzle patterns are functions of shared-memory address bits: align the base to 1024
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *sR = smem;                          // [RS][RAW_STAGE]
    unsigned char *sB = smem + RG::OFF_B;              // [2][S][B_STAGE]
    unsigned char *sA = smem + RG::OFF_A;              // [S][A_STAGE]
    BR *bars = reinterpret_cast<BR *>(smem + RG::BARS);
    volatile int *abort_flag = &bars->abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint64_t wait_ns = p.wait_ns;
    const uint32_t two = p.two;                        // the tile-1 producer and issuer take part

    if (tid == 0) {
        for (int s = 0; s < RS; ++s) { mbar_init(&bars->rawfull[s], 1); mbar_init(&bars->rawempty[s], WPG); }
        for (int s = 0; s < S; ++s)
            for (int j = 0; j < 2; ++j) {
                // full: the converter warps of the slab's group + the query producer's arrival
                mbar_init(&bars->full[j][s], WPG + 1);
                // empty: the tile-j MMA issuer's commit
                mbar_init(&bars->empty[j][s], 1);
            }
        for (int j = 0; j < 2; ++j) {
            mbar_init(&bars->accfull[j], 1);
            mbar_init(&bars->accfree[j], NEP);
            mbar_init(&bars->done[j], 1);
        }
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

    const uint64_t nk = (p.K + KS - 1) / KS;
    const uint64_t Mall = p.tab.row0[p.tab.n];
    const uint64_t t_first = blockIdx.x, t_step = gridDim.x;   // persistent tile sequence

    if (warp < NCV) {
        // ------------------------------------------------------------------ converter warps
        // NCG groups of WPG warps; group grp converts the slabs g with g mod NCG = grp, so NCG
        // slabs are converted at once; each warp converts ROWS_W rows of its group's slabs.
        // item it: rows sub ROWS_W + 16 it + 8 (lane >> 4) + (lane & 7); 16-byte chunks
        // [4 cj, 4 cj + 4) of the swizzled 128-byte raw row (k 8 cj .. 8 cj + 7) -> 16 bytes of
        // residues; every quarter-warp covers 8 consecutive rows with the same chunks (8 distinct
        // bank groups)
        const uint32_t grp = (uint32_t)warp % NCG, sub = (uint32_t)warp / NCG;
        const uint32_t lrow0 = sub * ROWS_W + ((uint32_t)(lane >> 4) << 3) + (lane & 7);
        const uint32_t cj = (lane >> 3) & 1;
        const uint32_t rsw = lane & 7;                                   // = row mod 8
        const uint32_t a_off0 = cj * 2048 + (lrow0 >> 3) * 128 + (lrow0 & 7) * 16;
        uint64_t g0 = 0;                                                 // global index of the tile's first slab
        bool alive = true;
        for (uint64_t tile = t_first; alive && tile < p.n_tiles; tile += t_step, g0 += nk) {
            const TileCoord tc = tile_coord(p, tile);
            const TcMod md = p.md[tc.mi];
            for (uint64_t kt = (grp + NCG - (uint32_t)(g0 % NCG)) % NCG; kt < nk; kt += NCG) {
                const uint64_t g = g0 + kt;
                const uint32_t rs = (uint32_t)(g % RS), ru = (uint32_t)(g / RS);
                const uint32_t s = (uint32_t)(g % S), su = (uint32_t)(g / S);
                bool ok = mbar_wait(&bars->rawfull[rs], ru & 1, abort_flag, p.sync, wait_ns);
                if (!__all_sync(0xffffffffu, ok)) { alive = false; break; }
                const unsigned char *r_s = sR + rs * RAW_STAGE + lrow0 * 128;
                uint32_t w0[ITEMS][4];
#pragma unroll
                for (int it = 0; it < ITEMS; ++it)
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const ulonglong2 zz =
                            *reinterpret_cast<const ulonglong2 *>(r_s + it * 16 * 128 + (((cj * 4 + h) ^ rsw) << 4));
                        w0[it][h] = res_pair(zz.x, zz.y, md.wlo, md.whi, md.cbias, md.magic, (uint32_t)md.m, md.hneg2);
                    }
                // every lane's raw reads are complete (their values are consumed) before lane 0
                // releases the raw slot
                __syncwarp();
                if (lane == 0) mbar_arrive(&bars->rawempty[rs]);
                // the A slot is free once the MMAs of both column tiles that read it have completed
                if (su > 0) {
                    ok = mbar_wait(&bars->empty[0][s], (su - 1) & 1, abort_flag, p.sync, wait_ns);
                    if (ok && two) ok = mbar_wait(&bars->empty[1][s], (su - 1) & 1, abort_flag, p.sync, wait_ns);
                }
                if (!__all_sync(0xffffffffu, ok)) { alive = false; break; }
#pragma unroll
                for (int it = 0; it < ITEMS; ++it)
                    *reinterpret_cast<uint4 *>(sA + s * A_STAGE + a_off0 + it * 2 * 128) =
                        make_uint4(w0[it][0], w0[it][1], w0[it][2], w0[it][3]);
                // residues written through the generic proxy are read by the tensor cores
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&bars->full[0][s]);
                    if (two) mbar_arrive(&bars->full[1][s]);
                }
            }
        }
    } else if (warp < W_EPI + NEP) {
        // ------------------------------------------------------------------ epilogue warps
        const uint32_t qtr = (uint32_t)warp & 3;                          // TMEM lane quarter
        const uint32_t half = (uint32_t)(warp - W_EPI) >> 2;              // column part of the accumulator
        const uint32_t trow = qtr * 32 + lane;                            // accumulator row of this thread
        uint32_t ev[2] = {0, 0};                                          // accfull completions consumed
        bool alive = true;
        for (uint64_t tile = t_first; alive && tile < p.n_tiles; tile += t_step) {
            const TileCoord tc = tile_coord(p, tile);
            const TcMod md = p.md[tc.mi];
            const float fm = (float)md.m;
            // reduce (final = false) or write out (final = true) accumulator j
            auto handle = [&](uint32_t j, bool final) -> bool {
                const bool ok = __all_sync(0xffffffffu, mbar_wait(&bars->accfull[j], ev[j] & 1, abort_flag, p.sync, wait_ns));
                if (!ok) return false;
                ++ev[j];
                tc_fence_after();
                const uint32_t tbase = tmem + ((qtr * 32) << 16) + j * BN + half * EP_COLS;
                // x - m round(x / m): the fma adds 1.5 2^23 to the exact x / m estimate and rounds
                // once, which rounds it to an integer (|x / m| < 2^22); the result is an exact
                // integer in (-m, m)
                const uint64_t row = tc.m0 + trow;
                uint8_t *Rl = p.R + ((size_t)tc.l * p.n_mod + tc.mi) * p.nch * Mall + p.tab.row0[tc.c];
                auto emit = [&](uint32_t (&v)[16], uint32_t c) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float x = __uint_as_float(v[i]);
                        const float t = __fsub_rn(fmaf(x, md.inv_m, 12582912.0f), 12582912.0f);
                        v[i] = __float_as_uint(fmaf(-fm, t, x));
                    }
                    if (!final) {
                        tmem_st16(tbase + c * 16, v);
                        return;
                    }
                    const uint64_t col0 = tc.col_base + j * BN + half * EP_COLS + c * 16;   // column of the launch
                    uint8_t *dst = Rl + col0 * Mall + row;
                    if (row < tc.M && col0 + 16 <= p.nch && p.n0 + col0 + 16 <= p.N) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const float r = __uint_as_float(v[i]);
                            dst[i * Mall] = (uint8_t)__float2int_rn(r < 0.0f ? r + fm : r);
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (row < tc.M && col0 + i < p.nch && p.n0 + col0 + i < p.N) {
                                const float r = __uint_as_float(v[i]);
                                dst[i * Mall] = (uint8_t)__float2int_rn(r < 0.0f ? r + fm : r);
                            }
                    }
                };
                // 16 columns per load, the next load in flight while the current chunk is reduced
                uint32_t va[16], vb[16];
                tmem_ld16_nw(tbase, va);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                for (uint32_t c = 0; c < EP_COLS / 16; c += 2) {
                    tmem_ld16_nw(tbase + (c + 1) * 16, vb);
                    emit(va, c);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (c + 2 < EP_COLS / 16) tmem_ld16_nw(tbase + (c + 2) * 16, va);
                    emit(vb, c + 1);
                    if (c + 2 < EP_COLS / 16) asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                }
                if (!final) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bars->accfree[j]);
                return true;
            };
            // the issuers' reduction points in slab order (tile 1 at 31, 95, ..; tile 0 at 63, 127, ..)
            for (uint64_t e = STAGGER - 1; alive && e + 1 < nk; e += STAGGER) {
                const uint32_t j = (e + 1) % FLUSH == 0 ? 0u : 1u;
                if (j == 1 && !tc.two) continue;
                alive = handle(j, false);
            }
            if (alive) alive = handle(0, true);
            if (alive && tc.two) alive = handle(1, true);
        }
    } else if (warp == W_RAW) {
        // ------------------------------------------------------------------ raw database producer
        if (lane == 0) {
            uint64_t g = 0;
            uint32_t w = 0;
            bool alive = true;
            for (uint64_t tile = t_first; alive && tile < p.n_tiles; tile += t_step, ++w) {
                const TileCoord tc = tile_coord(p, tile);
                if (SYNC && !wave_wait(p, w, abort_flag)) break;
                for (uint64_t kt = 0; kt < nk; ++kt, ++g) {
                    const uint32_t rs = (uint32_t)(g % RS), ru = (uint32_t)(g / RS);
                    if (ru > 0 && !mbar_wait(&bars->rawempty[rs], (ru - 1) & 1, abort_flag, p.sync, wait_ns)) {
                        alive = false;
                        break;
                    }
                    mbar_expect_tx(&bars->rawfull[rs], RAW_STAGE);
                    tma_load_3d(smem_u32(sR + rs * RAW_STAGE), &p.tmA[tc.c], (int)(kt * KS), (int)tc.m0, (int)tc.l,
                                &bars->rawfull[rs]);
                }
                if (SYNC && alive) atomicAdd(&p.sync[0], 1u);
            }
            // every load issued by this thread has landed before the block exits
            const uint64_t deadline = gtime() + wait_ns;
            for (uint64_t i = (g > (uint64_t)RS ? g - RS : 0); i < g; ++i)
                mbar_wait_until(&bars->rawfull[i % RS], (uint32_t)((i / RS) & 1), deadline);
        }
    } else if (warp < W_MMA) {
        // ------------------------------------------------------------------ query plane producers
        const uint32_t j = (uint32_t)(warp - W_QRY);                     // column tile
        if (lane == 0 && (j == 0 || two)) {
            uint64_t g = 0, issued = 0;
            uint32_t w = 0;
            bool alive = true;
            const bool stall = j == 0 && p.inject_stall;
            // blocks of consecutive slabs of one column tile are adjacent; the tiles of a
            // (limb, modulus) plane are Kp / 16 blocks apart
            const size_t tstep = (size_t)(p.Kp / KS) * B_STAGE;
            for (uint64_t tile = t_first; alive && tile < p.n_tiles && !stall; tile += t_step, ++w) {
                const TileCoord tc = tile_coord(p, tile);
                if (SYNC && !wave_wait(p, w, abort_flag)) break;
                const bool copy = j == 0 || tc.two;                      // the round has this column tile
                const unsigned char *b_src = p.Bt + ((size_t)tc.l * p.n_mod + tc.mi) * p.plane +
                                             (size_t)((p.n0 + tc.col_base) / BN + j) * tstep;
                for (uint64_t kt = 0; kt < nk; ++kt, ++g) {
                    const uint32_t s = (uint32_t)(g % S), su = (uint32_t)(g / S);
                    // the slot's B half of this tile is free once its tile-j MMA has completed
                    if (su > 0 && !mbar_wait(&bars->empty[j][s], (su - 1) & 1, abort_flag, p.sync, wait_ns)) {
                        alive = false;
                        break;
                    }
                    if (copy) {
                        mbar_expect_tx(&bars->full[j][s], B_STAGE);
                        bulk_load(smem_u32(sB + (j * S + s) * B_STAGE), b_src + kt * B_STAGE, B_STAGE, &bars->full[j][s]);
                        ++issued;
                    } else {
                        mbar_arrive(&bars->full[j][s]);
                    }
                }
                if (SYNC && alive) atomicAdd(&p.sync[0], 1u);
            }
            // every copy issued by this thread has landed before the block exits ("full" also needs
            // the converters' arrivals, which a block that gave up may not make: one deadline bounds
            // the whole drain; the last S slabs are in the last tile, whose copies all ran)
            const uint64_t deadline = gtime() + wait_ns;
            const uint64_t first = issued > (uint64_t)S ? g - S : g - issued;
            for (uint64_t i = first; i < g; ++i)
                mbar_wait_until(&bars->full[j][i % S], (uint32_t)((i / S) & 1), deadline);
        }
    } else {
        // ------------------------------------------------------------------ MMA issuers (one thread per column tile)
        const uint32_t j = (uint32_t)(warp - W_MMA);
        if (lane == 0 && (j == 0 || two)) {
            // descriptors of slot 0; slot s adds s A_STAGE / 16 to A's start-address field and
            // s B_STAGE / 16 to B's
            const uint64_t adesc0 = sdesc(smem_u32(sA), 2048, 128);
            const uint64_t bdesc0 = sdesc(smem_u32(sB + j * S * B_STAGE), 4096, 128);
            const uint32_t dcol = j * BN;
            const uint32_t nk32 = (uint32_t)nk;
            uint32_t u = 0, s = 0;                                       // ring passes, slot
            uint32_t ev = 0;
            bool pending = false;                                        // accumulator handed to the epilogue
            bool alive = true;
            for (uint64_t tile = t_first; alive && tile < p.n_tiles; tile += t_step) {
                const bool mine = j == 0 || tile_coord(p, tile).two;     // the round has this column tile
                // one slab: wait for the slot (relaxed: see mbar_try_rlx), issue the MMA, release
                // the slot; at a reduction point commit the accumulator to the epilogue
                auto slab = [&](uint32_t ss, uint32_t par, uint32_t kt) -> bool {
                    if (pending) {
                        if (!mbar_wait(&bars->accfree[j], (ev - 1) & 1, abort_flag, p.sync, wait_ns)) return false;
                        pending = false;
                    }
                    if (!mbar_wait<true>(&bars->full[j][ss], par, abort_flag, p.sync, wait_ns)) return false;
                    tc_fence_after();
                    if (mine)
                        umma(tmem + dcol, adesc0 + (uint64_t)(ss * (A_STAGE >> 4)), bdesc0 + (uint64_t)(ss * (B_STAGE >> 4)),
                             kt > 0 ? 1u : 0u);
                    umma_commit(&bars->empty[j][ss]);
                    if (mine && acc_event(j, kt, nk32)) {
                        umma_commit(&bars->accfull[j]);
                        ++ev;
                        pending = true;
                    }
                    return true;
                };
                if (nk32 % S == 0) {
                    // whole ring passes (every tile starts at slot 0): slot indices, barrier
                    // addresses and descriptor offsets are constants of the unrolled body
                    for (uint32_t kt0 = 0; kt0 < nk32 && alive; kt0 += S, ++u) {
#pragma unroll
                        for (uint32_t ss = 0; ss < (uint32_t)S; ++ss)
                            if (alive) alive = slab(ss, u & 1, kt0 + ss);
                    }
                } else {
                    for (uint32_t kt = 0; kt < nk32; ++kt) {
                        if (!slab(s, u & 1, kt)) { alive = false; break; }
                        if (++s == S) { s = 0; ++u; }
                    }
                }
            }
            // every MMA issued by this thread has completed before TMEM is freed
            umma_commit(&bars->done[j]);
            mbar_wait_until(&bars->done[j], 0, gtime() + wait_ns);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS) : "memory");
}

// ---------------------------------------------------------------- host side

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda).
EncodeTiled encode_fn() {
    static std::once_flag once;
    static EncodeTiled fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(f);
    });
    return fn;
}

// kernel instantiations: variant -> (converter groups, wave bound, raw slots, operand slots)
#define ICM_TC_V1 4, false, 8, 4
#define ICM_TC_V2 4, true, 8, 4
#define ICM_TC_V3 4, false, 4, 8

template <int NCG, bool SYNC, int RS, int S>
cudaError_t launch_variant(const TcArgs &a, int sms, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)std::min<uint64_t>(a.n_tiles, (uint64_t)sms));
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = Ring<RS, S>::SMEM;
    cfg.stream = st;
    if (SYNC) {
        // every block must be resident at once: a cooperative launch fails instead of stalling
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, k_crt_tc<NCG, SYNC, RS, S>, a);
}

template <int NCG, bool SYNC, int RS, int S>
cudaError_t set_smem_attr() {
    return cudaFuncSetAttribute(k_crt_tc<NCG, SYNC, RS, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Ring<RS, S>::SMEM);
}

}  // namespace

namespace icm {

cudaError_t crt_tc_set_attributes() {
    cudaError_t e = set_smem_attr<ICM_TC_V1>();
    if (e == cudaSuccess) e = set_smem_attr<ICM_TC_V2>();
    if (e == cudaSuccess) e = set_smem_attr<ICM_TC_V3>();
    return e;
}

// The tcgen05 path needs an even K (tensor-map row strides are multiples of 16 bytes); the caller
// uses the mma.sync kernel otherwise.
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

cudaError_t launch_ppmm_crt_tc(const I8Consts &k, const ChunkTab &tab, const void *Bp, uint64_t N, uint64_t K,
                               uint64_t Kp, void *scratch, int variant, cudaStream_t st) {
    const uint64_t Mall = tab.row0[tab.n];
    if (Mall == 0 || N == 0) return cudaSuccess;
    if (!crt_tc_supported(K) || Kp % KS || !crt_tc_variant(variant)) return cudaErrorInvalidValue;
    EncodeTiled enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

    static_assert(sizeof(TcArgs) <= 32000, "kernel parameter space");
    TcArgs a{};
    // database chunks: [L][M_c][K] u64, box 16 words x 128 rows x 1 limb
    for (uint32_t c = 0; c < tab.n; ++c) {
        const cuuint64_t M = tab.M[c] ? tab.M[c] : 1;
        const cuuint64_t dims[3] = {K, M, k.n_limbs};
        const cuuint64_t strides[2] = {K * 8, M * K * 8};
        const cuuint32_t box[3] = {KS, BM, 1}, estr[3] = {1, 1, 1};
        if (enc(&a.tmA[c], CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<uint64_t *>(tab.A[c]), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    // query planes: tiled fp16 blocks (crt_f16_off), 16-byte aligned for the bulk copies
    if (reinterpret_cast<uintptr_t>(Bp) % 16) return cudaErrorInvalidValue;
    a.Bt = reinterpret_cast<const unsigned char *>(Bp);
    a.Kp = Kp;
    a.plane = crt_f16_ncols(N) * Kp * 2;
    a.tab = tab;
    a.R = reinterpret_cast<uint8_t *>(scratch);
    // wave counter and give-up word after the residue scratch (crt_scratch_bytes reserves them)
    a.sync = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(scratch) +
                                          crt_scratch_main_bytes(k.n_limbs, k.n_mod, N, Mall));
    a.N = N; a.K = K;
    a.n_mod = k.n_mod;
    a.n_limbs = k.n_limbs;
    a.wait_ns = k.tc_wait_ns ? k.tc_wait_ns : 2000000000ull;
    a.inject_stall = k.tc_inject_stall;
    for (uint32_t i = 0; i < k.n_mod; ++i)
        a.md[i] = TcMod{k.mod[i], k.wlo[i], k.whi[i], k.cbias[i], k.magic[i], k.hneg2[i], k.inv_m[i]};
    // one launch (all its 512-column rounds) and one combine per 1,024 columns
    for (uint64_t n0 = 0; n0 < N; n0 += LAUNCH_COLS) {
        const uint64_t nch = std::min<uint64_t>(LAUNCH_COLS, N - n0);
        a.n0 = n0; a.nch = nch;
        a.two = nch > (uint64_t)BN ? 1u : 0u;
        a.n_tiles = ((nch + ROUND - 1) / ROUND) * (uint64_t)k.n_limbs * tab.mt0[tab.n] * k.n_mod;
        if (a.n_tiles == 0) continue;
        cudaError_t e = cudaMemsetAsync(a.sync, 0, 2 * sizeof(uint32_t), st);
        if (e != cudaSuccess) return e;
        if (variant == 1) e = launch_variant<ICM_TC_V1>(a, sms, st);
        else if (variant == 2) e = launch_variant<ICM_TC_V2>(a, sms, st);
        else e = launch_variant<ICM_TC_V3>(a, sms, st);
        if (e != cudaSuccess) return e;
        e = launch_crt_combine(k, tab, scratch, N, n0, nch, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace icm
