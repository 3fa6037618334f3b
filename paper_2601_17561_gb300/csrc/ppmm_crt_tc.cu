// Phase 1 of the fp16 small-modulus CRT product on the tcgen05 tensor cores (Blackwell 5th-gen
// MMA with accumulators in tensor memory).  Same arithmetic as k_crt_p1<fp16> (ppmm_crt.cu):
// for one (limb, database chunk, 128-row tile, modulus m_i, 512-column round) it computes
// c_i = (sum_k a[k] b[k]) mod m_i over residues held exactly in fp16 (|r| <= 127), accumulating
// in fp32 TMEM (two 256-column accumulators, one per column tile, all 512 columns) and
// reducing the accumulators modulo m_i every 1024 columns of K so that they stay exact integers
// below 2^24 (odd moduli: |r| <= 127, 1024 * 127^2 + 1.5 * 255 < 2^24); c_i goes to the byte
// scratch that phase 2 (k_crt_combine) recombines.
//
// One modulus on 512 columns: each raw database slab is loaded and converted once for two MMAs
// (N = 256 each) that share the converted operand, so every residue the converters compute
// feeds 512 columns.  (Two moduli on 256 columns each read the raw slab as often but convert it
// twice: the conversion, integer work on the CUDA cores, was what bounded that layout.)
//
// Block: 16 or 8 converter warps, 2 MMA issuer warps, 2 TMA producer warps; K advances in slabs
// of 16.
//  * Raw producer: one TMA load per slab of the 128 x 16 balanced-digit storage words of the
//    database rows (128-byte swizzle: the 16-byte chunk c of row r sits at chunk c ^ (r mod 8)),
//    into a ring of RS raw slots ("rawfull" / "rawempty" mbarriers).
//  * Query producer: per slab, one bulk copy per modulus of the query's 8 KB residue block (the
//    planes are stored pre-tiled in the MMA's K-major core-matrix layout, so a 256 x 16 operand is
//    one contiguous block: 64 requests of 128 bytes, where a row-by-row tensor load of 32-byte rows
//    needs 256) for each of the two column tiles into the B half of a ring of S operand slots.  It
//    arrives on the slot's "full" mbarrier with the expected byte count, so "full" completes when
//    the converters have written the A half and the B bytes have landed; the MMA issuers release
//    the slot through "empty".
//  * Converters: warps w, w + 4, w + 8 and w + 12 own operand slot w and raw slots w and w + 4, and
//    convert every slab g with g mod 4 = w, 32 rows each: 8 consecutive storage words of a row become 8 fp16
//    residues (two dp4a and a multiply-high division per residue, an f16x2 add per pair; no
//    conversion-pipe instructions), written to the A half of the slot (K-major, no swizzle, 8-row
//    x 16-byte core matrices).  Every quarter-warp reads 8 distinct bank groups of the swizzled
//    raw slot and writes 128 contiguous bytes.  The conversion is latency-bound integer work, so
//    four warps per scheduler (rather than two) keep the integer pipes fed.
//  * MMA: two issuing threads in different warps, one per 256-column tile (their accumulators are
//    independent), each issue one tcgen05.mma (M = 128, N = 256, K = 16) per slab and commit to
//    the slot's "empty" mbarrier (count 2).  Splitting the issue halves the per-slab control work
//    on each thread, which bounded the single-issuer loop.  Every 64 slabs and at the end of a tile it
//    commits to "acc_full"; the converters (warp w serves TMEM lane quarter w mod 4 and columns
//    128 floor(w / 4) .. + 127 of the 512 accumulator columns) reduce the accumulators in place
//    (tcgen05.ld / st) or write the final residues, and arrive on "acc_free".
//
// Every wait is bounded by %globaltimer (2 s); on expiry the block records ICM_DEV_TIMEOUT in the
// device status word, stops issuing work, waits (bounded) for its own MMAs and TMA loads, and
// frees its TMEM.
#include "icm_internal.h"
#include "ppmm_i8.h"

#include <algorithm>
#include <cuda.h>
#include <cuda_fp16.h>
#include <mutex>

namespace {

constexpr int BM = 128, BN = 256, KS = 16;
constexpr int MAX_RING = 8;                       // deepest operand or raw ring of any variant
constexpr int FLUSH_SLABS = 64;                   // 1024 columns of K between reductions
constexpr int A_STAGE = BM * KS * 2;              // 4 KB
constexpr int B_STAGE = BN * KS * 2;              // 8 KB per column tile
constexpr int RAW_STAGE = BM * KS * 8;            // 16 KB
constexpr uint32_t TMEM_COLS = 512;               // two 256-column fp32 accumulators
constexpr uint64_t WAIT_NS = 2000000000ull;       // bound of every wait
// Shared memory of a ring configuration (S operand slots: A residues + B planes of 2 column
// tiles; RS raw database slots): raw slots first (1024-byte aligned for the 128-byte swizzle),
// then the B halves of the operand slots (column tile 0 then 1), the A halves, then the mbarriers.
template <int S, int RS>
struct Ring {
    static constexpr int OFF_B = RS * RAW_STAGE;
    static constexpr int OFF_A = OFF_B + S * 2 * B_STAGE;
    static constexpr int BARS = OFF_A + S * A_STAGE;
    static constexpr int SMEM = BARS + 2048;      // + barriers + slack to align the base to 1024
    static_assert(SMEM <= 227 * 1024, "shared memory budget");
    static_assert(OFF_B % 1024 == 0 && OFF_A % 1024 == 0, "stage alignment");
    static_assert(S <= MAX_RING && RS <= MAX_RING, "barrier arrays");
    // raw slot g mod RS must always be consumed by the converters of operand slot g mod S: a warp
    // may only wait for the next parity of a barrier whose previous phase it consumed itself (a
    // waiter two phases ahead would see the parity it waits for as already complete)
    static_assert(RS % S == 0, "each raw slot belongs to one operand slot's converters");
};
// Progress bound between blocks (kernel option): blocks publish how many windows of SYNC_W slabs
// they have issued, and no block starts a window more than SYNC_LAG windows ahead of the slowest.
constexpr int SYNC_W = 64, SYNC_LAG = 2;
static_assert(icm::CRT_PROGRESS_BYTES >= 1024 * 4, "progress words for up to 1024 blocks");
constexpr uint64_t NCHUNK = 512;

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
    uint64_t N, K, n0, nch;
    uint32_t n_mod;
    uint32_t two;                     // the round has a second 256-column tile (nch > 256)
    uint64_t n_tiles;                 // L x row tiles x moduli
    uint32_t *prog;                   // per-block progress words (progress bound), zeroed per launch
    uint32_t pt0[ICM_MAX_CHUNKS + 1]; // prefix sums of 256-row pair tiles per chunk (2-SM variant)
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
// non-blocking probe with cluster-scope acquire
__device__ __forceinline__ bool mbar_test_cl(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// Bounded wait of the kernel's roles.  In the 2-SM form phases are completed by the other block
// of the pair (relayed arrivals, multicast commits): those waits poll with test_wait and
// cluster-scope acquire instead of suspending in try_wait.
template <bool CL>
__device__ __forceinline__ bool mbar_wait_s(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    if (!CL) return mbar_wait(bar, parity, abort_flag);
    if (mbar_test_cl(bar, parity)) return true;
    const uint64_t t0 = gtime();
    for (;;) {
        if (mbar_test_cl(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtime() - t0 > WAIT_NS) {
            *abort_flag = 1;
            atomicExch(&g_status, (uint32_t)ICM_DEV_TIMEOUT);
            return false;
        }
    }
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// every thread of both blocks of the pair: release this block's prior work, acquire the peer's
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// arrive (release, cluster scope) on the mbarrier at the same offset in block `rank` of the cluster
__device__ __forceinline__ void mbar_arrive_remote(uint64_t *bar, uint32_t rank) {
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_u32(bar)), "r"(rank));
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" :: "r"(ra) : "memory");
}

// Bounded wait that ignores the abort flag (drains this block's own copies before it exits).
__device__ __forceinline__ void mbar_wait_drain(uint64_t *bar, uint32_t parity) {
    const uint64_t t0 = gtime();
    while (!mbar_try(bar, parity))
        if (gtime() - t0 > WAIT_NS) {
            atomicExch(&g_status, (uint32_t)ICM_DEV_TIMEOUT);
            return;
        }
}

// TMA tile loads into this block's shared memory, completing on an mbarrier.
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
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t swz) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)swz << 61);
}
// Instruction descriptor, kind::f16: D = f32 [4,6), A = B = f16 [7,10) [10,13), both K-major,
// N >> 3 [17,23), M >> 4 [24,29).
constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(d_tmem), "l"(a), "l"(b), "r"(IDESC), "r"(accumulate) : "memory");
}
// 2-SM form (cta_group::2, issued by the leader block of a pair): M = 256, rows 0-127 from the
// leader's shared memory and TMEM, rows 128-255 from the peer's; B's columns 0-127 from the
// leader's shared memory, 128-255 from the peer's, at the same offsets.
constexpr uint32_t IDESC2 = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);
__device__ __forceinline__ void umma2(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(d_tmem), "l"(a), "l"(b), "r"(IDESC2), "r"(accumulate) : "memory");
}
// arrive on the mbarrier at this offset in both blocks of the pair once the MMAs complete
__device__ __forceinline__ void umma_commit2_both(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
                 :: "r"(smem_u32(bar)), "h"((uint16_t)3) : "memory");
}
__device__ __forceinline__ void umma_commit2_self(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(bar)) : "memory");
}

#define LD32_REGS                                                                                   \
    "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25," \
    "%26,%27,%28,%29,%30,%31}"
// 32 columns of 32-bit TMEM words per thread (lane quarter of the warp), without the wait: several
// loads can be in flight before one tcgen05.wait::ld
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

struct __align__(8) Bars {
    uint64_t rawfull[MAX_RING], rawempty[MAX_RING], full[MAX_RING], empty[MAX_RING], acc_full, acc_free, done;
    uint32_t tmem;
    int abort_flag;
};
static_assert(sizeof(Bars) <= 1024, "barrier block");

struct TileCoord {
    uint32_t l, c, mi;                // limb, chunk, modulus
    uint64_t m0, M;
};
// PAIR: tiles are 256-row pair tiles; block `rank` of the pair takes rows 128 rank .. + 127.
template <bool PAIR>
__device__ __forceinline__ TileCoord tile_coord(const TcArgs &p, uint64_t tile, uint32_t rank) {
    TileCoord t;
    uint64_t tt = tile;
    t.mi = (uint32_t)(tt % p.n_mod); tt /= p.n_mod;
    const uint32_t *t0 = PAIR ? p.pt0 : p.tab.mt0;
    const uint32_t mt_total = t0[p.tab.n];
    const uint32_t mtg = (uint32_t)(tt % mt_total);
    t.l = (uint32_t)(tt / mt_total);
    uint32_t c = 0;
    while (c + 1 < p.tab.n && mtg >= t0[c + 1]) ++c;
    t.c = c;
    t.M = p.tab.M[c];
    t.m0 = PAIR ? (uint64_t)(mtg - t0[c]) * (2 * BM) + rank * BM : (uint64_t)(mtg - t0[c]) * BM;
    return t;
}

// Converter warps w, w + 4, w + 8 and w + 12 convert slab g (g mod 4 = w) together, 32 rows each,
// using operand slot w and raw slot g mod 8; each warp meets its slots' phases in order.  The MMA
// thread issues one MMA per modulus and slab.
//
// NWC: converter warps (16: four per scheduler, register-capped at 96; 8: two per scheduler).
// SYNC: bound the drift between blocks (see SYNC_W); the blocks that share a database row tile,
// and those that share a modulus's query planes, then read each slab from L2 within a few
// windows of one another instead of re-reading it from HBM.  Needs every block resident (the
// launch is cooperative).
// PAIR: 2-SM MMA over a cluster of two blocks (M = 256): each block converts its own 128 rows and
// loads half of every query tile (128 columns); the leader (rank 0) issues the MMAs for both; a
// relay thread in the peer forwards its "full" phases to the leader's "full" barrier; the
// leader's commits go to both blocks; the peer's converters arrive on the leader's "acc_free".
// S, RS: operand and raw ring depths (more operand slots keep more MMAs in flight across the
// slot round trip: MMA completion -> converters -> MMA issue).
template <int NWC, bool SYNC, bool PAIR, int S, int RS>
__global__ void __launch_bounds__(NWC * 32 + 128, 1) k_crt_tc(const __grid_constant__ TcArgs p) {
    using RG = Ring<S, RS>;
    static_assert(!(SYNC && PAIR), "the progress bound is not combined with the 2-SM form");
    // warps: converters 0 .. NWC-1, MMA issuer of column tile 0, raw producer, query producer,
    // MMA issuer of column tile 1
    constexpr int W_MMA = NWC, W_RAW = NWC + 1, W_QRY = NWC + 2, W_MMA1 = NWC + 3;
    constexpr int WPS = NWC / S;                  // converter warps per operand slot
    constexpr int ROWS_W = BM / WPS;              // rows of a slab converted by one warp
    static_assert(NWC % S == 0 && ROWS_W % 16 == 0, "slot ownership");
    static_assert(NWC % 4 == 0 && NWC / 4 <= 16, "accumulator split over the lane quarters");
    // a warp performs the reduction after flush point f before it converts a slab past f + LAG;
    // a slab y can be converted while the MMA is blocked at f when its slot is free (y - S <= f)
    constexpr int LAG = S - 1;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the swizzle patterns are functions of shared-memory address bits: align the base to 1024
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *sR = smem;                          // [RS][RAW_STAGE]
    unsigned char *sB = smem + RG::OFF_B;              // [S][2][B_STAGE]
    unsigned char *sA = smem + RG::OFF_A;              // [S][A_STAGE]
    Bars *bars = reinterpret_cast<Bars *>(smem + RG::BARS);
    volatile int *abort_flag = &bars->abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t rank = PAIR ? cluster_rank() : 0u;                     // block of the pair
    const bool leader = rank == 0;
    // persistent tile loop: one tile sequence per block (or per pair)
    const uint64_t t_first = PAIR ? blockIdx.x / 2 : blockIdx.x, t_step = PAIR ? gridDim.x / 2 : gridDim.x;

    if (tid == 0) {
        for (int s = 0; s < RS; ++s) { mbar_init(&bars->rawfull[s], 1); mbar_init(&bars->rawempty[s], WPS); }
        for (int s = 0; s < S; ++s) {
            // converters + the query producer (+ the peer's relay at the leader of a pair)
            mbar_init(&bars->full[s], WPS + 1 + (PAIR && leader ? 1 : 0));
            mbar_init(&bars->empty[s], 2);
        }
        mbar_init(&bars->acc_full, 2);
        mbar_init(&bars->acc_free, PAIR && leader ? 2 * NWC : NWC);
        mbar_init(&bars->done, 2);
        bars->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        if constexpr (PAIR) {
            // one warp of each block of the pair allocates collectively
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;"
                         :: "r"(smem_u32(&bars->tmem)), "r"(TMEM_COLS) : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                         :: "r"(smem_u32(&bars->tmem)), "r"(TMEM_COLS) : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    // the peer's barriers are initialised before the leader's commits or the relay's arrivals
    if (PAIR) cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem = bars->tmem;

    const uint64_t K = p.K, N = p.N;
    const uint64_t nk = (K + KS - 1) / KS;
    const uint64_t Mall = p.tab.row0[p.tab.n];

    if (warp < W_MMA) {
        // ------------------------------------------------------------------ converter warps
        uint32_t acc_uses = 0;                   // acc_full completions consumed
        // TMEM lane quarter (a warp reaches lanes 32 (warp mod 4) ..) and this warp's share of the
        // 16 32-column chunks of the two accumulators (the NWC / 4 warps of a quarter split them)
        const uint32_t qtr = warp & 3, wq = (uint32_t)(warp >> 2);
        const uint32_t c_lo = wq * 16 / (NWC / 4), c_hi = (wq + 1) * 16 / (NWC / 4);
        const uint32_t slot = warp % S, sub = warp / S;                  // operand slot, row block
        const uint32_t trow = qtr * 32 + lane;                           // accumulator row of this thread
        // conversion map, item it: row sub*ROWS_W + it*16 + lrow, 16-byte chunks [4 cj, 4 cj + 4)
        // of the swizzled 128-byte raw row -> 16 bytes of residues per modulus; every quarter-warp
        // covers 8 consecutive rows with the same chunks (8 distinct bank groups)
        const uint32_t lrow = sub * ROWS_W + ((uint32_t)(lane >> 4) << 3) + (lane & 7);
        const uint32_t cj = (lane >> 3) & 1;
        const uint32_t rsw = lane & 7;                                   // = row mod 8 for every item
        const uint32_t a_off = (cj * 16 + (lrow >> 3)) * 128 + (lrow & 7) * 16;
        unsigned char *a_slot = sA + slot * A_STAGE + a_off;
        uint64_t g0 = 0;                         // global index of the tile's first slab
        // every loop decision below is warp-uniform (__all_sync), because drain() issues
        // warp-collective TMEM instructions
        auto go = [&]() { return __all_sync(0xffffffffu, *abort_flag == 0); };
        for (uint64_t tile = t_first; tile < p.n_tiles && go(); tile += t_step) {
            const TileCoord tc = tile_coord<PAIR>(p, tile, rank);
            const TcMod md = p.md[tc.mi];
            const float fm = (float)md.m;

            // the reduction (or final write) of this warp's part of the accumulators
            auto drain = [&](bool final) {
                const bool ok = __all_sync(0xffffffffu, mbar_wait_s<PAIR>(&bars->acc_full, acc_uses & 1, abort_flag));
                if (!ok) {
                    *abort_flag = 1;
                    return;
                }
                ++acc_uses;
                tc_fence_after();
                {
                    // LDP loads of 32 columns in flight per wait (two when registers allow: 8
                    // converter warps, 8 chunks each, pairs within one accumulator)
                    constexpr int LDP = NWC == 8 ? 2 : 1;
                    for (uint32_t c = c_lo; c < c_hi; c += LDP) {
                        if (c * 32 >= (uint32_t)BN && !p.two) break;        // the round has no second tile
                        uint32_t v[LDP][32];
#pragma unroll
                        for (int q = 0; q < LDP; ++q) tmem_ld32_nw(tmem + ((qtr * 32) << 16) + (c + q) * 32, v[q]);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                        for (int q = 0; q < LDP; ++q) {
                            const uint32_t col0 = (c + q) * 32;                  // column of the round
                            const uint32_t taddr = tmem + ((qtr * 32) << 16) + col0;
                            if (!final) {
                                // x - m round(x / m): the fma adds 1.5 2^23 to the exact x / m
                                // estimate and rounds once, which rounds it to an integer (|x / m| < 2^22)
#pragma unroll
                                for (int j = 0; j < 32; ++j) {
                                    const float x = __uint_as_float(v[q][j]);
                                    const float t = __fsub_rn(fmaf(x, md.inv_m, 12582912.0f), 12582912.0f);
                                    v[q][j] = __float_as_uint(fmaf(-fm, t, x));
                                }
                                tmem_st32(taddr, v[q]);
                            } else {
                                const uint64_t row = tc.m0 + trow;
                                uint8_t *Rl = p.R + ((size_t)tc.l * p.n_mod + tc.mi) * p.nch * Mall + p.tab.row0[tc.c];
#pragma unroll
                                for (int j = 0; j < 32; ++j) {
                                    const uint64_t col = col0 + j;
                                    if (row < tc.M && col < p.nch && p.n0 + col < N) {
                                        int val = __float2int_rn(__uint_as_float(v[q][j])) % md.m;
                                        val = val < 0 ? val + md.m : val;
                                        Rl[col * Mall + row] = (uint8_t)val;
                                    }
                                }
                            }
                        }
                    }
                    if (!final) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if (PAIR && !leader) mbar_arrive_remote(&bars->acc_free, 0);
                    else mbar_arrive(&bars->acc_free);
                }
            };

            uint64_t next_flush = FLUSH_SLABS - 1;                       // next reduction point to serve
            bool alive = true;
            for (uint64_t kt = (uint64_t)((slot + S - (uint32_t)(g0 % S)) % S); kt < nk; kt += S) {
                while (next_flush + 1 < nk && kt > next_flush + LAG) {
                    drain(false);
                    next_flush += FLUSH_SLABS;
                }
                const uint64_t g = g0 + kt;
                const uint32_t use = (uint32_t)(g / S);                   // uses of operand slot `slot`
                const uint32_t rslot = (uint32_t)(g % RS), ruse = (uint32_t)(g / RS);
                bool ok = mbar_wait_s<PAIR>(&bars->rawfull[rslot], ruse & 1, abort_flag);
                if (ok && use > 0) ok = mbar_wait_s<PAIR>(&bars->empty[slot], (use - 1) & 1, abort_flag);
                if (!__all_sync(0xffffffffu, ok)) {
                    *abort_flag = 1;
                    alive = false;
                    break;
                }
                const unsigned char *r_base = sR + rslot * RAW_STAGE + lrow * 128;
#pragma unroll
                for (int it = 0; it < ROWS_W / 16; ++it) {
                    const unsigned char *r_s = r_base + it * 16 * 128;
                    uint32_t w0[4];
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const ulonglong2 zz = *reinterpret_cast<const ulonglong2 *>(r_s + (((cj * 4 + h) ^ rsw) << 4));
                        w0[h] = res_pair(zz.x, zz.y, md.wlo, md.whi, md.cbias, md.magic, (uint32_t)md.m, md.hneg2);
                    }
                    *reinterpret_cast<uint4 *>(a_slot + it * 2 * 128) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
                }
                // residues written to this block's shared memory through the generic proxy are read
                // by the tensor cores (of this block, or of the pair's leader after the relay)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                // the warp barrier orders every lane's raw reads and residue writes before lane 0's
                // release of the raw slot and the operand slot
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&bars->rawempty[rslot]);
                    mbar_arrive(&bars->full[slot]);
                }
                if (!go()) { alive = false; break; }
            }
            if (!alive) break;
            // remaining reductions, then the final residues of the tile
            for (; next_flush + 1 < nk && go(); next_flush += FLUSH_SLABS) drain(false);
            if (go()) drain(true);
            g0 += nk;
        }
    } else if ((warp == W_MMA || warp == W_MMA1) && lane == 0) {
        // ------------------------------------------------------------------ MMA issuers (one thread each)
        if (PAIR && !leader) {
            // peer block of a pair: warp W_MMA relays each completed local "full" phase (its A
            // residues written, its query half landed) to the leader's "full" barrier
            if (warp == W_MMA) {
                uint32_t s = 0, u = 0;
                for (uint64_t tile = t_first; tile < p.n_tiles && !*abort_flag; tile += t_step) {
                    bool alive = true;
                    for (uint64_t kt = 0; kt < nk; ++kt) {
                        if (!mbar_wait_s<PAIR>(&bars->full[s], u & 1, abort_flag)) { alive = false; break; }
                        mbar_arrive_remote(&bars->full[s], 0);
                        if (++s == S) { s = 0; ++u; }
                    }
                    if (!alive) break;
                }
            }
        } else {
        const uint32_t j = warp == W_MMA ? 0u : 1u;                      // column tile of this issuer
        uint32_t s = 0, u = 0;
        uint32_t acc_commits = 0;
        bool wait_free = false;
        // descriptors of slot 0 (column tile 0); slot s adds s A_STAGE / 16 to A's start-address
        // field, and column tile j of slot s adds (2 s + j) B_STAGE / 16 to B's.  A pair's blocks
        // hold 128 columns of each tile: k 8-15 start 2 KB after k 0-7 instead of 4 KB.
        const uint64_t adesc0 = sdesc(smem_u32(sA), 2048, 128, 0),
                       bdesc0 = sdesc(smem_u32(sB), PAIR ? 2048 : 4096, 128, 0);
        // without a second column tile the second issuer only takes part in the slot and
        // reduction handshakes (its commits arrive at once)
        const bool issue = j == 0 || p.two != 0;
        const uint32_t dcol = j * BN;
        // one slab: wait for the slot, issue this tile's MMA, release the slot; at a reduction
        // point commit the accumulators and wait for the converters to hand them back
        auto slab = [&](uint32_t ss, uint32_t par, uint32_t kt, uint32_t &to_flush, bool last) -> bool {
            if (wait_free) {
                if (!mbar_wait_s<PAIR>(&bars->acc_free, (acc_commits - 1) & 1, abort_flag)) return false;
                wait_free = false;
            }
            if (!mbar_wait_s<PAIR>(&bars->full[ss], par, abort_flag)) return false;
            tc_fence_after();
            const uint64_t ad = adesc0 + (uint64_t)(ss * (A_STAGE >> 4));
            const uint64_t bd = bdesc0 + (uint64_t)((2 * ss + j) * (B_STAGE >> 4));
            if constexpr (PAIR) {
                if (issue) umma2(tmem + dcol, ad, bd, kt > 0 ? 1u : 0u);
                umma_commit2_both(&bars->empty[ss]);
            } else {
                if (issue) umma(tmem + dcol, ad, bd, kt > 0 ? 1u : 0u);
                umma_commit(&bars->empty[ss]);
            }
            if (--to_flush == 0 || last) {                               // a reduction point
                if constexpr (PAIR) umma_commit2_both(&bars->acc_full);
                else umma_commit(&bars->acc_full);
                ++acc_commits;
                wait_free = true;
                to_flush = FLUSH_SLABS;
            }
            return true;
        };
        const uint32_t nk32 = (uint32_t)nk;
        for (uint64_t tile = t_first; tile < p.n_tiles && !*abort_flag; tile += t_step) {
            bool alive = true;
            uint32_t to_flush = FLUSH_SLABS;                             // slabs to the next reduction
            if (nk32 % S == 0) {
                // whole ring passes (every tile starts at slot 0): slot indices, barrier addresses
                // and descriptor offsets are constants of the unrolled body
                for (uint32_t kt0 = 0; kt0 < nk32 && alive; kt0 += S, ++u) {
#pragma unroll
                    for (uint32_t ss = 0; ss < (uint32_t)S; ++ss)
                        if (alive) alive = slab(ss, u & 1, kt0 + ss, to_flush, kt0 + ss + 1 == nk32);
                }
            } else {
                for (uint32_t kt = 0; kt < nk32; ++kt) {
                    if (!slab(s, u & 1, kt, to_flush, kt + 1 == nk32)) { alive = false; break; }
                    if (++s == S) { s = 0; ++u; }
                }
            }
            if (!alive) break;
        }
        // make sure every MMA issued by this thread has completed before TMEM is freed
        if constexpr (PAIR) umma_commit2_self(&bars->done);
        else umma_commit(&bars->done);
        mbar_wait_drain(&bars->done, 0);
        }
    } else if (warp == W_RAW) {
        // ------------------------------------------------------------------ raw database producer
        // lane 0 issues the loads; the whole warp evaluates the progress bound
        uint32_t rs = 0, ur = 0;
        uint64_t issued = 0;
        const uint32_t wpt = (uint32_t)((nk + SYNC_W - 1) / SYNC_W);       // windows per tile
        uint32_t it = 0;                                                 // tiles begun by this block
        bool alive = true;
        for (uint64_t tile = t_first; alive && tile < p.n_tiles && !*abort_flag; tile += t_step, ++it) {
            const TileCoord tc = tile_coord<PAIR>(p, tile, rank);
            for (uint64_t kt = 0; kt < nk; ++kt) {
                if (SYNC && kt % SYNC_W == 0) {
                    const uint32_t gw = it * wpt + (uint32_t)(kt / SYNC_W);    // window about to start
                    if (lane == 0 && gw > 0) *(volatile uint32_t *)&p.prog[blockIdx.x] = gw;
                    if (gw > (uint32_t)SYNC_LAG) {
                        const uint64_t t0 = gtime();
                        for (;;) {
                            uint32_t lo = 0xFFFFFFFFu;
                            for (uint32_t b = lane; b < gridDim.x; b += 32)
                                lo = min(lo, *(volatile const uint32_t *)&p.prog[b]);
                            lo = __reduce_min_sync(0xffffffffu, lo);
                            if (lo >= gw - (uint32_t)SYNC_LAG) break;
                            if (__any_sync(0xffffffffu, *abort_flag != 0)) { alive = false; break; }
                            if (gtime() - t0 > WAIT_NS) {
                                if (lane == 0) { *abort_flag = 1; atomicExch(&g_status, (uint32_t)ICM_DEV_TIMEOUT); }
                                alive = false;
                                break;
                            }
                            __nanosleep(256);
                        }
                        if (!alive) break;
                    }
                }
                bool ok = true;
                if (lane == 0) {
                    ok = ur == 0 || mbar_wait_s<PAIR>(&bars->rawempty[rs], (ur - 1) & 1, abort_flag);
                    if (ok) {
                        mbar_expect_tx(&bars->rawfull[rs], RAW_STAGE);
                        tma_load_3d(smem_u32(sR + rs * RAW_STAGE), &p.tmA[tc.c], (int)(kt * KS), (int)tc.m0, (int)tc.l,
                                    &bars->rawfull[rs]);
                    }
                }
                if (!__shfl_sync(0xffffffffu, ok, 0)) { alive = false; break; }
                ++issued;
                if (++rs == RS) { rs = 0; ++ur; }
            }
        }
        // this block holds no one back any more
        if (SYNC && lane == 0) *(volatile uint32_t *)&p.prog[blockIdx.x] = 0xFFFFFFFFu;
        // every load issued by this thread has landed before the block exits
        if (lane == 0)
            for (uint64_t i = (issued > (uint64_t)RS ? issued - RS : 0); i < issued; ++i)
                mbar_wait_drain(&bars->rawfull[i % RS], (uint32_t)((i / RS) & 1));
    } else if (warp == W_QRY && lane == 0) {
        // ------------------------------------------------------------------ query plane producer
        uint32_t s = 0, u = 0;
        uint64_t issued = 0;
        for (uint64_t tile = t_first; tile < p.n_tiles && !*abort_flag; tile += t_step) {
            const TileCoord tc = tile_coord<PAIR>(p, tile, rank);
            // first block of this (limb, modulus) for the round's first 256-column tile; the second
            // tile's blocks follow Kp / 16 blocks later
            const size_t tstep = (size_t)(p.Kp / KS) * B_STAGE;
            const unsigned char *b_src = p.Bt + ((size_t)tc.l * p.n_mod + tc.mi) * p.plane + (size_t)(p.n0 / BN) * tstep;
            bool alive = true;
            for (uint64_t kt = 0; kt < nk; ++kt) {
                if (u > 0 && !mbar_wait_s<PAIR>(&bars->empty[s], (u - 1) & 1, abort_flag)) { alive = false; break; }
                unsigned char *b_s = sB + s * 2 * B_STAGE;
                if (PAIR) {
                    // this block's 128 columns of each tile: rows 16 rank .. + 15 of both k halves
                    constexpr uint32_t H = B_STAGE / 4;                  // 2 KB: 16 row groups x 128 bytes
                    mbar_expect_tx(&bars->full[s], p.two ? 4 * H : 2 * H);
                    for (uint32_t t = 0; t < (p.two ? 2u : 1u); ++t) {
                        const unsigned char *src = b_src + t * tstep + kt * B_STAGE + rank * H;
                        bulk_load(smem_u32(b_s + t * B_STAGE), src, H, &bars->full[s]);
                        bulk_load(smem_u32(b_s + t * B_STAGE + H), src + 2 * H, H, &bars->full[s]);
                    }
                } else {
                    mbar_expect_tx(&bars->full[s], p.two ? 2 * B_STAGE : B_STAGE);
                    bulk_load(smem_u32(b_s), b_src + kt * B_STAGE, B_STAGE, &bars->full[s]);
                    if (p.two) bulk_load(smem_u32(b_s + B_STAGE), b_src + tstep + kt * B_STAGE, B_STAGE, &bars->full[s]);
                }
                ++issued;
                if (++s == S) { s = 0; ++u; }
            }
            if (!alive) break;
        }
        // every load issued by this thread has landed before the block exits ("full" also needs
        // the converters' arrivals, which a normal run always makes)
        for (uint64_t i = (issued > (uint64_t)S ? issued - S : 0); i < issued; ++i)
            mbar_wait_drain(&bars->full[i % S], (uint32_t)((i / S) & 1));
    }
    tc_fence_before();
    __syncthreads();
    // a pair's leader has seen all its MMAs (which read the peer's shared memory and write the
    // peer's TMEM) complete before either block frees TMEM or exits
    if (PAIR) cluster_sync_all();
    tc_fence_after();
    if (warp == 0) {
        if constexpr (PAIR) asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS) : "memory");
        else asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS) : "memory");
    }
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

}  // namespace

namespace icm {

// kernel instantiations: variant -> (converter warps, progress bound, 2-SM, operand slots, raw slots)
#define ICM_TC_V1 16, false, false, 4, 8
#define ICM_TC_V2 16, true, false, 4, 8
#define ICM_TC_V3 8, false, false, 4, 8
#define ICM_TC_V4 8, true, false, 4, 8
#define ICM_TC_V5 8, false, true, 4, 8

cudaError_t crt_tc_set_attributes() {
    const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(k_crt_tc<ICM_TC_V1>, attr, Ring<4, 8>::SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_crt_tc<ICM_TC_V2>, attr, Ring<4, 8>::SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_crt_tc<ICM_TC_V3>, attr, Ring<4, 8>::SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_crt_tc<ICM_TC_V4>, attr, Ring<4, 8>::SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_crt_tc<ICM_TC_V5>, attr, Ring<4, 8>::SMEM);
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
    const int nwc = variant <= 2 ? 16 : 8;
    const bool sync = variant == 2 || variant == 4;
    const bool pair = variant == 5;
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
    // progress words after the residue scratch (crt_scratch_bytes reserves them)
    a.prog = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(scratch) +
                                          crt_scratch_main_bytes(k.n_limbs, k.n_mod, N, Mall));
    if (sms > 1024) return cudaErrorInvalidValue;
    a.N = N; a.K = K;
    a.n_mod = k.n_mod;
    a.pt0[0] = 0;
    for (uint32_t c = 0; c < tab.n; ++c) a.pt0[c + 1] = a.pt0[c] + (uint32_t)((tab.M[c] + 2 * BM - 1) / (2 * BM));
    for (uint32_t i = 0; i < k.n_mod; ++i)
        a.md[i] = TcMod{k.mod[i], k.wlo[i], k.whi[i], k.cbias[i], k.magic[i], k.hneg2[i], k.inv_m[i]};
    for (uint64_t n0 = 0; n0 < N; n0 += NCHUNK) {
        const uint64_t nch = std::min<uint64_t>(NCHUNK, N - n0);
        a.n0 = n0; a.nch = nch;
        a.two = nch > (uint64_t)BN ? 1u : 0u;
        a.n_tiles = (uint64_t)k.n_limbs * (pair ? a.pt0[tab.n] : tab.mt0[tab.n]) * k.n_mod;
        const uint64_t grid = std::min<uint64_t>(a.n_tiles, (uint64_t)sms);
        if (grid == 0) continue;
        cudaError_t e;
        if (sync) {
            // every block must be resident at once: a cooperative launch fails instead of stalling
            e = cudaMemsetAsync(a.prog, 0, grid * sizeof(uint32_t), st);
            if (e != cudaSuccess) return e;
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.gridDim = dim3((unsigned)grid);
            cfg.blockDim = dim3((unsigned)(nwc * 32 + 128));
            cfg.dynamicSmemBytes = Ring<4, 8>::SMEM;
            cfg.stream = st;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            e = nwc == 16 ? cudaLaunchKernelEx(&cfg, k_crt_tc<ICM_TC_V2>, a) : cudaLaunchKernelEx(&cfg, k_crt_tc<ICM_TC_V4>, a);
        } else if (pair) {
            // clusters of two blocks; as many pairs as can be resident, each running a sequence of
            // pair tiles
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 2;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.blockDim = dim3(8 * 32 + 128);
            cfg.dynamicSmemBytes = Ring<4, 8>::SMEM;
            cfg.stream = st;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            cfg.gridDim = dim3((unsigned)(2 * ((sms + 1) / 2)));
            int max_clusters = 0;
            e = cudaOccupancyMaxActiveClusters(&max_clusters, k_crt_tc<ICM_TC_V5>, &cfg);
            if (e != cudaSuccess) return e;
            if (max_clusters < 1) return cudaErrorInvalidConfiguration;
            const uint64_t n_cl = std::min<uint64_t>(a.n_tiles, (uint64_t)max_clusters);
            cfg.gridDim = dim3((unsigned)(2 * n_cl));
            e = cudaLaunchKernelEx(&cfg, k_crt_tc<ICM_TC_V5>, a);
        } else {
            if (nwc == 16) k_crt_tc<ICM_TC_V1><<<(unsigned)grid, 16 * 32 + 128, Ring<4, 8>::SMEM, st>>>(a);
            else k_crt_tc<ICM_TC_V3><<<(unsigned)grid, 8 * 32 + 128, Ring<4, 8>::SMEM, st>>>(a);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return e;
        e = launch_crt_combine(k, tab, scratch, N, n0, nch, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace icm
