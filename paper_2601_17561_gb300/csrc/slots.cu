// Slot-encoded database and normalisation of the scores (libicm).
//
// Section 2.2.1: Ecd_slot maps N/2 complex slot values z_j to the rounded real polynomial
// Delta * P of degree < N with P(zeta^(5^j)) = z_j, zeta = exp(I pi / N); Dcd inverts it.
// Section 2.3: the CCMM accepts a slot-encoded database matrix and returns results in the same
// encoding.  Algorithm 2: every result ciphertext is multiplied by the plaintext
// mu = Ecd((1 / ||m_q AND m_db||_1)_j) so that its slots hold <c'_q, c'_db> / ||m_q AND m_db||_1.
//
// One template per slot, in the slot's real part (block t holds templates t N/2 .. t N/2 + N/2 - 1);
// rounding is round-half-to-even of the fp64 value.
//
// Transforms.  With n = N/2, c_i = p_i + I p_{i+n} (i < n) and omega = zeta^4 = exp(2 pi I / n):
// since zeta^(n (4m+1)) = I for every slot root zeta^(4m+1), and the slot roots are exactly the
// zeta^(4m+1), m < n (5^j = 1 mod 4),
//     z_j = P(zeta^(4 m_j + 1)) = sum_i (c_i zeta^i) omega^(m_j i),   m_j = (5^j mod 2N - 1) / 4,
// a length-n complex DFT of the twisted coefficients c_i zeta^i.  Encoding is its inverse:
// c_i = zeta^-i (1/n) sum_m Z_m omega^(-m i) with Z_{m_j} = z_j.  Both run as one radix-2
// decimation-in-time FFT in shared memory (fp64), one transform per thread block at a time.
//
// Normalisation (ct (.) mu) multiplies both parts of every block of a result column by its mu in
// Z_q[X]/(X^N + 1) for each limb of Q (after the rescaling by Q'): negacyclic NTTs (Cooley-Tukey
// forward, Gentleman-Sande inverse, powers of a primitive 2N-th root psi in bit-reversed order,
// after Longa and Naehrig, CANS 2016), pointwise products, inverse NTTs.
#include <cmath>
#include <mutex>

#include "icm_internal.h"

namespace icm {

// ---------------------------------------------------------------- host tables

namespace {
using u128 = unsigned __int128;

uint64_t mulmod_h128(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)((u128)a * b % q); }
uint64_t powmod_h128(uint64_t b, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    b %= q;
    while (e) { if (e & 1) r = mulmod_h128(r, b, q); b = mulmod_h128(b, b, q); e >>= 1; }
    return r;
}
uint64_t shoup_h(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }
uint32_t bitrev(uint32_t x, uint32_t bits) {
    uint32_t r = 0;
    for (uint32_t i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}
}  // namespace

struct SlotTables {
    uint32_t N = 0, n = 0, logn = 0, Lq = 0;
    double2 *twist = nullptr;     // [n]   zeta^i
    double2 *tw = nullptr;        // [n/2] omega^k
    int32_t *pos = nullptr;       // [n]   m_j
    uint64_t *ntt = nullptr;      // [Lq][4][N] psi_rev, psi_rev Shoup, psi^-1 rev, psi^-1 rev Shoup
    uint64_t ninv[2] = {0, 0}, ninvs[2] = {0, 0};
    uint64_t q[2] = {0, 0}, rhi[2] = {0, 0}, rlo[2] = {0, 0};
    uint64_t q0inv_mod_q1 = 0;    // q_0^-1 mod q_1 (CRT of two limbs)
    ~SlotTables() {
        if (twist) cudaFree(twist);
        if (tw) cudaFree(tw);
        if (pos) cudaFree(pos);
        if (ntt) cudaFree(ntt);
    }
};

void free_slot_tables(SlotTables *t) { delete t; }

static std::mutex g_slot_mu;

// Tables of the slot transforms and NTTs for ring degree N_db and the limbs of Q (built once per
// context, on the context's device).
static const SlotTables *slot_tables(icm_ctx *c, std::string &why) {
    std::lock_guard<std::mutex> lk(g_slot_mu);
    if (c->slot_tab) return c->slot_tab;
    const uint32_t N = c->N_db, n = N / 2, Lq = c->p.n_limbs_q;
    uint32_t logn = 0;
    while ((1u << logn) < n) ++logn;
    auto *T = new (std::nothrow) SlotTables();
    if (!T) { why = "host allocation"; return nullptr; }
    T->N = N; T->n = n; T->logn = logn; T->Lq = Lq;
    std::vector<double2> twist(n), tw(n / 2 ? n / 2 : 1);
    std::vector<int32_t> pos(n);
    for (uint32_t i = 0; i < n; ++i) {
        const long double a = 3.14159265358979323846264338327950288L * (long double)i / (long double)N;
        twist[i] = make_double2((double)cosl(a), (double)sinl(a));
    }
    for (uint32_t k = 0; k < n / 2; ++k) {
        const long double a = 2.0L * 3.14159265358979323846264338327950288L * (long double)k / (long double)n;
        tw[k] = make_double2((double)cosl(a), (double)sinl(a));
    }
    uint64_t e = 1;
    for (uint32_t j = 0; j < n; ++j) {
        pos[j] = (int32_t)((e - 1) / 4);
        e = e * 5 % (2ull * N);
    }
    std::vector<uint64_t> ntt((size_t)Lq * 4 * N);
    uint32_t logN = logn + 1;
    for (uint32_t l = 0; l < Lq; ++l) {
        const uint64_t q = c->q[l];
        if ((q - 1) % (2ull * N)) { delete T; why = "primes must be 1 mod 2 N_db"; return nullptr; }
        // psi: a primitive 2N-th root of unity, g^((q-1)/2N) for a quadratic non-residue g
        uint64_t psi = 0;
        for (uint64_t g = 2; g < 1000 && !psi; ++g)
            if (powmod_h128(g, (q - 1) / 2, q) == q - 1) psi = powmod_h128(g, (q - 1) / (2ull * N), q);
        if (!psi || powmod_h128(psi, N, q) != q - 1) { delete T; why = "no primitive 2N-th root"; return nullptr; }
        const uint64_t ipsi = powmod_h128(psi, q - 2, q);
        uint64_t *pr = &ntt[((size_t)l * 4 + 0) * N], *prs = &ntt[((size_t)l * 4 + 1) * N];
        uint64_t *ir = &ntt[((size_t)l * 4 + 2) * N], *irs = &ntt[((size_t)l * 4 + 3) * N];
        uint64_t pw = 1, ipw = 1;
        for (uint32_t k = 0; k < N; ++k) {
            const uint32_t r = bitrev(k, logN);
            pr[r] = pw; prs[r] = shoup_h(pw, q);
            ir[r] = ipw; irs[r] = shoup_h(ipw, q);
            pw = mulmod_h128(pw, psi, q);
            ipw = mulmod_h128(ipw, ipsi, q);
        }
        T->ninv[l] = powmod_h128(N, q - 2, q);
        T->ninvs[l] = shoup_h(T->ninv[l], q);
        T->q[l] = q; T->rhi[l] = c->crt.rhi[l]; T->rlo[l] = c->crt.rlo[l];
    }
    if (Lq == 2) T->q0inv_mod_q1 = powmod_h128(c->q[0] % c->q[1], c->q[1] - 2, c->q[1]);
    cudaError_t err = cudaMalloc(&T->twist, n * sizeof(double2));
    if (err == cudaSuccess) err = cudaMalloc(&T->tw, tw.size() * sizeof(double2));
    if (err == cudaSuccess) err = cudaMalloc(&T->pos, n * sizeof(int32_t));
    if (err == cudaSuccess) err = cudaMalloc(&T->ntt, ntt.size() * sizeof(uint64_t));
    if (err == cudaSuccess) err = cudaMemcpy(T->twist, twist.data(), n * sizeof(double2), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(T->tw, tw.data(), tw.size() * sizeof(double2), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(T->pos, pos.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(T->ntt, ntt.data(), ntt.size() * sizeof(uint64_t), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) { delete T; why = cudaGetErrorString(err); return nullptr; }
    c->slot_tab = T;
    return T;
}

// ---------------------------------------------------------------- device helpers

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmul_conj(double2 a, double2 b) {      // a * conj(b)
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ uint32_t brev(uint32_t x, uint32_t bits) { return __brev(x) >> (32 - bits); }

// In-place radix-2 decimation-in-time FFT of n = 2^logn points in shared memory, input in
// bit-reversed order, output in natural order: X_m = sum_i x_i w^(m i) with w = omega (forward)
// or conj(omega) (inverse, unnormalised).  tw[k] = omega^k, k < n/2.  Ends with a barrier.
__device__ void fft_dit(double2 *d, const double2 *tw, uint32_t n, uint32_t logn, bool inverse) {
    for (uint32_t s = 1; s <= logn; ++s) {
        const uint32_t half = 1u << (s - 1), step = n >> s;
        for (uint32_t b = threadIdx.x; b < n / 2; b += blockDim.x) {
            const uint32_t j = b & (half - 1);
            const uint32_t i0 = ((b >> (s - 1)) << s) + j, i1 = i0 + half;
            double2 w = tw[j * step];
            if (inverse) w.y = -w.y;
            const double2 u = d[i0], v = cmul(d[i1], w);
            d[i0] = make_double2(u.x + v.x, u.y + v.y);
            d[i1] = make_double2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
}

// a * b mod q for a, b < q < 2^62, with R = floor(2^128 / q) = rhi 2^64 + rlo: the quotient
// estimate from the high words of x R / 2^128 is short by at most 4, so the remainder is below
// 5q < 2^64 and a few subtractions finish.
__device__ __forceinline__ uint64_t mulmod_r128(uint64_t a, uint64_t b, uint64_t q, uint64_t rhi, uint64_t rlo) {
    const uint64_t lo = a * b, hi = __umul64hi(a, b);
    const uint64_t qe = hi * rhi + __umul64hi(hi, rlo) + __umul64hi(lo, rhi);
    uint64_t r = lo - qe * q;
#pragma unroll 1
    for (int i = 0; i < 5 && r >= q; ++i) r -= q;
    return r;
}

// Negacyclic NTT of N = 2^logN residues in shared memory (forward: Cooley-Tukey with psi_rev,
// output in bit-reversed order; inverse: Gentleman-Sande with psi^-1 rev, input in bit-reversed
// order, scaled by N^-1).  Ends with a barrier.
__device__ void ntt_fwd(uint64_t *a, uint32_t N, const uint64_t *pr, const uint64_t *prs, uint64_t q) {
    for (uint32_t m = 1, t = N >> 1; m < N; m <<= 1, t >>= 1) {
        for (uint32_t b = threadIdx.x; b < N / 2; b += blockDim.x) {
            const uint32_t i = b / t, jj = b & (t - 1);
            const uint32_t j1 = 2 * i * t + jj, j2 = j1 + t;
            const uint64_t U = a[j1], V = mulmod_shoup(a[j2], pr[m + i], prs[m + i], q);
            a[j1] = add_mod(U, V, q);
            a[j2] = sub_mod(U, V, q);
        }
        __syncthreads();
    }
}
__device__ void ntt_inv(uint64_t *a, uint32_t N, const uint64_t *ir, const uint64_t *irs, uint64_t q, uint64_t ninv,
                        uint64_t ninvs) {
    for (uint32_t m = N, t = 1; m > 1; m >>= 1, t <<= 1) {
        const uint32_t h = m >> 1;
        for (uint32_t b = threadIdx.x; b < N / 2; b += blockDim.x) {
            const uint32_t i = b / t, jj = b & (t - 1);
            const uint32_t j1 = 2 * i * t + jj, j2 = j1 + t;
            const uint64_t U = a[j1], V = a[j2];
            a[j1] = add_mod(U, V, q);
            a[j2] = mulmod_shoup(sub_mod(U, V, q), ir[h + i], irs[h + i], q);
        }
        __syncthreads();
    }
    for (uint32_t j = threadIdx.x; j < N; j += blockDim.x) a[j] = mulmod_shoup(a[j], ninv, ninvs, q);
    __syncthreads();
}

__device__ __forceinline__ int tbit(const uint8_t *p, uint64_t b) { return (p[b >> 3] >> (b & 7)) & 1; }

// ---------------------------------------------------------------- kernels

struct EncDbArgs {
    const uint8_t *codes, *masks;   // [n_tpl][code_bits / 8]
    uint64_t n_tpl;
    uint32_t code_bits, d2, N, n, logn, n_blocks;
    double scale;                   // 2^log2_scale
    const double2 *twist, *tw;
    const int32_t *pos;
    int32_t *W;                     // [n_blocks N][d2], zero-filled beforehand
};

// Slot encoding of the database messages: one (block t, entry column k < code_bits) transform at
// a time per thread block.  Slot j of block t holds c' of template t n + j.
__global__ void __launch_bounds__(512) k_slot_db_encode(EncDbArgs a) {
    extern __shared__ double2 sm[];
    double2 *d = sm, *tw = sm + a.n;
    for (uint32_t k = threadIdx.x; k < a.n / 2; k += blockDim.x) tw[k] = a.tw[k];
    __syncthreads();
    const uint64_t total = (uint64_t)a.n_blocks * a.code_bits;
    const uint32_t tb = a.code_bits / 8;
    for (uint64_t x = blockIdx.x; x < total; x += gridDim.x) {
        const uint32_t t = (uint32_t)(x / a.code_bits), k = (uint32_t)(x % a.code_bits);
        for (uint32_t j = threadIdx.x; j < a.n; j += blockDim.x) {
            const uint64_t tpl = (uint64_t)t * a.n + j;
            int v = 0;
            if (tpl < a.n_tpl) {
                const int cb = tbit(a.codes + tpl * tb, k), mb = tbit(a.masks + tpl * tb, k);
                v = mb - 2 * (cb & mb);
            }
            d[brev((uint32_t)a.pos[j], a.logn)] = make_double2((double)v, 0.0);
        }
        __syncthreads();
        fft_dit(d, tw, a.n, a.logn, true);
        const double f = a.scale / (double)a.n;
        for (uint32_t i = threadIdx.x; i < a.n; i += blockDim.x) {
            const double2 c = cmul_conj(d[i], a.twist[i]);
            const uint64_t r0 = (uint64_t)t * a.N + i;
            a.W[r0 * a.d2 + k] = (int32_t)rint(c.x * f);
            a.W[(r0 + a.n) * a.d2 + k] = (int32_t)rint(c.y * f);
        }
        __syncthreads();
    }
}

// Rotated query masks: column j = e rho + r holds the mask of eye e shifted by s = r - (rho-1)/2
// columns of the 16 x 200 x 4 layout: bit (row, col, b) = mask bit (row, (col + s) mod 200, b).
__global__ void k_rotate_masks(const uint8_t *qm, uint32_t n_cols, uint32_t rho, uint8_t *out) {
    const uint32_t tb = 1600;
    const uint64_t total = (uint64_t)n_cols * tb;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t j = (uint32_t)(x / tb), byte = (uint32_t)(x % tb);
        const uint32_t e = j / rho, r = j % rho;
        const int s = (int)r - (int)(rho - 1) / 2;
        uint32_t v = 0;
        for (uint32_t bb = 0; bb < 8; ++bb) {
            const uint32_t bit = byte * 8 + bb;
            const uint32_t row = bit / 800, rem = bit % 800, col = rem / 4, pl = rem % 4;
            const uint32_t sc = (uint32_t)(((int)col + s + 200) % 200);
            v |= (uint32_t)tbit(qm + (uint64_t)e * tb, (uint64_t)row * 800 + sc * 4 + pl) << bb;
        }
        out[x] = (uint8_t)v;
    }
}

// Mask overlaps den[j][i] = ||m_j AND m_i||_1: a block takes 8 columns (their rotated masks in
// shared memory) against 256 templates, one per thread.
__global__ void __launch_bounds__(256) k_mask_den(const uint64_t *rq, const uint64_t *dm, uint32_t n_cols,
                                                  uint64_t n_tpl, int32_t *den) {
    __shared__ uint64_t sq[8][200];
    const uint32_t j0 = blockIdx.y * 8;
    for (uint32_t x = threadIdx.x; x < 8 * 200; x += blockDim.x) {
        const uint32_t jj = x / 200, w = x % 200;
        sq[jj][w] = (j0 + jj < n_cols) ? rq[(uint64_t)(j0 + jj) * 200 + w] : 0;
    }
    __syncthreads();
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tpl) return;
    int acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const uint64_t *m = dm + i * 200;
    for (uint32_t w = 0; w < 200; ++w) {
        const uint64_t v = m[w];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) acc[jj] += __popcll(v & sq[jj][w]);
    }
    for (int jj = 0; jj < 8; ++jj)
        if (j0 + jj < n_cols) den[(uint64_t)(j0 + jj) * n_tpl + i] = acc[jj];
}

struct MuArgs {
    const int32_t *den;             // [n_cols][n_tpl]
    uint64_t n_tpl;
    uint32_t n_cols, N, n, logn, n_blocks, Lq;
    double scale;                   // 2^log2_scale_mu
    const double2 *twist, *tw;
    const int32_t *pos;
    uint64_t q[2];
    uint64_t *mu;                   // [Lq][n_cols][n_blocks][N] residues
};

// mu = round(2^s Ecd(1 / den)) per (column, block), reduced modulo each limb of Q.
__global__ void __launch_bounds__(512) k_mu_encode(MuArgs a) {
    extern __shared__ double2 sm[];
    double2 *d = sm, *tw = sm + a.n;
    for (uint32_t k = threadIdx.x; k < a.n / 2; k += blockDim.x) tw[k] = a.tw[k];
    __syncthreads();
    const uint64_t total = (uint64_t)a.n_cols * a.n_blocks;
    const uint64_t per_limb = total * a.N;
    for (uint64_t x = blockIdx.x; x < total; x += gridDim.x) {
        const uint32_t j = (uint32_t)(x / a.n_blocks), t = (uint32_t)(x % a.n_blocks);
        for (uint32_t i = threadIdx.x; i < a.n; i += blockDim.x) {
            const uint64_t tpl = (uint64_t)t * a.n + i;
            double v = 0.0;
            if (tpl < a.n_tpl) {
                const int dd = a.den[(uint64_t)j * a.n_tpl + tpl];
                if (dd > 0) v = 1.0 / (double)dd;
            }
            d[brev((uint32_t)a.pos[i], a.logn)] = make_double2(v, 0.0);
        }
        __syncthreads();
        fft_dit(d, tw, a.n, a.logn, true);
        const double f = a.scale / (double)a.n;
        for (uint32_t i = threadIdx.x; i < a.n; i += blockDim.x) {
            const double2 c = cmul_conj(d[i], a.twist[i]);
            const int64_t v[2] = {(int64_t)rint(c.x * f), (int64_t)rint(c.y * f)};
            for (int h = 0; h < 2; ++h)
                for (uint32_t l = 0; l < a.Lq; ++l) {
                    const uint64_t q = a.q[l];
                    const uint64_t m = (uint64_t)(v[h] < 0 ? -v[h] : v[h]) % q;
                    a.mu[l * per_limb + x * a.N + i + h * a.n] = (v[h] < 0 && m) ? q - m : m;
                }
        }
        __syncthreads();
    }
}

struct NttTab {
    const uint64_t *tab;            // [Lq][4][N]
    uint64_t q[2], ninv[2], ninvs[2], rhi[2], rlo[2];
};

// Forward NTT of polynomials: poly p of limb l reads src + l src_ls + p src_ps and writes
// dst + l dst_ls + p dst_ps (N words each).
struct FwdArgs {
    NttTab T;
    uint32_t N, Lq, per_limb;
    const uint64_t *src; uint64_t src_ls, src_ps;
    uint64_t *dst; uint64_t dst_ls, dst_ps;
};
__global__ void __launch_bounds__(1024) k_ntt_fwd(FwdArgs a) {
    extern __shared__ uint64_t su[];
    const uint64_t total = (uint64_t)a.Lq * a.per_limb;
    for (uint64_t x = blockIdx.x; x < total; x += gridDim.x) {
        const uint32_t l = (uint32_t)(x / a.per_limb);
        const uint64_t p = x % a.per_limb;
        const uint64_t *s = a.src + l * a.src_ls + p * a.src_ps;
        for (uint32_t i = threadIdx.x; i < a.N; i += blockDim.x) su[i] = s[i];
        __syncthreads();
        const uint64_t *tb = a.T.tab + (uint64_t)l * 4 * a.N;
        ntt_fwd(su, a.N, tb, tb + a.N, a.T.q[l]);
        uint64_t *dd = a.dst + l * a.dst_ls + p * a.dst_ps;
        for (uint32_t i = threadIdx.x; i < a.N; i += blockDim.x) dd[i] = su[i];
        __syncthreads();
    }
}

// Output (limb l, column j, block t, part h): part 0 = a_j mu_{j,t}, part 1 = b_{j,t} mu_{j,t};
// a_ntt holds NTT(a_j), mu_ntt NTT(mu_{j,t}); b rows are read from the rescaled scores.
struct MulArgs {
    NttTab T;
    uint32_t N, Lq, n_cols, n_blocks;
    uint64_t M;                     // rows of the scores
    const uint64_t *scores;         // [Lq][n_cols][M]
    const uint64_t *a_ntt;          // [Lq][n_cols][N]
    const uint64_t *mu_ntt;         // [Lq][n_cols][n_blocks][N]
    uint64_t *out;                  // [Lq][n_cols][n_blocks][2][N]
};
__global__ void __launch_bounds__(1024) k_ntt_mul_inv(MulArgs a) {
    extern __shared__ uint64_t su[];
    const uint64_t per_limb = (uint64_t)a.n_cols * a.n_blocks * 2;
    const uint64_t total = (uint64_t)a.Lq * per_limb;
    for (uint64_t x = blockIdx.x; x < total; x += gridDim.x) {
        const uint32_t l = (uint32_t)(x / per_limb);
        const uint64_t r = x % per_limb;
        const uint32_t h = (uint32_t)(r & 1);
        const uint64_t jt = r >> 1;                                   // j n_blocks + t
        const uint32_t j = (uint32_t)(jt / a.n_blocks), t = (uint32_t)(jt % a.n_blocks);
        const uint64_t q = a.T.q[l];
        const uint64_t *tb = a.T.tab + (uint64_t)l * 4 * a.N;
        if (h == 0) {
            const uint64_t *s = a.a_ntt + ((uint64_t)l * a.n_cols + j) * a.N;
            for (uint32_t i = threadIdx.x; i < a.N; i += blockDim.x) su[i] = s[i];
            __syncthreads();
        } else {
            const uint64_t *s = a.scores + ((uint64_t)l * a.n_cols + j) * a.M + a.N + (uint64_t)t * a.N;
            for (uint32_t i = threadIdx.x; i < a.N; i += blockDim.x) su[i] = s[i];
            __syncthreads();
            ntt_fwd(su, a.N, tb, tb + a.N, q);
        }
        const uint64_t *m = a.mu_ntt + (((uint64_t)l * a.n_cols + j) * a.n_blocks + t) * a.N;
        for (uint32_t i = threadIdx.x; i < a.N; i += blockDim.x)
            su[i] = mulmod_r128(su[i], m[i], q, a.T.rhi[l], a.T.rlo[l]);
        __syncthreads();
        ntt_inv(su, a.N, tb + 2 * a.N, tb + 3 * a.N, q, a.T.ninv[l], a.T.ninvs[l]);
        uint64_t *o = a.out + ((((uint64_t)l * a.n_cols + j) * a.n_blocks + t) * 2 + h) * a.N;
        for (uint32_t i = threadIdx.x; i < a.N; i += blockDim.x) o[i] = su[i];
        __syncthreads();
    }
}

// Decryption of every normalised block for checking: dec = a' s_{db,t} + b' per limb of Q.
struct DecArgs2 {
    uint32_t N, Lq, n_cols, n_blocks, h;
    uint64_t q[2];
    const int32_t *spos; const int8_t *ssgn;     // [blocks][h]
    const uint64_t *norm;                        // [Lq][n_cols][n_blocks][2][N]
    uint64_t *dec;                               // [Lq][n_cols][n_blocks][N]
};
__global__ void __launch_bounds__(512) k_slot_dec_limbs(DecArgs2 a) {
    extern __shared__ uint64_t su[];
    const uint64_t per_limb = (uint64_t)a.n_cols * a.n_blocks;
    const uint64_t total = (uint64_t)a.Lq * per_limb;
    for (uint64_t x = blockIdx.x; x < total; x += gridDim.x) {
        const uint32_t l = (uint32_t)(x / per_limb);
        const uint64_t jt = x % per_limb;
        const uint32_t t = (uint32_t)(jt % a.n_blocks);
        const uint64_t q = a.q[l];
        const uint64_t *ap = a.norm + (((uint64_t)l * per_limb + jt) * 2) * a.N, *bp = ap + a.N;
        for (uint32_t i = threadIdx.x; i < a.N; i += blockDim.x) su[i] = ap[i];
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < a.N; i += blockDim.x) {
            uint64_t acc = bp[i];
            for (uint32_t c = 0; c < a.h; ++c) {
                const uint32_t p = (uint32_t)a.spos[(uint64_t)t * a.h + c];
                const int s = a.ssgn[(uint64_t)t * a.h + c];
                // X^p * a: coefficient i takes a[i - p], negated when it wraps
                const bool wrap = i < p;
                const uint64_t term = wrap ? su[i + a.N - p] : su[i - p];
                const bool neg = wrap ? (s > 0) : (s < 0);
                acc = neg ? sub_mod(acc, term, q) : add_mod(acc, term, q);
            }
            a.dec[((uint64_t)l * per_limb + jt) * a.N + i] = acc;
        }
        __syncthreads();
    }
}

// Decoding of the decrypted blocks: CRT over the limbs of Q to the centred integer, division by
// the three scales, Dcd, and the distance (1 - s) / 2 of every slot holding a template.
struct DecodeArgs {
    uint32_t N, n, logn, Lq, n_cols, n_blocks;
    uint64_t n_tpl;
    uint64_t q[2], rhi1, rlo1, q0inv;            // CRT constants (q0inv = q_0^-1 mod q_1)
    double inv_scale;                            // 2^-(log2 Delta + s_db + s_mu)
    const double2 *twist, *tw;
    const int32_t *pos;
    const uint64_t *dec;                         // [Lq][n_cols][n_blocks][N]
    double *hd;                                  // [n_cols][n_tpl]
};
__device__ __forceinline__ double centred_value(const DecodeArgs &a, uint64_t r0, uint64_t r1) {
    if (a.Lq == 1) {
        const bool neg = r0 > a.q[0] / 2;
        return neg ? -(double)(a.q[0] - r0) : (double)r0;
    }
    // x = r0 + q0 ((r1 - r0) q0^-1 mod q1) in [0, q0 q1)
    const uint64_t q0 = a.q[0], q1 = a.q[1];
    const uint64_t r0m = r0 >= q1 ? r0 - q1 * (r0 / q1) : r0;
    const uint64_t dlt = r1 >= r0m ? r1 - r0m : r1 + q1 - r0m;
    const uint64_t k = mulmod_r128(dlt, a.q0inv, q1, a.rhi1, a.rlo1);
    const unsigned __int128 Q = (unsigned __int128)q0 * q1;
    unsigned __int128 x = (unsigned __int128)q0 * k + r0;
    const bool neg = x > Q / 2;
    if (neg) x = Q - x;
    const double v = (double)(uint64_t)(x >> 64) * 18446744073709551616.0 + (double)(uint64_t)x;
    return neg ? -v : v;
}
__global__ void __launch_bounds__(512) k_slot_decode(DecodeArgs a) {
    extern __shared__ double2 sm[];
    double2 *d = sm, *tw = sm + a.n;
    for (uint32_t k = threadIdx.x; k < a.n / 2; k += blockDim.x) tw[k] = a.tw[k];
    __syncthreads();
    const uint64_t per_limb = (uint64_t)a.n_cols * a.n_blocks;
    for (uint64_t x = blockIdx.x; x < per_limb; x += gridDim.x) {
        const uint32_t j = (uint32_t)(x / a.n_blocks), t = (uint32_t)(x % a.n_blocks);
        const uint64_t *d0 = a.dec + x * a.N, *d1 = a.dec + (per_limb + x) * a.N;
        for (uint32_t i = threadIdx.x; i < a.n; i += blockDim.x) {
            const double lo = centred_value(a, d0[i], a.Lq > 1 ? d1[i] : 0) * a.inv_scale;
            const double hi = centred_value(a, d0[i + a.n], a.Lq > 1 ? d1[i + a.n] : 0) * a.inv_scale;
            d[brev(i, a.logn)] = cmul(make_double2(lo, hi), a.twist[i]);
        }
        __syncthreads();
        fft_dit(d, tw, a.n, a.logn, false);
        for (uint32_t i = threadIdx.x; i < a.n; i += blockDim.x) {
            const uint64_t tpl = (uint64_t)t * a.n + i;
            if (tpl < a.n_tpl) a.hd[(uint64_t)j * a.n_tpl + tpl] = (1.0 - d[a.pos[i]].x) * 0.5;
        }
        __syncthreads();
    }
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

NttTab ntt_tab(const SlotTables *T) {
    NttTab t{};
    t.tab = T->ntt;
    for (uint32_t l = 0; l < T->Lq; ++l) {
        t.q[l] = T->q[l]; t.ninv[l] = T->ninv[l]; t.ninvs[l] = T->ninvs[l];
        t.rhi[l] = T->rhi[l]; t.rlo[l] = T->rlo[l];
    }
    return t;
}

template <typename K>
cudaError_t set_smem(K kern, size_t bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

// Workspace layout of icm_normalize (offsets 256-byte aligned): rotated query masks [n_cols][1600],
// mask overlaps [n_cols][n_tpl] int32, mu residues [Lq][n_cols][n_blocks][N], NTT(a) [Lq][n_cols][N].
struct NormWs {
    size_t rq, den, mu, antt, total;
};
static size_t a256(size_t x) { return (x + 255) / 256 * 256; }
static NormWs norm_ws(uint32_t Lq, uint32_t n_cols, uint64_t n_tpl, uint32_t n_blocks, uint32_t N) {
    NormWs w{};
    w.rq = 0;
    w.den = w.rq + a256((size_t)n_cols * 1600);
    w.mu = w.den + a256((size_t)n_cols * n_tpl * 4);
    w.antt = w.mu + a256((size_t)Lq * n_cols * n_blocks * N * 8);
    w.total = w.antt + a256((size_t)Lq * n_cols * N * 8);
    return w;
}

}  // namespace icm

namespace icm {
icm_status api_fail(icm_status s, const char *msg);
}
using namespace icm;

namespace {
icm_status sfail(icm_status s, const std::string &m) { return api_fail(s, m.c_str()); }
#define SL_TRY(expr)                                                                    \
    do {                                                                                \
        cudaError_t _e = (expr);                                                        \
        if (_e != cudaSuccess) return sfail(ICM_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

// Bounds of the slot encoding (worst case): message entries |W| <= 2^s + 1 and their products
// with the query secret, sum of h (d2 / N_q) of them, must fit int32; the CCMM must not wrap
// modulo Q_db (Q' Delta 2^s d2 below Q_db / 2 with room for the noise terms the context already
// bounds), i.e. Delta 2^s d2 < Q / 4.
icm_status slot_db_bounds(const icm_ctx *c, uint32_t s) {
    if (s == 0 || s > 24) return sfail(ICM_EINVAL, "log2 slot scale of the database must be 1..24");
    const long double terms = (long double)c->p.hamming_weight * c->n_qblk;
    if (terms * (exp2l((long double)s) + 1) >= 2147483647.0L)
        return sfail(ICM_EBOUND, "slot scale too large for int32 messages (h d2 / N_q (2^s + 1) >= 2^31)");
    long double lQ = 0;
    for (uint32_t l = 0; l < c->p.n_limbs_q; ++l) lQ += log2l((long double)c->q[l]);
    if (c->p.log2_delta + s + log2l((long double)c->p.d2) >= lQ - 2)
        return sfail(ICM_EBOUND, "Delta 2^s d2 must stay below Q / 4");
    return ICM_OK;
}
}  // namespace

extern "C" {

icm_status icm_db_bytes_slots(const icm_ctx *c, size_t n_db, size_t *bytes, size_t *m_rows) {
    if (!c || !bytes || !m_rows) return sfail(ICM_EINVAL, "null argument");
    const uint64_t nb = (n_db + c->N_db / 2 - 1) / (c->N_db / 2);
    const DbLayout L = make_layout(nb * c->N_db, c->N_db, c->p.rho);
    *m_rows = L.M;
    *bytes = (size_t)c->p.n_limbs * L.M * c->K * 8;
    return ICM_OK;
}

icm_status icm_db_encrypt_slots(icm_ctx *c, const uint8_t *codes, const uint8_t *masks, size_t n_db,
                                uint32_t log2_scale, uint64_t chunk_id, void *dev_buf, size_t bytes, void *stream,
                                icm_db **out) {
    if (!c || !out || !dev_buf || !n_db || !codes || !masks) return sfail(ICM_EINVAL, "null argument or no templates");
    if (!c->have_keys) return sfail(ICM_EINVAL, "icm_keygen has not run");
    icm_status s = slot_db_bounds(c, log2_scale);
    if (s != ICM_OK) return s;
    const uint32_t N = c->N_db, n = N / 2;
    const uint64_t nb = (n_db + n - 1) / n;
    DbLayout L = make_layout(nb * N, N, c->p.rho);
    if (L.n_blocks() > c->max_db_blocks) return sfail(ICM_EUNSUPPORTED, "chunk larger than the keyed blocks");
    size_t need, m;
    icm_db_bytes_slots(c, n_db, &need, &m);
    if (bytes < need) return sfail(ICM_ENOMEM, "database buffer too small");
    if ((uintptr_t)dev_buf % 16) return sfail(ICM_EINVAL, "database buffer must be 16-byte aligned");
    if (L.M > 0xFFFFFFFFull) return sfail(ICM_EUNSUPPORTED, "chunk too large");
    std::string why;
    const SlotTables *T = slot_tables(c, why);
    if (!T) return sfail(ICM_ECUDA, "slot tables: " + why);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t tb = c->p.code_bits / 8;
    const size_t wbytes = (size_t)nb * N * c->p.d2 * 4;
    uint8_t *d_t = nullptr;
    int32_t *d_w = nullptr;
    SL_TRY(cudaMallocAsync((void **)&d_t, 2 * n_db * tb, st));
    cudaError_t e = cudaMallocAsync((void **)&d_w, wbytes, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_t, codes, n_db * tb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_t + n_db * tb, masks, n_db * tb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_w, 0, wbytes, st);
    if (e == cudaSuccess) {
        EncDbArgs a{};
        a.codes = d_t; a.masks = d_t + n_db * tb; a.n_tpl = n_db;
        a.code_bits = c->p.code_bits; a.d2 = c->p.d2; a.N = N; a.n = n; a.logn = T->logn; a.n_blocks = (uint32_t)nb;
        a.scale = ldexp(1.0, (int)log2_scale);
        a.twist = T->twist; a.tw = T->tw; a.pos = T->pos; a.W = d_w;
        const size_t smem = (size_t)n * 16 + (size_t)(n / 2) * 16;
        e = set_smem(k_slot_db_encode, smem);
        if (e == cudaSuccess) {
            const uint64_t total = nb * c->p.code_bits;
            const unsigned grid = (unsigned)std::min<uint64_t>(total, (uint64_t)sm_count() * (smem > 110000 ? 1 : 2));
            k_slot_db_encode<<<grid, 512, smem, st>>>(a);
            e = cudaGetLastError();
        }
    }
    icm_db *db = nullptr;
    if (e == cudaSuccess) {
        db = new (std::nothrow) icm_db();
        if (!db) e = cudaErrorMemoryAllocation;
    }
    uint64_t *d = (uint64_t *)dev_buf;
    if (e == cudaSuccess) e = launch_db_messages(c, to_dev(L), nullptr, nullptr, d, st, d_w);
    if (e == cudaSuccess) e = launch_db_apart_and_b(c, to_dev(L), chunk_id, d, st);
    if (d_w) cudaFreeAsync(d_w, st);
    if (d_t) cudaFreeAsync(d_t, st);
    if (e != cudaSuccess) { delete db; return sfail(ICM_ECUDA, std::string("slot db encrypt: ") + cudaGetErrorString(e)); }
    L.n_tpl = n_db;
    L.slot_log2 = log2_scale;
    db->ctx = c; db->lay = L; db->chunk_id = chunk_id; db->dev = d; db->bytes = bytes;
    *out = db;
    return ICM_OK;
}

icm_status icm_normalize_bytes(const icm_scores *in, size_t *out_bytes, size_t *ws_bytes) {
    if (!in || !out_bytes || !ws_bytes) return sfail(ICM_EINVAL, "null argument");
    const icm_ctx *c = in->ctx;
    if (!in->lay.slot_log2 || !in->rescaled || in->folded)
        return sfail(ICM_EINVAL, "normalisation takes unfolded scores of a slot-encoded database after the rescaling");
    const uint32_t N = in->lay.N, nb = in->lay.n_blocks();
    *out_bytes = (size_t)c->p.n_limbs_q * in->n_cols * nb * 2 * N * 8;
    *ws_bytes = norm_ws(c->p.n_limbs_q, in->n_cols, in->lay.n_tpl, nb, N).total;
    return ICM_OK;
}

icm_status icm_normalize(icm_ctx *c, const icm_scores *in, const uint8_t *dev_q_masks, const uint8_t *dev_db_masks,
                         uint32_t log2_scale_mu, void *dev_out, size_t bytes, void *dev_ws, size_t ws_bytes,
                         void *stream) {
    if (!c || !in || !dev_q_masks || !dev_db_masks || !dev_out || !dev_ws) return sfail(ICM_EINVAL, "null argument");
    if (in->ctx != c) return sfail(ICM_EINVAL, "scores of another context");
    size_t ob, wb;
    icm_status s = icm_normalize_bytes(in, &ob, &wb);
    if (s != ICM_OK) return s;
    if (bytes < ob || ws_bytes < wb) return sfail(ICM_ENOMEM, "output or workspace too small");
    if ((uintptr_t)dev_ws % 16 || (uintptr_t)dev_out % 16 || (uintptr_t)dev_db_masks % 8)
        return sfail(ICM_EINVAL, "output and workspace must be 16-byte aligned, database masks 8-byte aligned");
    long double lQ = 0;
    for (uint32_t l = 0; l < c->p.n_limbs_q; ++l) lQ += log2l((long double)c->q[l]);
    if (log2_scale_mu == 0 || log2_scale_mu > 62 ||
        (long double)c->p.log2_delta + in->lay.slot_log2 + log2_scale_mu + 1 >= lQ - 1)
        return sfail(ICM_EBOUND, "Delta 2^s_db 2^s_mu must stay below Q / 4 (normalised scores are at most 1)");
    std::string why;
    const SlotTables *T = slot_tables(c, why);
    if (!T) return sfail(ICM_ECUDA, "slot tables: " + why);
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t N = in->lay.N, n = N / 2, nb = in->lay.n_blocks(), Lq = c->p.n_limbs_q, d3 = in->n_cols;
    const uint64_t n_tpl = in->lay.n_tpl;
    const NormWs W = norm_ws(Lq, d3, n_tpl, nb, N);
    char *ws = (char *)dev_ws;
    uint8_t *rq = (uint8_t *)(ws + W.rq);
    int32_t *den = (int32_t *)(ws + W.den);
    uint64_t *mu = (uint64_t *)(ws + W.mu), *antt = (uint64_t *)(ws + W.antt);
    const int sms = sm_count();
    // 1. rotated query masks and mask overlaps
    k_rotate_masks<<<(unsigned)std::min<uint64_t>(((uint64_t)d3 * 1600 + 255) / 256, (uint64_t)sms * 16), 256, 0, st>>>(
        dev_q_masks, d3, c->p.rho, rq);
    SL_TRY(cudaGetLastError());
    k_mask_den<<<dim3((unsigned)((n_tpl + 255) / 256), (d3 + 7) / 8), 256, 0, st>>>(
        reinterpret_cast<const uint64_t *>(rq), reinterpret_cast<const uint64_t *>(dev_db_masks), d3, n_tpl, den);
    SL_TRY(cudaGetLastError());
    // 2. mu per (column, block), residues modulo each limb of Q
    {
        MuArgs a{};
        a.den = den; a.n_tpl = n_tpl; a.n_cols = d3; a.N = N; a.n = n; a.logn = T->logn; a.n_blocks = nb; a.Lq = Lq;
        a.scale = ldexp(1.0, (int)log2_scale_mu);
        a.twist = T->twist; a.tw = T->tw; a.pos = T->pos;
        for (uint32_t l = 0; l < Lq; ++l) a.q[l] = c->q[l];
        a.mu = mu;
        const size_t smem = (size_t)n * 16 + (size_t)(n / 2) * 16;
        SL_TRY(set_smem(k_mu_encode, smem));
        const unsigned grid = (unsigned)std::min<uint64_t>((uint64_t)d3 * nb, (uint64_t)sms * (smem > 110000 ? 1 : 2));
        k_mu_encode<<<grid, 512, smem, st>>>(a);
        SL_TRY(cudaGetLastError());
    }
    // 3. NTT of every mu (in place) and of every a-part
    const NttTab NT = ntt_tab(T);
    const size_t psm = (size_t)N * 8;
    SL_TRY(set_smem(k_ntt_fwd, psm));
    SL_TRY(set_smem(k_ntt_mul_inv, psm));
    const unsigned per_sm = psm > 110000 ? 1 : (psm > 70000 ? 2 : 4);
    // one polynomial per block in shared memory: the largest rings fit one block per SM, which
    // then takes 1,024 threads to hide the latency of the butterflies' 64-bit products
    const unsigned ntt_threads = psm > 70000 ? 1024 : 512;
    {
        FwdArgs a{};
        a.T = NT; a.N = N; a.Lq = Lq; a.per_limb = d3 * nb;
        a.src = mu; a.src_ls = (uint64_t)d3 * nb * N; a.src_ps = N;
        a.dst = mu; a.dst_ls = a.src_ls; a.dst_ps = N;
        k_ntt_fwd<<<(unsigned)std::min<uint64_t>((uint64_t)Lq * d3 * nb, (uint64_t)sms * per_sm), ntt_threads, psm, st>>>(a);
        SL_TRY(cudaGetLastError());
        FwdArgs b{};
        b.T = NT; b.N = N; b.Lq = Lq; b.per_limb = d3;
        b.src = in->dev; b.src_ls = (uint64_t)d3 * in->lay.M; b.src_ps = in->lay.M;
        b.dst = antt; b.dst_ls = (uint64_t)d3 * N; b.dst_ps = N;
        k_ntt_fwd<<<(unsigned)std::min<uint64_t>((uint64_t)Lq * d3, (uint64_t)sms * per_sm), ntt_threads, psm, st>>>(b);
        SL_TRY(cudaGetLastError());
    }
    // 4. products and inverse NTTs
    {
        MulArgs a{};
        a.T = NT; a.N = N; a.Lq = Lq; a.n_cols = d3; a.n_blocks = nb; a.M = in->lay.M;
        a.scores = in->dev; a.a_ntt = antt; a.mu_ntt = mu; a.out = (uint64_t *)dev_out;
        k_ntt_mul_inv<<<(unsigned)std::min<uint64_t>((uint64_t)Lq * d3 * nb * 2, (uint64_t)sms * per_sm), ntt_threads, psm, st>>>(a);
        SL_TRY(cudaGetLastError());
    }
    return ICM_OK;
}

icm_status icm_decrypt_slots(icm_ctx *c, const icm_scores *in, const void *dev_norm, size_t norm_bytes,
                             uint32_t log2_scale_mu, double *dev_hd, size_t n, void *stream) {
    if (!c || !in || !dev_norm || !dev_hd) return sfail(ICM_EINVAL, "null argument");
    if (in->ctx != c) return sfail(ICM_EINVAL, "scores of another context");
    size_t ob, wb;
    icm_status s = icm_normalize_bytes(in, &ob, &wb);
    if (s != ICM_OK) return s;
    if (norm_bytes < ob) return sfail(ICM_EINVAL, "normalised buffer too small");
    if (n < (size_t)in->n_cols * in->lay.n_tpl) return sfail(ICM_ENOMEM, "output too small: n_cols x n_db distances");
    std::string why;
    const SlotTables *T = slot_tables(c, why);
    if (!T) return sfail(ICM_ECUDA, "slot tables: " + why);
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t N = in->lay.N, n2 = N / 2, nb = in->lay.n_blocks(), Lq = c->p.n_limbs_q, d3 = in->n_cols;
    uint64_t *dec = nullptr;
    SL_TRY(cudaMallocAsync((void **)&dec, (size_t)Lq * d3 * nb * N * 8, st));
    const int sms = sm_count();
    cudaError_t e;
    {
        DecArgs2 a{};
        a.N = N; a.Lq = Lq; a.n_cols = d3; a.n_blocks = nb; a.h = c->p.hamming_weight;
        for (uint32_t l = 0; l < Lq; ++l) a.q[l] = c->q[l];
        a.spos = c->d_sdb_pos; a.ssgn = c->d_sdb_sgn;
        a.norm = (const uint64_t *)dev_norm; a.dec = dec;
        const size_t psm = (size_t)N * 8;
        e = set_smem(k_slot_dec_limbs, psm);
        if (e == cudaSuccess) {
            k_slot_dec_limbs<<<(unsigned)std::min<uint64_t>((uint64_t)Lq * d3 * nb, (uint64_t)sms * 2), 512, psm, st>>>(a);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        DecodeArgs a{};
        a.N = N; a.n = n2; a.logn = T->logn; a.Lq = Lq; a.n_cols = d3; a.n_blocks = nb; a.n_tpl = in->lay.n_tpl;
        a.q[0] = c->q[0]; a.q[1] = Lq > 1 ? c->q[1] : 0;
        a.rhi1 = Lq > 1 ? T->rhi[1] : 0; a.rlo1 = Lq > 1 ? T->rlo[1] : 0; a.q0inv = T->q0inv_mod_q1;
        a.inv_scale = ldexp(1.0, -(int)(c->p.log2_delta + in->lay.slot_log2 + log2_scale_mu));
        a.twist = T->twist; a.tw = T->tw; a.pos = T->pos; a.dec = dec; a.hd = dev_hd;
        const size_t smem = (size_t)n2 * 16 + (size_t)(n2 / 2) * 16;
        e = set_smem(k_slot_decode, smem);
        if (e == cudaSuccess) {
            k_slot_decode<<<(unsigned)std::min<uint64_t>((uint64_t)d3 * nb, (uint64_t)sms * (smem > 110000 ? 1 : 2)),
                            512, smem, st>>>(a);
            e = cudaGetLastError();
        }
    }
    cudaFreeAsync(dec, st);
    if (e != cudaSuccess) return sfail(ICM_ECUDA, std::string("slot decrypt: ") + cudaGetErrorString(e));
    return ICM_OK;
}

}  // extern "C"
