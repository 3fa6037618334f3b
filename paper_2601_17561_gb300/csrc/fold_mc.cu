// Cleartext check of a folding polynomial: the Monte Carlo experiments of Appendix C.2 for the
// (k, N_f, P_f)-folding-polynomial definition of Section 4.1.2, one trial per thread.
//
// Trial t draws 2k - 1 negative scores from D = N(mu, sigma^2): x_0..x_{k-1} and y_0..y_{k-2}
// (Appendix C.2 draws the two sets independently), then forms S_k = sum f(x_i) and
// S_{k-1} = sum f(y_i) and counts S_k outside N_f and min/max of f over P plus S_{k-1} outside P_f.
// Random numbers: Philox4x64-10 (Salmon et al., SC 2011) at counters (t, j, 0, 0) with key
// (seed, 0); normal n of a trial comes from the Box-Muller transform (Box and Muller, 1958) of
// words (2p, 2p+1), p = n / 2.  The scores, f and the sums are computed in fp32 (the log of the
// Box-Muller radius from a 64-bit uniform, so the deviates reach 9.4 sigma).
#include <algorithm>
#include <cmath>

#include "icm_internal.h"

namespace {

constexpr int FMC_THREADS = 256;
constexpr uint32_t FMC_MAX_BINS = 8192;
constexpr uint64_t FMC_TRIALS_PER_LAUNCH = 1ull << 32;   // keeps every block's u32 counters exact

struct FmcArgs {
    float c[16];                      // f(x) = sum c[i] x^i, zero above the degree
    uint64_t rk0[10], rk1[10];        // Philox round keys (seed + r W0, 0 + r W1)
    uint32_t k, n_bins;
    float mu, sigma;
    float nf_lo, nf_hi, pf_lo, pf_hi, fmin, fmax;
    float h_lo, h_scale;              // bin of s: floor((s - h_lo) h_scale), clamped to [-1, n_bins]
    uint64_t t0, n;
    unsigned long long *counts;       // [6]
    unsigned long long *hist;         // [2][n_bins + 2] or null
    float2 *sums;                     // [n] or null
};

// Philox4x64-10 block at counter (t, j, 0, 0).
__device__ __forceinline__ void philox_block(const FmcArgs &a, uint64_t t, uint64_t j, uint64_t w[4]) {
    constexpr uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    uint64_t c0 = t, c1 = j, c2 = 0, c3 = 0;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t h0 = __umul64hi(M0, c0), l0 = M0 * c0;
        const uint64_t h1 = __umul64hi(M1, c2), l1 = M1 * c2;
        c0 = h1 ^ c1 ^ a.rk0[r];
        c1 = l1;
        c2 = h0 ^ c3 ^ a.rk1[r];
        c3 = l0;
    }
    w[0] = c0; w[1] = c1; w[2] = c2; w[3] = c3;
}

// Box-Muller on u1 = (a + 1/2) 2^-64 and u2 = b 2^-64, with the fp32 operands built from the
// words' bits (64-bit integer to float conversions would run on the slow fp64 pipe).  u1 < 1/2:
// u1 = v 2^-65 with v = 2a + 1, normalised as y 2^(-1-lz), y in [1/2, 1] rounded to 24 bits, so
// ln u1 = log1p(y - 1) - (1 + lz) ln 2.  u1 >= 1/2: 1 - u1 = v 2^-65 with v = 2(~a) + 1, so
// ln u1 = log1p(-y 2^(-1-lz)) keeps every digit near u1 = 1.  u2 is rounded to a multiple of 2^-23
// (angle error below 4e-7).
__device__ __forceinline__ void box_muller(uint64_t a, uint64_t b, float &z0, float &z1) {
    constexpr float LN2_HI = 0x1.62e430p-1f, LN2_LO = -0x1.05c610p-29f;    // ln 2 = LN2_HI + LN2_LO
    const bool top = (int64_t)a < 0;
    const uint64_t v = 2 * (top ? ~a : a) + 1;                             // odd, below 2^64
    const int lz = __clzll(v);
    const uint32_t mant = (uint32_t)(((v << lz) >> 39) + 1) >> 1;           // 24 bits incl. the leading one
    const float y = __int_as_float(0x3E800000u + mant);                     // (2^23 + frac) 2^-24 in [1/2, 1]
    const float sc = __int_as_float((uint32_t)(126 - lz) << 23);            // 2^(-1-lz)
    const float e = top ? 0.f : 0x1p23f - __int_as_float(0x4B000000 + 1 + lz);   // -(1 + lz), exact
    const float l = fmaf(e, LN2_HI, fmaf(e, LN2_LO, log1pf(top ? -(y * sc) : y - 1.f)));
    const float r = sqrtf(-2.f * l);
    const float u2 = __int_as_float(0x3F800000u + ((uint32_t)((b >> 40) + 1) >> 1)) - 1.f;   // round(u2 2^23) 2^-23
    float s, c;
    sincospif(2.f * u2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

template <int DEG>
__device__ __forceinline__ float horner(const FmcArgs &a, float x) {
    float y = a.c[DEG];
#pragma unroll
    for (int d = DEG - 1; d >= 0; --d) y = fmaf(y, x, a.c[d]);
    return y;
}

template <int DEG>
__global__ void __launch_bounds__(FMC_THREADS, 5) k_fold_mc(const __grid_constant__ FmcArgs a) {
    extern __shared__ uint32_t sh_hist[];                    // [2][n_bins + 2]
    __shared__ unsigned long long sh_cnt[6];
    const uint32_t nh = a.hist ? a.n_bins + 2 : 0;
    for (uint32_t i = threadIdx.x; i < 2 * nh; i += blockDim.x) sh_hist[i] = 0;
    if (threadIdx.x < 6) sh_cnt[threadIdx.x] = 0;
    __syncthreads();

    uint32_t cnt[6] = {0, 0, 0, 0, 0, 0};
    const uint32_t n_norm = 2 * a.k - 1, n_blk = (a.k + 1) / 2;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        const uint64_t t = a.t0 + i;
        float sk = 0.f, sk1 = 0.f;
        for (uint32_t j = 0; j < n_blk; ++j) {
            uint64_t w[4];
            philox_block(a, t, j, w);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t n0 = 4 * j + 2 * h;
                if (n0 >= n_norm) break;
                float z0, z1;
                box_muller(w[2 * h], w[2 * h + 1], z0, z1);
                const float f0 = horner<DEG>(a, fmaf(a.sigma, z0, a.mu));
                if (n0 < a.k) sk += f0; else sk1 += f0;
                if (n0 + 1 < n_norm) {
                    const float f1 = horner<DEG>(a, fmaf(a.sigma, z1, a.mu));
                    if (n0 + 1 < a.k) sk += f1; else sk1 += f1;
                }
            }
        }
        cnt[0] += sk < a.nf_lo;
        cnt[1] += sk > a.nf_hi;
        const float pmin = a.fmin + sk1, pmax = a.fmax + sk1;
        cnt[2] += pmin < a.pf_lo;
        cnt[3] += pmin > a.pf_hi;
        cnt[4] += pmax < a.pf_lo;
        cnt[5] += pmax > a.pf_hi;
        if (nh) {
            const float top = (float)a.n_bins;
            const int b0 = __float2int_rd(fminf(fmaxf((sk - a.h_lo) * a.h_scale, -1.f), top)) + 1;
            const int b1 = __float2int_rd(fminf(fmaxf((sk1 - a.h_lo) * a.h_scale, -1.f), top)) + 1;
            atomicAdd(&sh_hist[b0], 1u);
            atomicAdd(&sh_hist[nh + b1], 1u);
        }
        if (a.sums) a.sums[i] = make_float2(sk, sk1);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const uint32_t v = __reduce_add_sync(0xffffffffu, cnt[c]);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&sh_cnt[c], (unsigned long long)v);
    }
    __syncthreads();
    if (threadIdx.x < 6 && sh_cnt[threadIdx.x]) atomicAdd(&a.counts[threadIdx.x], sh_cnt[threadIdx.x]);
    for (uint32_t i = threadIdx.x; i < 2 * nh; i += blockDim.x)
        if (sh_hist[i]) atomicAdd(&a.hist[i], (unsigned long long)sh_hist[i]);
}

double poly_eval(const double *c, uint32_t deg, double x) {
    double y = c[deg];
    for (int d = (int)deg - 1; d >= 0; --d) y = y * x + c[d];
    return y;
}

// Range of f over [lo, hi]: the ends and every sign change of f' on a grid of 4096 cells,
// refined by bisection (a zero of f' without a sign change is not an extremum).
void poly_range(const double *c, uint32_t deg, double lo, double hi, double *mn, double *mx) {
    double d[16];
    for (uint32_t i = 1; i <= deg; ++i) d[i - 1] = c[i] * i;
    double vmin = std::fmin(poly_eval(c, deg, lo), poly_eval(c, deg, hi));
    double vmax = std::fmax(poly_eval(c, deg, lo), poly_eval(c, deg, hi));
    if (deg >= 2 && hi > lo) {
        const int cells = 4096;
        double xa = lo, da = poly_eval(d, deg - 1, lo);
        for (int i = 1; i <= cells; ++i) {
            const double xb = i == cells ? hi : lo + (hi - lo) * i / cells;
            const double db = poly_eval(d, deg - 1, xb);
            if ((da < 0) != (db < 0) || db == 0) {
                double u = xa, v = xb, du = da;
                for (int it = 0; it < 200 && u < v; ++it) {
                    const double m = 0.5 * (u + v);
                    if (m <= u || m >= v) break;
                    const double dm = poly_eval(d, deg - 1, m);
                    if ((dm < 0) == (du < 0) && dm != 0) { u = m; du = dm; } else v = m;
                }
                for (double x : {u, v}) {
                    const double y = poly_eval(c, deg, x);
                    vmin = std::fmin(vmin, y);
                    vmax = std::fmax(vmax, y);
                }
            }
            xa = xb;
            da = db;
        }
    }
    *mn = vmin;
    *mx = vmax;
}

}  // namespace

extern "C" icm_status icm_fold_poly_range(const double *coef, uint32_t degree, double lo, double hi, double *fmin,
                                          double *fmax) {
    if (!coef || !fmin || !fmax || degree > 15 || !(lo <= hi) || !std::isfinite(lo) || !std::isfinite(hi)) {
        icm::set_error("icm_fold_poly_range: bad arguments");
        return ICM_EINVAL;
    }
    for (uint32_t i = 0; i <= degree; ++i)
        if (!std::isfinite(coef[i])) { icm::set_error("icm_fold_poly_range: non-finite coefficient"); return ICM_EINVAL; }
    poly_range(coef, degree, lo, hi, fmin, fmax);
    return ICM_OK;
}

extern "C" icm_status icm_fold_mc(const icm_fold_mc_args *p, uint64_t *dev_counts, uint64_t *dev_hist,
                                  float *dev_sums, void *stream) {
    auto bad = [](const char *why) { icm::set_error(std::string("icm_fold_mc: ") + why); return ICM_EINVAL; };
    if (!p || !p->coef || !dev_counts) return bad("null argument");
    if (p->degree > 15) return bad("degree above 15");
    if (p->k < 1 || p->k > 32) return bad("k outside 1..32");
    if (!(p->sigma > 0) || !std::isfinite(p->sigma) || !std::isfinite(p->mu)) return bad("bad normal law");
    if (!(p->nf_lo <= p->nf_hi) || !(p->pf_lo <= p->pf_hi)) return bad("empty interval N_f or P_f");
    if (!(p->pos_lo <= p->pos_hi) || !std::isfinite(p->pos_lo) || !std::isfinite(p->pos_hi))
        return bad("bad positive interval");
    if (p->n_bins > FMC_MAX_BINS) return bad("more than 8192 bins");
    if (p->n_bins && (!dev_hist || !(p->hist_lo < p->hist_hi) || !std::isfinite(p->hist_lo) ||
                      !std::isfinite(p->hist_hi)))
        return bad("bad histogram range or buffer");
    if (p->trial0 + p->n_trials < p->trial0) return bad("trial range wraps around 2^64");
    if (((uintptr_t)dev_counts | (uintptr_t)dev_hist | (uintptr_t)dev_sums) & 7)
        return bad("counts, histogram or sums not 8-byte aligned");

    FmcArgs a{};
    for (uint32_t i = 0; i <= p->degree; ++i) {
        if (!std::isfinite(p->coef[i])) return bad("non-finite coefficient");
        a.c[i] = (float)p->coef[i];
    }
    double fmin = 0, fmax = 0;
    poly_range(p->coef, p->degree, p->pos_lo, p->pos_hi, &fmin, &fmax);
    uint64_t k0 = p->seed, k1 = 0;
    for (int r = 0; r < 10; ++r) {
        a.rk0[r] = k0;
        a.rk1[r] = k1;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
    a.k = p->k;
    a.n_bins = p->n_bins;
    a.mu = (float)p->mu;
    a.sigma = (float)p->sigma;
    a.nf_lo = (float)p->nf_lo; a.nf_hi = (float)p->nf_hi;
    a.pf_lo = (float)p->pf_lo; a.pf_hi = (float)p->pf_hi;
    a.fmin = (float)fmin; a.fmax = (float)fmax;
    a.h_lo = (float)p->hist_lo;
    a.h_scale = p->n_bins ? (float)(p->n_bins / (p->hist_hi - p->hist_lo)) : 0.f;
    a.counts = (unsigned long long *)dev_counts;
    a.hist = p->n_bins ? (unsigned long long *)dev_hist : nullptr;

    cudaStream_t st = (cudaStream_t)stream;
    const size_t shm = a.hist ? 2 * (p->n_bins + 2) * sizeof(uint32_t) : 0;
    const bool low = p->degree <= 7;
    const void *fn = low ? (const void *)k_fold_mc<7> : (const void *)k_fold_mc<15>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, FMC_THREADS, shm);
    if (e == cudaSuccess && !p->accumulate) {
        e = cudaMemsetAsync(dev_counts, 0, 6 * sizeof(uint64_t), st);
        if (e == cudaSuccess && a.hist) e = cudaMemsetAsync(dev_hist, 0, 2 * (p->n_bins + 2) * sizeof(uint64_t), st);
    }
    if (e != cudaSuccess) { icm::set_error(cudaGetErrorString(e)); return ICM_ECUDA; }
    for (uint64_t done = 0; done < p->n_trials; done += a.n) {           // a.n >= 1: no wrap-around
        a.t0 = p->trial0 + done;
        a.n = std::min<uint64_t>(FMC_TRIALS_PER_LAUNCH, p->n_trials - done);
        a.sums = dev_sums ? (float2 *)dev_sums + done : nullptr;
        const uint64_t want = (a.n + FMC_THREADS - 1) / FMC_THREADS;
        const unsigned blocks = (unsigned)std::min<uint64_t>(want, (uint64_t)sms * std::max(per_sm, 1));
        if (low) k_fold_mc<7><<<blocks, FMC_THREADS, shm, st>>>(a);
        else k_fold_mc<15><<<blocks, FMC_THREADS, shm, st>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) { icm::set_error(cudaGetErrorString(e)); return ICM_ECUDA; }
    }
    return ICM_OK;
}
