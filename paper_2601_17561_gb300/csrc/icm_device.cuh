// Device-side helpers of libicm: modular arithmetic on u64 residues (q < 2^60), the
// counter-based generator, and the per-limb constant tables passed to kernels by value.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define ICM_MAX_LIMBS 8

// Random-stream kinds.  Keys are key(seed, kind, a, b) = sm(sm(sm(seed, kind), a), b) with
// sm(s, i) = output i of SplitMix64 seeded with s (Steele, Lea & Flood 2014).
enum : uint64_t { ICM_KIND_SK_DB = 1, ICM_KIND_SK_Q = 2, ICM_KIND_A_DB = 3, ICM_KIND_E_DB = 4,
                  ICM_KIND_A_Q = 5, ICM_KIND_E_Q = 6 };

struct LimbTable {
    uint32_t n;                          // number of limbs
    uint64_t q[ICM_MAX_LIMBS];           // primes
    uint64_t r64[ICM_MAX_LIMBS];         // floor(2^64 / q)
    uint64_t pw64[ICM_MAX_LIMBS], pw64s[ICM_MAX_LIMBS];     // 2^64 mod q and Shoup companion
    uint64_t pw128[ICM_MAX_LIMBS], pw128s[ICM_MAX_LIMBS];   // 2^128 mod q and Shoup companion
};

__host__ __device__ __forceinline__ uint64_t sm_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
// Output i (0-based) of SplitMix64 seeded with s.
__host__ __device__ __forceinline__ uint64_t sm64(uint64_t s, uint64_t i) {
    return sm_mix64(s + (i + 1) * 0x9E3779B97F4A7C15ULL);
}
__host__ __device__ __forceinline__ uint64_t stream_key(uint64_t seed, uint64_t kind, uint64_t a, uint64_t b) {
    return sm64(sm64(sm64(seed, kind), a), b);
}

__device__ __forceinline__ uint64_t uniform_mod(uint64_t w, uint64_t q) { return __umul64hi(w, q); }

__device__ __forceinline__ int cbd_sample(uint64_t w, int eta) {
    const uint64_t m = (1ULL << eta) - 1;
    return __popcll(w & m) - __popcll((w >> eta) & m);
}

// ---------------------------------------------------------------- modular arithmetic (q < 2^62)

__device__ __forceinline__ uint64_t add_mod(uint64_t a, uint64_t b, uint64_t q) {
    uint64_t s = a + b;
    return s >= q ? s - q : s;
}
__device__ __forceinline__ uint64_t sub_mod(uint64_t a, uint64_t b, uint64_t q) {
    return a >= b ? a - b : a + q - b;
}
// x mod q for any x < 2^64, with r64 = floor(2^64 / q): the quotient estimate is short by at
// most one, so one conditional subtraction finishes.
__device__ __forceinline__ uint64_t reduce64(uint64_t x, uint64_t q, uint64_t r64) {
    uint64_t t = x - __umul64hi(x, r64) * q;
    return t >= q ? t - q : t;
}
// a * w mod q for a < 2^64 and a constant w < q with ws = floor(w 2^64 / q) (Shoup).
__device__ __forceinline__ uint64_t mulmod_shoup(uint64_t a, uint64_t w, uint64_t ws, uint64_t q) {
    uint64_t t = a * w - __umul64hi(a, ws) * q;
    return t >= q ? t - q : t;
}
// Signed 64-bit value modulo q.
__device__ __forceinline__ uint64_t reduce_s64(int64_t x, uint64_t q, uint64_t r64) {
    if (x >= 0) return reduce64((uint64_t)x, q, r64);
    uint64_t m = reduce64((uint64_t)(-x), q, r64);
    return m ? q - m : 0;
}

// ---------------------------------------------------------------- balanced-digit storage form

// The database stores each residue x in [0, q) as the word z whose bytes are the signed balanced
// base-256 digits d_t in [-128, 127] of its centred lift c (c = x or x - q, |c| < q/2 < 2^59):
// c = sum_t d_t 256^t, and the bytes of c + 0x80..80 are d_t + 128, so z = (c + B) ^ B with
// B = 0x8080808080808080.  Tensor-core forms read the digits directly; the u64 form maps back.
#define ICM_DIGIT_BIAS 0x8080808080808080ull
__host__ __device__ __forceinline__ uint64_t to_digit_form(uint64_t x, uint64_t q) {
    const uint64_t c = (x > (q >> 1)) ? x - q : x;            // two's complement centred lift
    return (c + ICM_DIGIT_BIAS) ^ ICM_DIGIT_BIAS;
}
__host__ __device__ __forceinline__ uint64_t from_digit_form(uint64_t z, uint64_t q) {
    const uint64_t c = (z ^ ICM_DIGIT_BIAS) - ICM_DIGIT_BIAS;
    return ((int64_t)c < 0) ? c + q : c;
}

// ---------------------------------------------------------------- bounded device waits

// Device status word values written by kernels that give up a bounded wait or find bad input.
enum : uint32_t { ICM_DEV_OK = 0, ICM_DEV_TIMEOUT = 1, ICM_DEV_BADINPUT = 2 };
