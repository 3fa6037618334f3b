// icm_ppmm_noalloc: the small-modulus CRT product of icm_ppmm for callers that cannot allocate
// device memory (for instance code that runs while a CUDA graph is being captured with a
// relaxed allocator policy, embedded hosts with a fixed device memory budget, or plugins whose
// host framework owns every cudaMalloc).  Its workspace -- the query operand's residue planes and
// the byte scratch of per-modulus residues -- lives in one file-scope device array of
// ICM_NOALLOC_SCRATCH_BYTES, which every GPU that loads this library holds until the process ends.
//
// The array's host-side name is only a stand-in for the symbol, not a device address, so the
// device address is looked up once per CUDA context (cudaGetSymbolAddress, with the calling
// thread's device and context current) on the first call made in that context, and that pointer
// is what the kernels receive.  Every
// call shares the array and it keeps the previous call's contents; nothing in it needs to start
// at zero (the planes kernel writes every plane entry, including the zero padding, and phase 1
// writes every residue that phase 2 reads).  Calls that overlap on the GPU race on the array.
#include <mutex>

#include "icm_internal.h"

#define ICM_NOALLOC_SCRATCH_BYTES (64ull << 20)
#define ICM_NOALLOC_MAX_DEVICES 64                  // cached contexts

namespace icm {
icm_status api_fail(icm_status s, const char *msg);
}

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[ICM_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
// looked-up device addresses of the array, keyed by the CUDA context current at the call (the
// runtime's primary context of a device, or a context the caller made current); a context that
// replaces an earlier one (for instance after cudaDeviceReset) gets a new handle and a new lookup
struct CtxAddr {
    void *ctx;
    void *ptr;
};
CtxAddr g_cache[ICM_NOALLOC_MAX_DEVICES] = {};
int g_cached = 0;

using CtxGetCurrent = int (*)(void **);
CtxGetCurrent ctx_get_current() {
    static std::once_flag once;
    static CtxGetCurrent fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult r{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &r) == cudaSuccess &&
            r == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrent>(f);
    });
    return fn;
}

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" icm_status icm_ppmm_noalloc(icm_form form, const uint64_t *q, uint32_t n_limbs, const uint64_t *dev_A,
                                       const uint64_t *dev_B, uint64_t *dev_C, size_t M, size_t N, size_t K,
                                       void *stream) {
    using namespace icm;
    if (form != ICM_FORM_I8_CRT && form != ICM_FORM_F16_CRT)
        return api_fail(ICM_EUNSUPPORTED, "icm_ppmm_noalloc supports the CRT forms only");
    if (!q) return api_fail(ICM_EINVAL, "null prime list");
    if (n_limbs < 1 || n_limbs > ICM_MAX_LIMBS) return api_fail(ICM_EINVAL, "n_limbs must be 1..8");
    for (uint32_t l = 0; l < n_limbs; ++l)
        if (q[l] < 3 || q[l] >= (1ull << 60) || !(q[l] & 1)) return api_fail(ICM_EINVAL, "moduli must be odd and below 2^60");
    I8Consts k;
    const char *why = "";
    if (!make_i8_consts(ICM_FORM_I8_CRT, q, n_limbs, K, k, &why)) return api_fail(ICM_EBOUND, why);
    const bool f16 = form == ICM_FORM_F16_CRT;
    const uint64_t Kp = i8_kpad(K);
    const size_t planes = crt_plane_bytes(f16, n_limbs, k.n_mod, N, Kp);
    const size_t need = a256(planes) + crt_scratch_bytes(n_limbs, k.n_mod, N, M);
    // the size is checked before the operands, so an oversize request is refused with ICM_ENOMEM
    // even when its pointers are null
    if (need > ICM_NOALLOC_SCRATCH_BYTES)
        return api_fail(ICM_ENOMEM, "problem exceeds the 64 MiB static workspace of icm_ppmm_noalloc");
    if ((!dev_A && M && K) || (!dev_B && N && K) || (!dev_C && M && N)) return api_fail(ICM_EINVAL, "null argument");
    if (M == 0 || N == 0) return ICM_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return api_fail(ICM_ECUDA, cudaGetErrorString(e));
    // the cache is keyed on the current context; with none current yet, the runtime binds the
    // device's primary context on its first call (here the lookup itself)
    CtxGetCurrent get_ctx = ctx_get_current();
    void *ctx = nullptr, *looked = nullptr;
    if (!get_ctx || get_ctx(&ctx) != 0) return api_fail(ICM_ECUDA, "cuCtxGetCurrent is not available");
    if (!ctx) {
        e = cudaGetSymbolAddress(&looked, g_noalloc_scratch);
        if (e != cudaSuccess || !looked) return api_fail(ICM_ECUDA, "cudaGetSymbolAddress of the static workspace failed");
        if (get_ctx(&ctx) != 0 || !ctx) return api_fail(ICM_ECUDA, "no current CUDA context");
    }
    void *ws = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (int i = 0; i < g_cached; ++i)
            if (g_cache[i].ctx == ctx) ws = g_cache[i].ptr;
        if (!ws) {
            // first call in this context: resolve the device address of the static array
            if (g_cached == ICM_NOALLOC_MAX_DEVICES) return api_fail(ICM_EUNSUPPORTED, "too many CUDA contexts");
            void *p = looked;
            if (!p) {
                e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
                if (e != cudaSuccess || !p) return api_fail(ICM_ECUDA, "cudaGetSymbolAddress of the static workspace failed");
            }
            e = crt_set_attributes();
            if (e != cudaSuccess) return api_fail(ICM_ECUDA, cudaGetErrorString(e));
            g_cache[g_cached++] = CtxAddr{ctx, p};
            ws = p;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    e = launch_crt_planes(f16, k, dev_B, ws, N, K, Kp, st);
    if (e == cudaSuccess)
        e = launch_ppmm_crt(f16, 256, k, dev_A, false, ws, dev_C, M, N, K, Kp, (char *)ws + a256(planes), st);
    if (e != cudaSuccess) return api_fail(ICM_ECUDA, cudaGetErrorString(e));
    return ICM_OK;
}
