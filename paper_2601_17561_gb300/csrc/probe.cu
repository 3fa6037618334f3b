// Peak-rate probes for roofline denominators (not part of the paper's method): issue-bound loops
// of one instruction class, all operands in registers, timed with CUDA events on the caller's
// stream.  kind 0: IMAD.WIDE (u32 x u32 + u64), kind 1: mma.sync m16n8k32 s8 (MACs), kind 2:
// mma.sync m16n8k16 f16 -> f32 (MACs).
#include "icm_internal.h"

namespace {

__global__ void k_probe_imadw(uint64_t *out, int iters) {
    uint32_t x[8];
    for (int j = 0; j < 8; ++j) x[j] = 2654435761u * (threadIdx.x + j + 1);
    uint64_t acc[16];
    for (int j = 0; j < 16; ++j) acc[j] = j;
    uint32_t y = threadIdx.x * 7 + 3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] += (uint64_t)x[j & 7] * y;
        y += 1;
    }
    uint64_t s = 0;
    for (int j = 0; j < 16; ++j) s ^= acc[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_probe_s8(uint64_t *out, int iters) {
    int a0 = threadIdx.x, a1 = a0 * 3, a2 = a0 ^ 5, a3 = a0 + 7, b0 = a0 * 11, b1 = a0 ^ 13;
    int c[8][4] = {};
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                         : "+r"(c[j][0]), "+r"(c[j][1]), "+r"(c[j][2]), "+r"(c[j][3])
                         : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
    int s = 0;
    for (int j = 0; j < 8; ++j) for (int t = 0; t < 4; ++t) s += c[j][t];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (uint64_t)s;
}

__global__ void k_probe_f16(uint64_t *out, int iters) {
    uint32_t a0 = 0x3C003C00u + threadIdx.x, b0 = 0x3C003C00u;
    float c[8][4] = {};
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                         : "+f"(c[j][0]), "+f"(c[j][1]), "+f"(c[j][2]), "+f"(c[j][3])
                         : "r"(a0), "r"(a0), "r"(a0), "r"(a0), "r"(b0), "r"(b0));
    }
    float s = 0;
    for (int j = 0; j < 8; ++j) for (int t = 0; t < 4; ++t) s += c[j][t];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (uint64_t)s;
}

}  // namespace

extern "C" icm_status icm_probe_peak(int kind, double *ops_per_s, void *stream) {
    if (!ops_per_s || kind < 0 || kind > 2) { icm::set_error("bad probe arguments"); return ICM_EINVAL; }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 4, threads = 256;
    const int iters = kind == 0 ? 40000 : 8000;
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t *out = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&out, (size_t)blocks * threads * 8, st);
    if (e != cudaSuccess) { icm::set_error(cudaGetErrorString(e)); return ICM_ECUDA; }
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    auto launch = [&](int it) {
        if (kind == 0) k_probe_imadw<<<blocks, threads, 0, st>>>(out, it);
        else if (kind == 1) k_probe_s8<<<blocks, threads, 0, st>>>(out, it);
        else k_probe_f16<<<blocks, threads, 0, st>>>(out, it);
    };
    launch(iters / 8);                                   // warm-up
    cudaEventRecord(a, st);
    launch(iters);
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaFreeAsync(out, st);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) { icm::set_error(cudaGetErrorString(e)); return ICM_ECUDA; }
    const double warps = (double)blocks * threads / 32;
    double ops;
    if (kind == 0) ops = (double)blocks * threads * iters * 16;
    else if (kind == 1) ops = warps * iters * 8 * 4096.0;
    else ops = warps * iters * 8 * 2048.0;
    *ops_per_s = ops / (ms * 1e-3);
    return ICM_OK;
}
