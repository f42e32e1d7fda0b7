// Peak-rate probes: the arithmetic rates the roofline fractions of the
// CUDA-core paths and of the legacy int8 tensor path are judged against,
// measured on the device that runs them.  Every thread runs independent
// dependency chains long enough to hide the pipeline latency; the result is
// folded into one word so the compiler cannot drop the work.
#include <stdint.h>

#include "hai_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 4;

// kind 0: scalar FP32 FMA, 2 FLOP each.
__global__ void __launch_bounds__(kThreads) probe_ffma_kernel(long long iters, float seed, unsigned *sink) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) a[c] = seed + (float)(threadIdx.x + c);
    const float m = 0.9999999f, k = 1e-7f;
    for (long long i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) a[c] = fmaf(a[c], m, k);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += a[c];
    if (s == -1.0f) atomicAdd(sink, 1u);
}

// kind 1: packed FP32 FMA on pairs (FFMA2), 4 FLOP each.
__global__ void __launch_bounds__(kThreads) probe_ffma2_kernel(long long iters, float seed, unsigned *sink) {
    float2 a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) a[c] = make_float2(seed + (float)(threadIdx.x + c), seed - (float)c);
    const float2 m = make_float2(0.9999999f, 0.9999998f), k = make_float2(1e-7f, 2e-7f);
    for (long long i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) a[c] = __ffma2_rn(a[c], m, k);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += a[c].x + a[c].y;
    if (s == -1.0f) atomicAdd(sink, 1u);
}

// kind 2: warp-level int8 MMA, mma.sync m16n8k32 s8 x s8 -> s32, 2 x 16 x 8 x
// 32 integer operations each, four independent accumulators per warp.
__global__ void __launch_bounds__(kThreads) probe_imma_kernel(long long iters, unsigned seed, unsigned *sink) {
    const uint32_t a0 = seed ^ threadIdx.x, a1 = a0 * 3u, a2 = a0 * 5u, a3 = a0 * 7u;
    const uint32_t b0 = seed + threadIdx.x, b1 = b0 * 11u;
    int32_t d[4][4] = {};
    for (long long i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < 4; c++)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+r"(d[c][0]), "+r"(d[c][1]), "+r"(d[c][2]), "+r"(d[c][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
    int32_t s = 0;
#pragma unroll
    for (int c = 0; c < 4; c++) s += d[c][0] + d[c][1] + d[c][2] + d[c][3];
    if (s == 0x7fffffff) atomicAdd(sink, 1u);
}

}  // namespace

extern "C" hai_status hai_probe_peak(hai_ctx *ctx, int kind, long long iters, double *ops, void *stream) {
    if (!ctx || !ops) return hai_fail(HAI_ERR_INVALID_ARG, "hai_probe_peak: NULL argument");
    if (kind < 0 || kind > 2 || iters < 1 || iters > (1ll << 24))
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_probe_peak: kind must be 0..2 and iters in [1, 2^24]");
    HAI_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = ctx->num_sms * kCtasPerSm;
    const double threads = (double)blocks * kThreads;
    unsigned *sink = ctx->d_status + 2;                 // the context's probe sink word
    switch (kind) {
        case 0:
            probe_ffma_kernel<<<blocks, kThreads, 0, st>>>(iters, 1.0f, sink);
            *ops = threads * kChains * 2.0 * (double)iters;
            break;
        case 1:
            probe_ffma2_kernel<<<blocks, kThreads, 0, st>>>(iters, 1.0f, sink);
            *ops = threads * kChains * 4.0 * (double)iters;
            break;
        default:
            probe_imma_kernel<<<blocks, kThreads, 0, st>>>(iters, 12345u, sink);
            *ops = (threads / 32.0) * 4.0 * 2.0 * 16 * 8 * 32 * (double)iters;
            break;
    }
    prof_count(ctx, 1);
    HAI_CUDA_TRY(cudaGetLastError());
    return HAI_OK;
}
