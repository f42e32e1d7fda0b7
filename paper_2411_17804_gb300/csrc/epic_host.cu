// EPIC image from host buffers (Eq. intra-station EPIC, then Eq.
// intra-station squaring), the cadence streamed through the GPU in chunks of
// channels so that the copies overlap the imaging.
//
// The channels of a cadence are independent, so chunk k is imaged by
// hai_epic_image on the caller's stream while the context's copy stream moves
// chunk k + 1's voltages in and chunk k - 1's images out (the first two chunks
// are shorter, so the imaging starts early).  Two voltage and
// two image staging buffers alternate between chunks; events order each
// buffer's reuse:
//   copy stream:    H2D(0) | H2D(1) D2H(0) | H2D(2) D2H(1) | ...
//   caller stream:         | image(0)      | image(1)      | ...
// H2D(k + 1) waits for image(k - 1) (its buffer), D2H(k) for image(k); the
// caller's stream finally waits for the last D2H, so the call is as
// asynchronous as hai_epic_image and the caller synchronises its stream
// before reading img.
#include <algorithm>
#include <vector>

#include "hai_internal.h"

namespace {

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Events {
    cudaEvent_t in[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr}, start = nullptr, end = nullptr;
    ~Events() {
        for (cudaEvent_t e : {in[0], in[1], done[0], done[1], start, end})
            if (e) cudaEventDestroy(e);
    }
    cudaError_t create() {
        for (cudaEvent_t *e : {&in[0], &in[1], &done[0], &done[1], &start, &end}) {
            const cudaError_t r = cudaEventCreateWithFlags(e, cudaEventDisableTiming);
            if (r != cudaSuccess) return r;
        }
        return cudaSuccess;
    }
};

}  // namespace

extern "C" hai_status hai_epic_image_host(hai_ctx *ctx, const hai_layout *L, const int8_t *volt, int C, int T,
                                          hai_precision prec, float *img, int accumulate, int chunk, void *stream) {
    if (!ctx || !L) return hai_fail(HAI_ERR_INVALID_ARG, "hai_epic_image_host: NULL ctx or layout");
    if (L->ctx != ctx) return hai_fail(HAI_ERR_INVALID_ARG, "hai_epic_image_host: layout of another context");
    if (C < 0 || T < 0 || chunk < 0) return hai_fail(HAI_ERR_INVALID_ARG, "hai_epic_image_host: negative size");
    if (accumulate != 0 && accumulate != 1)
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_epic_image_host: accumulate must be 0 or 1");
    if (C == 0) return HAI_OK;
    if (!img || (T > 0 && !volt)) return hai_fail(HAI_ERR_INVALID_ARG, "hai_epic_image_host: NULL buffer");
    if (hai_fault_injected("launch")) return hai_fail(HAI_ERR_CUDA, "hai_epic_image_host: injected launch failure");
    HAI_CUDA_TRY(cudaSetDevice(ctx->device));
    const int Q = (L->n_pol == 2) ? 4 : 1, N = L->grid_n;
    const size_t v_ch = (size_t)T * L->n_pol * L->n_elem * 2;            // voltage bytes per channel
    const size_t i_ch = sizeof(float) * Q * (size_t)N * N;               // image bytes per channel
    if (chunk == 0) chunk = std::max(1, (C + 3) / 4);
    chunk = std::min(chunk, C);
    const size_t vb = round256((size_t)chunk * v_ch), ib = round256((size_t)chunk * i_ch);
    if (!ctx->copy_stream) HAI_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    if (ctx->stage_bytes < 2 * (vb + ib)) {
        // cudaFree waits for the device, so no earlier call still uses the old buffers
        HAI_CUDA_TRY(cudaFree(ctx->d_stage));
        ctx->d_stage = nullptr;
        ctx->stage_bytes = 0;
        HAI_CUDA_TRY(cudaMalloc(&ctx->d_stage, 2 * (vb + ib)));
        ctx->stage_bytes = 2 * (vb + ib);
    }
    uint8_t *base = static_cast<uint8_t *>(ctx->d_stage);
    int8_t *vin[2] = {reinterpret_cast<int8_t *>(base), reinterpret_cast<int8_t *>(base + vb)};
    float *idev[2] = {reinterpret_cast<float *>(base + 2 * vb), reinterpret_cast<float *>(base + 2 * vb + ib)};
    cudaStream_t cs = (cudaStream_t)stream, xs = ctx->copy_stream;
    Events ev;
    HAI_CUDA_TRY(ev.create());
    // the copies follow whatever the caller queued before this call
    HAI_CUDA_TRY(cudaEventRecord(ev.start, cs));
    HAI_CUDA_TRY(cudaStreamWaitEvent(xs, ev.start, 0));
    // chunk boundaries: the first two chunks are a quarter and a half of
    // `chunk`, so the imaging starts after a short first copy (the pipeline fill)
    std::vector<int> c0s{0};
    for (int step : {std::max(1, chunk / 4), std::max(1, chunk / 2)})
        if (c0s.back() < C) c0s.push_back(std::min(C, c0s.back() + step));
    while (c0s.back() < C) c0s.push_back(std::min(C, c0s.back() + chunk));
    const int nchunk = (int)c0s.size() - 1;
    auto h2d = [&](int k) -> cudaError_t {
        const int b = k & 1, c0 = c0s[k], cc = c0s[k + 1] - c0s[k];
        cudaError_t e = cudaSuccess;
        if (k >= 2) e = cudaStreamWaitEvent(xs, ev.done[b], 0);   // image(k - 2) has read vin[b]
        if (e == cudaSuccess && T > 0)
            e = cudaMemcpyAsync(vin[b], volt + (size_t)c0 * v_ch, (size_t)cc * v_ch, cudaMemcpyHostToDevice, xs);
        if (e == cudaSuccess && accumulate)
            e = cudaMemcpyAsync(idev[b], img + (size_t)c0 * (i_ch / sizeof(float)), (size_t)cc * i_ch,
                                cudaMemcpyHostToDevice, xs);
        if (e == cudaSuccess) e = cudaEventRecord(ev.in[b], xs);
        return e;
    };
    HAI_CUDA_TRY(h2d(0));
    for (int k = 0; k < nchunk; k++) {
        const int b = k & 1, c0 = c0s[k], cc = c0s[k + 1] - c0s[k];
        if (k + 1 < nchunk) HAI_CUDA_TRY(h2d(k + 1));
        // D2H(k - 2) of idev[b] precedes H2D(k) on the copy stream, so in[b] also
        // means idev[b] is free
        HAI_CUDA_TRY(cudaStreamWaitEvent(cs, ev.in[b], 0));
        const hai_status s = hai_epic_image(ctx, L, vin[b], cc, T, prec, idev[b], accumulate, cs);
        if (s != HAI_OK) return s;
        HAI_CUDA_TRY(cudaEventRecord(ev.done[b], cs));
        HAI_CUDA_TRY(cudaStreamWaitEvent(xs, ev.done[b], 0));
        HAI_CUDA_TRY(cudaMemcpyAsync(img + (size_t)c0 * (i_ch / sizeof(float)), idev[b], (size_t)cc * i_ch,
                                     cudaMemcpyDeviceToHost, xs));
    }
    HAI_CUDA_TRY(cudaEventRecord(ev.end, xs));
    HAI_CUDA_TRY(cudaStreamWaitEvent(cs, ev.end, 0));
    return HAI_OK;
}
