// Autotuner of the large-grid tensor-core EPIC (N = 256, 512, and the split
// operands at N = 128): the channels imaged per internal chunk, which sets
// the samples per batch of the HBM scratch (the scratch holds a fixed number of (channel, sample) pairs, so
// fewer channels per chunk mean longer sample blocks, fewer image read-modify-
// writes per sample and fewer items split between CTAs, but fewer stage-2
// items per batch).  Candidates are timed on a synthetic cadence of the
// caller's shape (random int8 voltages: the kernels' times do not depend on
// the values) and the choice is kept in the layout and, when a cache path is
// given, in a text cache keyed by (device, N, K, P, N_e bucket, precision).
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "hai_internal.h"

namespace {

__global__ void fill_random_kernel(uint32_t *p, size_t n, uint32_t seed) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)i * 2654435761u ^ seed;       // a 32-bit integer hash per word
        x ^= x >> 16;
        x *= 0x7feb352du;
        x ^= x >> 15;
        x *= 0x846ca68bu;
        x ^= x >> 16;
        p[i] = x;
    }
}

std::string cache_key(const hai_layout *L, hai_precision prec) {
    cudaDeviceProp prop;
    std::string dev = "unknown";
    if (cudaGetDeviceProperties(&prop, L->ctx->device) == cudaSuccess)
        dev = "sm" + std::to_string(prop.major) + std::to_string(prop.minor) + "x" + std::to_string(prop.multiProcessorCount);
    int bucket = 0;                                  // N_e bucket: floor(log2 N_e)
    while ((2 << bucket) <= L->n_elem) bucket++;
    return dev + " N" + std::to_string(L->grid_n) + " K" + std::to_string(L->ksize) + " P" + std::to_string(L->n_pol) +
           " ne2^" + std::to_string(bucket) + " prec" + std::to_string((int)prec);
}

bool cache_lookup(const char *path, const std::string &key, int &chunk) {
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        // "<key> | chunk <c> | <ms> ms"
        const char *bar = strchr(line, '|');
        if (!bar) continue;
        std::string k(line, bar - line);
        while (!k.empty() && k.back() == ' ') k.pop_back();
        int c = 0;
        if (k == key && sscanf(bar, "| chunk %d", &c) == 1 && c > 0) {
            chunk = c;                               // the last matching line wins
            found = true;
        }
    }
    fclose(f);
    return found;
}

}  // namespace

extern "C" hai_status hai_autotune(hai_ctx *ctx, hai_layout *L, int C, int T, hai_precision prec, const char *cache_path,
                                   int *chosen) {
    if (!ctx || !L || L->ctx != ctx || C <= 0 || T <= 0)
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_autotune: NULL context or layout, or C, T not positive");
    if (chosen) *chosen = 0;
    if (!epic_big_used(L, prec)) return HAI_OK;      // nothing to tune on this precision's path
    const std::string key = cache_key(L, prec);
    int chunk = 0;
    if (cache_path && cache_lookup(cache_path, key, chunk)) {
        L->big_chunk = chunk;
        if (chosen) *chosen = chunk;
        return HAI_OK;
    }
    HAI_CUDA_TRY(cudaSetDevice(ctx->device));
    const int Ct = std::min(C, 16), Tt = std::min(T, 1024);
    const int Q = L->n_pol == 2 ? 4 : 1;
    const size_t vbytes = (size_t)Ct * Tt * L->n_pol * L->n_elem * 2;
    const size_t ibytes = sizeof(float) * Ct * Q * (size_t)L->grid_n * L->grid_n;
    void *buf = nullptr;
    if (cudaMalloc(&buf, ((vbytes + 255) & ~(size_t)255) + ibytes) != cudaSuccess)
        return hai_fail(HAI_ERR_NO_MEMORY, "hai_autotune: no device memory for the trial cadence");
    int8_t *volt = static_cast<int8_t *>(buf);
    float *img = reinterpret_cast<float *>(static_cast<uint8_t *>(buf) + ((vbytes + 255) & ~(size_t)255));
    fill_random_kernel<<<1024, 256>>>(reinterpret_cast<uint32_t *>(volt), vbytes / 4, 0x9e3779b9u);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    std::vector<int> cands;
    for (int c = 1; c < Ct; c *= 2) cands.push_back(c);
    cands.push_back(Ct);
    const int old = L->big_chunk;
    int best = 0;
    double best_ms = 1e30;
    hai_status st = HAI_OK;
    const int prof = ctx->prof_on;
    ctx->prof_on = 0;                                // trial launches stay out of the profile
    for (int c : cands) {
        if (e != cudaSuccess) break;
        L->big_chunk = c;
        st = hai_epic_image(ctx, L, volt, Ct, Tt, prec, img, 0, nullptr);       // warm-up
        if (st != HAI_OK) break;
        e = cudaEventRecord(e0, nullptr);
        for (int r = 0; r < 2 && e == cudaSuccess && st == HAI_OK; r++)
            st = hai_epic_image(ctx, L, volt, Ct, Tt, prec, img, 0, nullptr);
        if (e == cudaSuccess) e = cudaEventRecord(e1, nullptr);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (st != HAI_OK || e != cudaSuccess) break;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    ctx->prof_on = prof;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (st != HAI_OK) {
        L->big_chunk = old;
        return st;
    }
    if (e != cudaSuccess) {
        L->big_chunk = old;
        return hai_cuda_fail(e, "hai_autotune: trial timing");
    }
    L->big_chunk = best;
    if (chosen) *chosen = best;
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s | chunk %d | %.4f ms per trial cadence of %d x %d\n", key.c_str(), best, best_ms / 2, Ct, Tt);
            fclose(f);
        }
    }
    return HAI_OK;
}
