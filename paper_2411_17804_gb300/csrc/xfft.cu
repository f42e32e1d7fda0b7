// Correlator + FFT imager (Eq. intra-station XFFT).
//
// For every ordered element pair (a, b), autos included, the visibility
// V^{alpha beta}_{ab} is gridded with the autocorrelation of the two elements'
// illumination kernels, K_ab[d] = sum_j g_a[j + d] conj(g_b[j]) with g the
// placed conjugate taps, at lags d = (anchor_a - anchor_b) + (ex, ey),
// |ex|, |ey| < K, on the circular N grid; then the grid is multiplied by
// (-1)^(dx+dy) and transformed with exp(+2 pi i l.d / N).  With this kernel
// the result equals the EPIC image of the same voltages.
//
// Only the lower triangle a >= b is stored; the pair (b, a) contributes
// conj(V^{beta alpha}_{ab} K_ab[d]) at lag -d (Hermitian mirror).
//
// A cluster of kRanks CTAs per channel: every CTA holds the grids of the
// needed polarisation products (XX, YY, XY) in shared memory as FP32 and adds
// its share of the baselines' 2 (2K-1)^2 terms with shared-memory atomics;
// the other CTAs then add their grids into rank 0's through distributed
// shared memory, and rank 0 runs the 2D FFTs in place.
#include <cooperative_groups.h>
#include <math.h>

#include "hai_internal.h"

namespace cg = cooperative_groups;

namespace {

constexpr int kThreads = 512;
constexpr int kRanks = 4;              // CTAs per channel (one cluster)

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place radix-2 FFT of n points at stride s in shared memory, exponent +,
// computed by one thread (n <= 64: grids are small and per cadence).
template <int N>
__device__ void fft_line(float2 *x, int s) {
    for (int i = 1, j = 0; i < N; i++) {
        int bit = N >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            const float2 t = x[i * s];
            x[i * s] = x[j * s];
            x[j * s] = t;
        }
    }
    for (int len = 2; len <= N; len <<= 1) {
        const int half = len >> 1;
        for (int k = 0; k < half; k++) {
            float sn, cs;
            sincospif(2.0f * (float)k / (float)len, &sn, &cs);
            const float2 w = make_float2(cs, sn);
            for (int st = 0; st < N; st += len) {
                const float2 a = x[(st + k) * s], b = cmul(x[(st + k + half) * s], w);
                x[(st + k) * s] = make_float2(a.x + b.x, a.y + b.y);
                x[(st + k + half) * s] = make_float2(a.x - b.x, a.y - b.y);
            }
        }
    }
}

template <int N>
__global__ void __cluster_dims__(kRanks, 1, 1) __launch_bounds__(kThreads, 1)
xfft_kernel(const int32_t *__restrict__ vis, int ne, int P, int K, const int32_t *__restrict__ anchors,
            const float2 *__restrict__ taps, float *__restrict__ img, int accumulate) {
    extern __shared__ __align__(16) float2 grid[];          // [np][N][N]
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int np = (P == 2) ? 3 : 1;                         // XX, YY, XY
    const int c = blockIdx.x / kRanks;
    const long long nbl = (long long)ne * (ne + 1) / 2;
    for (int i = threadIdx.x; i < np * N * N; i += kThreads) grid[i] = make_float2(0.f, 0.f);
    __syncthreads();

    const int W = 2 * K - 1;
    for (long long bl = (long long)rank * kThreads + threadIdx.x; bl < nbl; bl += (long long)kRanks * kThreads) {
        // baseline index -> (a, b), a >= b
        int a = (int)((sqrt(8.0 * (double)bl + 1.0) - 1.0) * 0.5);
        while ((long long)(a + 1) * (a + 2) / 2 <= bl) a++;
        while ((long long)a * (a + 1) / 2 > bl) a--;
        const int b = (int)(bl - (long long)a * (a + 1) / 2);
        const int2 *v = reinterpret_cast<const int2 *>(vis) + (((size_t)c * nbl + bl) * P * P);
        float2 vv[4];
        for (int k = 0; k < P * P; k++) vv[k] = make_float2((float)v[k].x, (float)v[k].y);
        const int dx0 = anchors[2 * a] - anchors[2 * b], dy0 = anchors[2 * a + 1] - anchors[2 * b + 1];
        const float2 *ta = taps + (size_t)a * K * K, *tb = taps + (size_t)b * K * K;
        for (int ey = -(K - 1); ey <= K - 1; ey++)
            for (int ex = -(K - 1); ex <= K - 1; ex++) {
                // K_ab[e] = sum over tap pairs with (ua - ub, va - vb) = e of conj(w_a) w_b
                float2 kab = make_float2(0.f, 0.f);
                for (int vb = max(0, -ey); vb < min(K, K - ey); vb++)
                    for (int ub = max(0, -ex); ub < min(K, K - ex); ub++) {
                        const float2 wa = ta[(vb + ey) * K + (ub + ex)], wb = tb[vb * K + ub];
                        kab.x += wa.x * wb.x + wa.y * wb.y;       // conj(wa) wb
                        kab.y += wa.x * wb.y - wa.y * wb.x;
                    }
                if (kab.x == 0.f && kab.y == 0.f) continue;
                const int dx = ((dx0 + ex) % N + N) % N, dy = ((dy0 + ey) % N + N) % N;
                const int cell = dy * N + dx;
                const int mcell = ((N - dy) % N) * N + ((N - dx) % N);   // lag -d
                // products: XX = V^00, YY = V^11, XY = V^01; mirrors use V^00, V^11, V^10
                const int prod[3] = {0, 3, 1};
                const int mprod[3] = {0, 3, 2};
                for (int q = 0; q < np; q++) {
                    const float2 t = cmul(vv[P == 2 ? prod[q] : 0], kab);
                    float2 *g = grid + q * N * N;
                    atomicAdd(&g[cell].x, t.x);
                    atomicAdd(&g[cell].y, t.y);
                    if (a != b) {
                        const float2 m = cmul(vv[P == 2 ? mprod[q] : 0], kab);
                        atomicAdd(&g[mcell].x, m.x);
                        atomicAdd(&g[mcell].y, -m.y);
                    }
                }
                (void)W;
            }
    }
    // the other ranks' grids into rank 0's
    cluster.sync();
    if (rank != 0) {
        float *dst = reinterpret_cast<float *>(cluster.map_shared_rank(grid, 0));
        const float *src = reinterpret_cast<const float *>(grid);
        for (int i = threadIdx.x; i < 2 * np * N * N; i += kThreads) atomicAdd(&dst[i], src[i]);
    }
    cluster.sync();
    if (rank != 0) return;
    // (-1)^(dx+dy), then rows and columns
    for (int i = threadIdx.x; i < np * N * N; i += kThreads) {
        const int dx = i % N, dy = (i / N) % N;
        if ((dx + dy) & 1) grid[i] = make_float2(-grid[i].x, -grid[i].y);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < np * N; r += kThreads) fft_line<N>(grid + (size_t)r * N, 1);
    __syncthreads();
    for (int r = threadIdx.x; r < np * N; r += kThreads) {
        const int q = r / N, col = r % N;
        fft_line<N>(grid + (size_t)q * N * N + col, N);
    }
    __syncthreads();
    const int Q = (P == 2) ? 4 : 1;
    float *out = img + (size_t)c * Q * N * N;
    for (int i = threadIdx.x; i < N * N; i += kThreads) {
        float v0 = grid[i].x;
        if (accumulate) v0 += out[i];
        out[i] = v0;
        if (P == 2) {
            float v1 = grid[N * N + i].x, v2 = grid[2 * N * N + i].x, v3 = grid[2 * N * N + i].y;
            if (accumulate) {
                v1 += out[N * N + i];
                v2 += out[2 * N * N + i];
                v3 += out[3 * N * N + i];
            }
            out[N * N + i] = v1;
            out[2 * N * N + i] = v2;
            out[3 * N * N + i] = v3;
        }
    }
}

template <int N>
hai_status launch(const hai_layout *L, const int32_t *vis, int C, float *img, int accumulate, cudaStream_t st) {
    const int np = (L->n_pol == 2) ? 3 : 1;
    const size_t smem = sizeof(float2) * np * N * N;
    if (smem > (size_t)L->ctx->smem_optin)
        return hai_fail(HAI_ERR_UNSUPPORTED, "hai_xfft_image: grid does not fit in shared memory");
    HAI_CUDA_TRY(cudaFuncSetAttribute(xfft_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int pidx = prof_begin(L->ctx, st);
    xfft_kernel<N><<<C * kRanks, kThreads, smem, st>>>(vis, L->n_elem, L->n_pol, L->ksize, L->d_anchors, L->d_taps,
                                                       img, accumulate);
    prof_end(L->ctx, pidx, st);
    prof_count(L->ctx, 1);
    HAI_CUDA_TRY(cudaGetLastError());
    return HAI_OK;
}

}  // namespace

extern "C" hai_status hai_xfft_image(hai_ctx *ctx, const hai_layout *L, const int32_t *vis, int C, float *img,
                                     int accumulate, void *stream) {
    if (!ctx || !L) return hai_fail(HAI_ERR_INVALID_ARG, "hai_xfft_image: NULL ctx or layout");
    if (L->ctx != ctx) return hai_fail(HAI_ERR_INVALID_ARG, "hai_xfft_image: layout of another context");
    if (C < 0 || (accumulate != 0 && accumulate != 1))
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_xfft_image: bad channel count or flag");
    if (C == 0) return HAI_OK;
    if (!vis || !img) return hai_fail(HAI_ERR_INVALID_ARG, "hai_xfft_image: NULL buffer");
    if (hai_fault_injected("launch")) return hai_fail(HAI_ERR_CUDA, "hai_xfft_image: injected launch failure");
    HAI_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    switch (L->grid_n) {
        case 16: return launch<16>(L, vis, C, img, accumulate, st);
        case 32: return launch<32>(L, vis, C, img, accumulate, st);
        case 64: return launch<64>(L, vis, C, img, accumulate, st);
    }
    return hai_fail(HAI_ERR_UNSUPPORTED, "hai_xfft_image: grid size");
}
