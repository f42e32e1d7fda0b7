// EPIC direct imager, FP32 on CUDA cores, for large grids (N = 128 .. 512):
// Eq. intra-station EPIC followed by the squaring and temporal sum of Eq.
// intra-station squaring.
//
// A 512 x 512 complex field (2 MB) and its image accumulators (4 MB per
// channel) exceed one SM, and the direct DFT-as-GEMM would cost O(N^3), so
// the large grids take the FFT through L2 in two kernels per batch of fields
// (channels x samples x pols):
//   rows:    one warp per (field, box row): gather the row's cells from the
//            layout's gather table (conj(W~) E), place them at the start of an
//            N-point line, radix-2 FFT in shared memory, write the row of
//            H[field][y][l_x] to an L2-resident scratch (box rows only);
//   columns: one CTA per (channel, 16 columns): for each sample of the batch
//            and both pols, the 16 columns of H (box rows, zero elsewhere) are
//            transformed along y in shared memory, then every thread adds
//            |F_X|^2, |F_Y|^2 and F_X conj(F_Y) of its row l_y into register
//            accumulators; at the end of the batch the image columns are
//            read, added to and written once.
// As in the small-grid FP32 kernel the box sits at the transform's origin:
// the corner shift multiplies F by a phase common to both polarisations that
// cancels in every product, and the (-1)^(jx+jy) phase-centre factor is an
// output shift by N/2.
#include <math.h>

#include <algorithm>

#include "hai_internal.h"

namespace {

constexpr int kRowThreads = 512;        // 16 warps, one box row each
constexpr int kCols = 16;               // image columns per column CTA

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Twiddles exp(+2 pi i k / N), k < N / 2, into shared memory.
__device__ __forceinline__ void fill_twiddles(float2 *tw, int N) {
    for (int k = threadIdx.x; k < N / 2; k += blockDim.x) {
        float s, c;
        sincospif(2.0f * (float)k / (float)N, &s, &c);
        tw[k] = make_float2(c, s);
    }
}

// In-place radix-2 FFT (exponent +) of n points in bit-reversed order at
// x[0 .. n), by one warp, with the twiddle table of the full length N.
__device__ __forceinline__ void warp_fft(float2 *x, int n, int log2n, const float2 *tw, int lane) {
    for (int s = 0; s < log2n; s++) {
        const int half = 1 << s;
        const int tstep = n >> (s + 1);               // twiddle index stride
        for (int b = lane; b < n / 2; b += 32) {
            const int pos = b & (half - 1);
            const int i0 = ((b - pos) << 1) + pos, i1 = i0 + half;
            const float2 a = x[i0];
            const float2 t = cmul(x[i1], tw[pos * tstep]);
            x[i0] = make_float2(a.x + t.x, a.y + t.y);
            x[i1] = make_float2(a.x - t.x, a.y - t.y);
        }
        __syncwarp();
    }
}

struct Batch {
    int c0, cb;       // channels [c0, c0 + cb)
    int t0, tb;       // samples [t0, t0 + tb)
};

// Row pass: blockIdx.x = field (cc, tt, pol), blockIdx.y = group of 16 box rows.
__global__ void __launch_bounds__(kRowThreads) large_rows_kernel(
    const int8_t *__restrict__ volt, int T, int P, int ne, int N, int log2n, int box_w, int box_h,
    const int32_t *__restrict__ cell_start, const int32_t *__restrict__ entry_elem,
    const float2 *__restrict__ entry_w, Batch bt, float2 *__restrict__ H) {
    extern __shared__ float2 sm[];
    float2 *tw = sm;                                   // [N / 2]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 *line = sm + N / 2 + (size_t)warp * N;
    fill_twiddles(tw, N);
    __syncthreads();
    const int f = blockIdx.x;
    const int pol = f % P, tt = (f / P) % bt.tb, cc = f / (P * bt.tb);
    const int y = blockIdx.y * (kRowThreads / 32) + warp;
    if (y >= box_h) return;
    const char2 *E = reinterpret_cast<const char2 *>(volt) +
                     ((((size_t)(bt.c0 + cc) * T + (bt.t0 + tt)) * P + pol) * ne);
    for (int x = lane; x < N; x += 32) line[x] = make_float2(0.f, 0.f);
    __syncwarp();
    for (int x = lane; x < box_w; x += 32) {
        const int cell = y * box_w + x;
        float2 g = make_float2(0.f, 0.f);
        for (int k = cell_start[cell]; k < cell_start[cell + 1]; k++) {
            const char2 e = E[entry_elem[k]];
            const float2 w = entry_w[k];                // conj(W~)
            g.x = fmaf(w.x, (float)e.x, fmaf(-w.y, (float)e.y, g.x));
            g.y = fmaf(w.x, (float)e.y, fmaf(w.y, (float)e.x, g.y));
        }
        line[__brev(x) >> (32 - log2n)] = g;
    }
    __syncwarp();
    warp_fft(line, N, log2n, tw, lane);
    float2 *out = H + ((size_t)f * box_h + y) * N;
    for (int l = lane; l < N; l += 32) out[l] = line[l];
}

// Column pass: blockIdx.x = channel of the batch, blockIdx.y = block of 16
// columns; N threads, thread = image row l_y.
template <int P>
__global__ void __launch_bounds__(512) large_cols_kernel(const float2 *__restrict__ H, int N, int log2n, int box_h,
                                                         Batch bt, float *__restrict__ img, int add) {
    extern __shared__ float2 sm[];
    float2 *tw = sm;                                   // [N / 2]
    float2 *F = sm + N / 2;                            // [P][kCols][N + 1]: the pad spreads the columns over the banks
    const int Fs = N + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const int cc = blockIdx.x, l0 = blockIdx.y * kCols;
    const int ly = threadIdx.x;
    constexpr int Q = (P == 2) ? 4 : 1;
    float acc[Q][kCols];
#pragma unroll
    for (int q = 0; q < Q; q++)
#pragma unroll
        for (int j = 0; j < kCols; j++) acc[q][j] = 0.f;
    fill_twiddles(tw, N);
    for (int tt = 0; tt < bt.tb; tt++) {
        __syncthreads();
        // columns l0 .. l0+15 of the box rows, bit-reversed along y, zeros elsewhere
        for (int i = threadIdx.x; i < P * kCols * Fs; i += blockDim.x) F[i] = make_float2(0.f, 0.f);
        __syncthreads();
        for (int i = threadIdx.x; i < P * box_h * kCols; i += blockDim.x) {
            const int j = i % kCols, y = (i / kCols) % box_h, pol = i / (kCols * box_h);
            const size_t f = ((size_t)cc * bt.tb + tt) * P + pol;
            F[((size_t)pol * kCols + j) * Fs + (__brev(y) >> (32 - log2n))] = H[(f * box_h + y) * N + l0 + j];
        }
        __syncthreads();
        for (int line = warp; line < P * kCols; line += nwarp) warp_fft(F + (size_t)line * Fs, N, log2n, tw, lane);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kCols; j++) {
            const float2 a = F[(size_t)j * Fs + ly];
            acc[0][j] = fmaf(a.x, a.x, fmaf(a.y, a.y, acc[0][j]));
            if (P == 2) {
                const float2 b = F[((size_t)kCols + j) * Fs + ly];
                acc[1][j] = fmaf(b.x, b.x, fmaf(b.y, b.y, acc[1][j]));
                acc[2][j] = fmaf(a.x, b.x, fmaf(a.y, b.y, acc[2][j]));      // Re X conj(Y)
                acc[3][j] = fmaf(a.y, b.x, fmaf(-a.x, b.y, acc[3][j]));     // Im X conj(Y)
            }
        }
    }
    // output pixel: (l + N/2) mod N on both axes (phase centre at N/2)
    const int c = bt.c0 + cc;
    const size_t NN = (size_t)N * N;
    const int oy = (ly + N / 2) & (N - 1);
#pragma unroll
    for (int q = 0; q < Q; q++) {
        float *dst = img + ((size_t)c * Q + q) * NN + (size_t)oy * N;
#pragma unroll
        for (int j = 0; j < kCols; j++) {
            const int ox = (l0 + j + N / 2) & (N - 1);
            float v = acc[q][j];
            if (add) v += dst[ox];
            dst[ox] = v;
        }
    }
}

}  // namespace

bool epic_large_supported(int grid_n) { return grid_n == 128 || grid_n == 256 || grid_n == 512; }

size_t epic_large_scratch_bytes(int grid_n, int box_h) {
    (void)grid_n;
    (void)box_h;
    return (size_t)64 << 20;
}

hai_status epic_large_launch(const hai_layout *L, const int8_t *volt, int C, int T, float *img, int accumulate,
                             cudaStream_t st) {
    const int N = L->grid_n, P = L->n_pol;
    if (!epic_large_supported(N) || !L->d_large_scratch)
        return hai_fail(HAI_ERR_UNSUPPORTED, "epic fp32: large-grid path needs N = 128, 256 or 512");
    int log2n = 0;
    while ((1 << log2n) < N) log2n++;
    const size_t field_bytes = sizeof(float2) * (size_t)L->box_h * N;
    const long long fields_cap = (long long)(L->large_scratch_bytes / field_bytes);
    if (fields_cap < P) return hai_fail(HAI_ERR_UNSUPPORTED, "epic fp32: box too large for the row scratch");
    // batch: up to 8 samples of as many channels as the scratch holds
    const int tb_max = (int)std::max<long long>(1, std::min<long long>(8, fields_cap / P));
    const size_t row_smem = sizeof(float2) * ((size_t)N / 2 + (size_t)(kRowThreads / 32) * N);
    const size_t col_smem = sizeof(float2) * ((size_t)N / 2 + (size_t)P * kCols * (N + 1));
    HAI_CUDA_TRY(hai_allow_dyn_smem(large_rows_kernel, L->ctx->smem_optin));
    if (P == 2)
        HAI_CUDA_TRY(hai_allow_dyn_smem(large_cols_kernel<2>, L->ctx->smem_optin));
    else
        HAI_CUDA_TRY(hai_allow_dyn_smem(large_cols_kernel<1>, L->ctx->smem_optin));
    float2 *H = static_cast<float2 *>(L->d_large_scratch);
    const int pidx = prof_begin(L->ctx, st);
    for (int t0 = 0; t0 < T; t0 += tb_max) {
        const int tb = std::min(tb_max, T - t0);
        const int cb_max = (int)std::max<long long>(1, fields_cap / ((long long)tb * P));
        for (int c0 = 0; c0 < C; c0 += cb_max) {
            Batch bt;
            bt.c0 = c0;
            bt.cb = std::min(cb_max, C - c0);
            bt.t0 = t0;
            bt.tb = tb;
            large_rows_kernel<<<dim3(bt.cb * tb * P, (L->box_h + 15) / 16), kRowThreads, row_smem, st>>>(
                volt, T, P, L->n_elem, N, log2n, L->box_w, L->box_h, L->d_cell_start, L->d_entry_elem,
                L->d_entry_w, bt, H);
            const int add = (t0 > 0 || accumulate) ? 1 : 0;
            if (P == 2)
                large_cols_kernel<2><<<dim3(bt.cb, N / kCols), N, col_smem, st>>>(H, N, log2n, L->box_h, bt, img, add);
            else
                large_cols_kernel<1><<<dim3(bt.cb, N / kCols), N, col_smem, st>>>(H, N, log2n, L->box_h, bt, img, add);
            prof_count(L->ctx, 2);
        }
    }
    prof_end(L->ctx, pidx, st);
    HAI_CUDA_TRY(cudaGetLastError());
    return HAI_OK;
}
