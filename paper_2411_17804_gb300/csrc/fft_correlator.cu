// FFT correlator (Section 4.1.2 and Section 5.2.2: visibilities obtained from
// the accumulated EPIC images by an inverse FFT).
//
// The accumulated image I_ab[l] = sum_t F_a[l] conj(F_b[l]) is the DFT (+) of
// the circular autocorrelation of the checkerboarded grids (-1)^j G[j], so
//   R_ab[d] = (-1)^(dx+dy) / N^2  sum_l I_ab[l] exp(-2 pi i l.d / N)
// is the grid sum_t sum_j G_a[j + d] conj(G_b[j]) at lag d, the same grid the
// correlator + XFFT path fills with V_ab K_ab[d] (zero lag at cell (0, 0)).
// On a lattice with one unit tap per element every lag holds the plain sum of
// the visibilities of the baselines separated by it.
//
// Two passes over the output buffer, which holds the rows in between:
//   rows:    one warp per (channel, product, row): the row of the real XX /
//            YY plane or of the complex XY plane, radix-2 FFT (exponent -)
//            in shared memory, complex row written to the output plane;
//   columns: one CTA per (channel, product, 16 columns), one warp per
//            column: FFT along y, times (-1)^(dx+dy) / N^2, written back; the
//            XY CTA also writes YX[-d] = conj(XY[d]) (I_YX = conj(I_XY)).
// N = 512 keeps each line in registers instead: 64 threads per line, three
// radix-8 passes and two shared-memory exchanges (fft512.cuh), the inverse
// transform taken as conj(FFT(conj(x))); 8 lines per CTA in both passes.
#include <algorithm>

#include "fft512.cuh"
#include "hai_internal.h"

namespace {

constexpr int kThreads = 512;
constexpr int kCols = 16;                 // columns per column CTA = warps per CTA

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Twiddles exp(-2 pi i k / N), k < N / 2.
__device__ __forceinline__ void fill_twiddles(float2 *tw, int N) {
    for (int k = threadIdx.x; k < N / 2; k += blockDim.x) {
        float s, c;
        sincospif(2.0f * (float)k / (float)N, &s, &c);
        tw[k] = make_float2(c, -s);
    }
}

// In-place radix-2 FFT (exponent -) of N points held in bit-reversed order,
// by one warp, with the twiddle table of length N / 2.
__device__ __forceinline__ void warp_ifft(float2 *x, int n, int log2n, const float2 *tw, int lane) {
    for (int s = 0; s < log2n; s++) {
        const int half = 1 << s;
        const int tstep = n >> (s + 1);
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

// Output plane (polarisation pair index alpha * P + beta) of source product
// pr (0 = XX, 1 = YY, 2 = XY).
__device__ __forceinline__ int out_plane(int pr, int P) { return P == 1 ? 0 : (pr == 0 ? 0 : (pr == 1 ? 3 : 1)); }

__global__ void __launch_bounds__(kThreads) fc_rows_kernel(const float *__restrict__ img, int N, int log2n, int P,
                                                           float2 *__restrict__ out) {
    extern __shared__ float2 sm[];
    float2 *tw = sm;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 *line = sm + N / 2 + (size_t)warp * N;
    fill_twiddles(tw, N);
    __syncthreads();
    const int np = (P == 2) ? 3 : 1, Q = (P == 2) ? 4 : 1;
    const int c = blockIdx.x / np, pr = blockIdx.x % np;
    const int y = blockIdx.y * (kThreads / 32) + warp;
    if (y >= N) return;
    const size_t NN = (size_t)N * N;
    const float *re = img + ((size_t)c * Q + (pr == 2 ? 2 : pr)) * NN + (size_t)y * N;
    const float *im = (pr == 2) ? re + NN : nullptr;
    // lane takes N / 32 consecutive points: their bit-reversed slots for one
    // step are a permutation of 32 adjacent entries (no bank conflicts; points
    // x = lane + 32 k would put the lanes N / 32 entries apart)
    if (N >= 32) {
        const int E = N / 32;
        for (int k = 0; k < E; k++) {
            const int x = E * lane + k;
            line[__brev(x) >> (32 - log2n)] = make_float2(__ldg(re + x), im ? __ldg(im + x) : 0.f);
        }
    } else {
        for (int x = lane; x < N; x += 32)
            line[__brev(x) >> (32 - log2n)] = make_float2(__ldg(re + x), im ? __ldg(im + x) : 0.f);
    }
    __syncwarp();
    warp_ifft(line, N, log2n, tw, lane);
    float2 *dst = out + ((size_t)c * P * P + out_plane(pr, P)) * NN + (size_t)y * N;
    for (int x = lane; x < N; x += 32) dst[x] = line[x];
}

__global__ void __launch_bounds__(kThreads) fc_cols_kernel(int N, int log2n, int P, float2 *__restrict__ out) {
    extern __shared__ float2 sm[];
    float2 *tw = sm;
    float2 *F = sm + N / 2;                         // [kCols][N + 1]: the pad spreads the columns over the banks
    const int Fs = N + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    fill_twiddles(tw, N);
    const int np = (P == 2) ? 3 : 1;
    const int c = blockIdx.x / np, pr = blockIdx.x % np;
    const int x0 = blockIdx.y * kCols;
    const size_t NN = (size_t)N * N;
    float2 *plane = out + ((size_t)c * P * P + out_plane(pr, P)) * NN;
    for (int i = threadIdx.x; i < N * kCols; i += kThreads) {
        const int j = i % kCols, y = i / kCols;
        F[(size_t)j * Fs + (__brev(y) >> (32 - log2n))] = plane[(size_t)y * N + x0 + j];
    }
    __syncthreads();
    warp_ifft(F + (size_t)warp * Fs, N, log2n, tw, lane);
    __syncthreads();
    const float inv = 1.0f / (float)NN;
    float2 *mirror = (pr == 2) ? out + ((size_t)c * P * P + 2) * NN : nullptr;   // YX
    for (int i = threadIdx.x; i < N * kCols; i += kThreads) {
        const int j = i % kCols, dy = i / kCols, dx = x0 + j;
        const float s = ((dx + dy) & 1) ? -inv : inv;
        const float2 v = F[(size_t)j * Fs + dy];
        const float2 r = make_float2(v.x * s, v.y * s);
        plane[(size_t)dy * N + dx] = r;
        if (mirror) mirror[(size_t)((N - dy) & (N - 1)) * N + ((N - dx) & (N - 1))] = make_float2(r.x, -r.y);
    }
}

// N = 512, rows: CTA = 8 rows of one (channel, product), thread (r, tau).
__global__ void __launch_bounds__(512) fc512_rows_kernel(const float *__restrict__ img, int P,
                                                         float2 *__restrict__ out) {
    constexpr int N = 512;
    extern __shared__ float2 sm[];
    float2 *tw = sm;                                          // [kTwFloat2]
    float2 *bufs = sm + hai_fft512::kTwFloat2;                // [8][kFftBuf]
    hai_fft512::fill_fft512_tables(tw);
    const int r = threadIdx.x >> 6, tau = threadIdx.x & 63;
    const int np = (P == 2) ? 3 : 1, Q = (P == 2) ? 4 : 1;
    const int c = blockIdx.x / np, pr = blockIdx.x % np;
    const int y = blockIdx.y * 8 + r;
    const size_t NN = (size_t)N * N;
    const float *re = img + ((size_t)c * Q + (pr == 2 ? 2 : pr)) * NN + (size_t)y * N;
    float2 a[8];
#pragma unroll
    for (int m = 0; m < 8; m++)                               // conj of the input: exponent -
        a[m] = make_float2(__ldg(re + tau + 64 * m), pr == 2 ? -__ldg(re + NN + tau + 64 * m) : 0.f);
    __syncthreads();
    hai_fft512::fft512<false>(a, tau, bufs + r * hai_fft512::kFftBuf, tw, [] { __syncthreads(); });
    float2 *dst = out + ((size_t)c * P * P + out_plane(pr, P)) * NN + (size_t)y * N;
#pragma unroll
    for (int j = 0; j < 8; j++) dst[tau + 64 * j] = make_float2(a[j].x, -a[j].y);
}

// N = 512, columns: CTA = 8 adjacent columns of one (channel, product).  The
// columns move between HBM and the registers through a shared tile [8][kTs]
// (which shares its memory with the exchange buffers): loads and stores of
// whole 64-byte row segments (a warp: 4 rows x 8 columns), and tile reads and
// writes of one column's rows by consecutive threads, both free of bank
// conflicts (kTs = 514: columns 4 banks apart).  Thread (col, tau) transforms
// its column; times (-1)^(dx+dy) / N^2; the XY CTA also writes the YX mirror.
constexpr int kTs = 514;

__global__ void __launch_bounds__(512) fc512_cols_kernel(int P, float2 *__restrict__ out) {
    constexpr int N = 512;
    extern __shared__ float2 sm[];
    float2 *tw = sm;
    float2 *bufs = sm + hai_fft512::kTwFloat2;                // exchange buffers, and the column tile
    float2 *tile = bufs;
    static_assert(8 * kTs <= 8 * hai_fft512::kFftBuf, "tile inside the exchange buffers");
    hai_fft512::fill_fft512_tables(tw);
    const int col = threadIdx.x >> 6, tau = threadIdx.x & 63;
    const int lc = threadIdx.x & 7, lr = threadIdx.x >> 3;     // row-segment mapping: column, row of 64
    const int np = (P == 2) ? 3 : 1;
    const int c = blockIdx.x / np, pr = blockIdx.x % np;
    const int x0 = blockIdx.y * 8;
    const size_t NN = (size_t)N * N;
    float2 *plane = out + ((size_t)c * P * P + out_plane(pr, P)) * NN;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const int y = lr + 64 * k;
        tile[lc * kTs + y] = plane[(size_t)y * N + x0 + lc];
    }
    __syncthreads();
    float2 a[8];
#pragma unroll
    for (int m = 0; m < 8; m++) {                             // conj of the input: exponent -
        const float2 v = tile[col * kTs + tau + 64 * m];
        a[m] = make_float2(v.x, -v.y);
    }
    __syncthreads();
    hai_fft512::fft512<false>(a, tau, bufs + col * hai_fft512::kFftBuf, tw, [] { __syncthreads(); });
    __syncthreads();                                          // exchange buffers free: the tile again
    const float inv = 1.0f / (float)NN;
    const int dx = x0 + col;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const int dy = tau + 64 * j;
        const float s = ((dx + dy) & 1) ? -inv : inv;
        tile[col * kTs + dy] = make_float2(a[j].x * s, -a[j].y * s);
    }
    __syncthreads();
    float2 *mirror = (pr == 2) ? out + ((size_t)c * P * P + 2) * NN : nullptr;   // YX
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const int dy = lr + 64 * k;
        const float2 v = tile[lc * kTs + dy];
        plane[(size_t)dy * N + x0 + lc] = v;
        if (mirror)
            mirror[(size_t)((N - dy) & (N - 1)) * N + ((N - x0 - lc) & (N - 1))] = make_float2(v.x, -v.y);
    }
}

}  // namespace

extern "C" hai_status hai_fft_correlate(hai_ctx *ctx, const float *img, int C, int N, int P, float *grid,
                                        void *stream) {
    if (!ctx) return hai_fail(HAI_ERR_INVALID_ARG, "hai_fft_correlate: NULL ctx");
    if (C < 0 || (P != 1 && P != 2)) return hai_fail(HAI_ERR_INVALID_ARG, "hai_fft_correlate: bad C or P");
    int log2n = 0;
    while ((1 << log2n) < N && log2n < 30) log2n++;
    if (N < 16 || N > 512 || (1 << log2n) != N)
        return hai_fail(HAI_ERR_UNSUPPORTED, "hai_fft_correlate: N must be a power of two in [16, 512]");
    if (C == 0) return HAI_OK;
    if (!img || !grid) return hai_fail(HAI_ERR_INVALID_ARG, "hai_fft_correlate: NULL buffer");
    if ((reinterpret_cast<uintptr_t>(img) & 3) || (reinterpret_cast<uintptr_t>(grid) & 7))
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_fft_correlate: img must be 4-byte and grid 8-byte aligned");
    if (hai_fault_injected("launch")) return hai_fail(HAI_ERR_CUDA, "hai_fft_correlate: injected launch failure");
    HAI_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int np = (P == 2) ? 3 : 1;
    const size_t smem = sizeof(float2) * ((size_t)N / 2 + (size_t)kCols * (N + 1));   // both passes
    HAI_CUDA_TRY(hai_allow_dyn_smem(fc_rows_kernel, ctx->smem_optin));
    HAI_CUDA_TRY(hai_allow_dyn_smem(fc_cols_kernel, ctx->smem_optin));
    float2 *out = reinterpret_cast<float2 *>(grid);
    if (N == 512) {
        const size_t smem512 = sizeof(float2) * (hai_fft512::kTwFloat2 + 8 * (size_t)hai_fft512::kFftBuf);
        HAI_CUDA_TRY(hai_allow_dyn_smem(fc512_rows_kernel, ctx->smem_optin));
        HAI_CUDA_TRY(hai_allow_dyn_smem(fc512_cols_kernel, ctx->smem_optin));
        const int pidx = prof_begin(ctx, st);
        fc512_rows_kernel<<<dim3(C * np, N / 8), 512, smem512, st>>>(img, P, out);
        fc512_cols_kernel<<<dim3(C * np, N / 8), 512, smem512, st>>>(P, out);
        prof_end(ctx, pidx, st);
        prof_count(ctx, 2);
        HAI_CUDA_TRY(cudaGetLastError());
        return HAI_OK;
    }
    const int pidx = prof_begin(ctx, st);
    fc_rows_kernel<<<dim3(C * np, (N + kThreads / 32 - 1) / (kThreads / 32)), kThreads, smem, st>>>(img, N, log2n,
                                                                                                     P, out);
    fc_cols_kernel<<<dim3(C * np, N / kCols), kThreads, smem, st>>>(N, log2n, P, out);
    prof_end(ctx, pidx, st);
    prof_count(ctx, 2);
    HAI_CUDA_TRY(cudaGetLastError());
    return HAI_OK;
}
