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
// N = 512 (the dense all-sky lattice) keeps each 512-point line in registers:
// the rows as radix-8 transforms over 64 threads, the columns of a box of at
// most 128 rows as four 128-point transforms per warp (see below), the
// column data staged through shared memory a few samples ahead.  There the
// batches are large (2 channels x 512 samples at a 128-row box, 1 GB of row
// output) and alternate between two scratches in HBM: the row pass of one
// batch runs on a second stream beside the column pass of the previous one.
// As in the small-grid FP32 kernel the box sits at the transform's origin:
// the corner shift multiplies F by a phase common to both polarisations that
// cancels in every product, and the (-1)^(jx+jy) phase-centre factor is an
// output shift by N/2.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "fft512.cuh"
#include "hai_internal.h"

namespace {

using namespace hai_fft512;

constexpr int kRowThreads = 512;        // 16 warps, one box row each
constexpr int kCols = 16;               // image columns per column CTA


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

// ------------------------------------------------------------------ N = 512
// The 512-point transforms of the dense grids in registers: fft512.cuh.

// Row pass, N = 512: blockIdx.x = field of the batch, blockIdx.y = group of
// RPC box rows; thread (r = tid / 64, tau): the row's cells x = tau + 64 m
// gathered from the layout's table, the transform, H[field][y][l] written
// for every l (coalesced: l = tau + 64 j).  The twiddle tables come from
// tw_g (built on the host) into shared memory.
template <int RPC>
__global__ void __launch_bounds__(64 * RPC) large512_rows_kernel(
    const int8_t *__restrict__ volt, int T, int P, int ne, int box_w, int box_h,
    const int32_t *__restrict__ cell_start, const int32_t *__restrict__ entry_elem,
    const float2 *__restrict__ entry_w, const int4 *__restrict__ cell_tab, const float2 *__restrict__ tw_g, Batch bt,
    float2 *__restrict__ H) {
    extern __shared__ float4 sm4[];
    float2 *tw = reinterpret_cast<float2 *>(sm4);      // [kTwFloat2]
    float2 *bufs = tw + kTwFloat2;                      // [RPC][kFftBuf]
    static_assert(kTwFloat2 % 2 == 0, "tables copied as float4");
    for (int i = threadIdx.x; i < kTwFloat2 / 2; i += blockDim.x)
        sm4[i] = reinterpret_cast<const float4 *>(tw_g)[i];
    const int r = threadIdx.x >> 6, tau = threadIdx.x & 63;
    const int f = blockIdx.x;
    const int pol = f % P, tt = (f / P) % bt.tb, cc = f / (P * bt.tb);
    const int y = blockIdx.y * RPC + r;
    const char2 *E = reinterpret_cast<const char2 *>(volt) +
                     ((((size_t)(bt.c0 + cc) * T + (bt.t0 + tt)) * P + pol) * ne);
    float2 a[8];
#pragma unroll
    for (int m = 0; m < 8; m++) {
        const int x = tau + 64 * m;
        float2 g = make_float2(0.f, 0.f);
        if (y < box_h && x < box_w) {
            const int cell = y * box_w + x;
            if (cell_tab) {                             // one entry at most: element and weight in one load
                const int4 d = cell_tab[cell];
                if (d.x >= 0) {
                    const char2 e = E[d.x];
                    const float2 w = make_float2(__int_as_float(d.y), __int_as_float(d.z));
                    g.x = fmaf(w.x, (float)e.x, -w.y * (float)e.y);
                    g.y = fmaf(w.x, (float)e.y, w.y * (float)e.x);
                }
            } else {
                for (int k = cell_start[cell]; k < cell_start[cell + 1]; k++) {
                    const char2 e = E[entry_elem[k]];
                    const float2 w = entry_w[k];        // conj(W~)
                    g.x = fmaf(w.x, (float)e.x, fmaf(-w.y, (float)e.y, g.x));
                    g.y = fmaf(w.x, (float)e.y, fmaf(w.y, (float)e.x, g.y));
                }
            }
        }
        a[m] = g;
    }
    __syncthreads();
    if (box_w <= 128) fft512<true>(a, tau, bufs + r * kFftBuf, tw, [] { __syncthreads(); });
    else fft512<false>(a, tau, bufs + r * kFftBuf, tw, [] { __syncthreads(); });
    if (y < box_h) {
        float2 *out = H + ((size_t)f * box_h + y) * 512;
#pragma unroll
        for (int j = 0; j < 8; j++) out[tau + 64 * j] = a[j];
    }
}

// Column pass, N = 512, two polarisations, boxes taller than 128 rows:
// blockIdx.x = channel of the batch, blockIdx.y = block of kCols512 columns;
// thread (c = tid / 64, tau) transforms column l0 + c of both polarisations
// for every sample of the batch and adds |F_X|^2, |F_Y|^2 and F_X conj(F_Y) at
// rows l_y = tau + 64 j into 32 register accumulators; at the end the image
// columns are read, added to and written once (output pixel shifted by N/2:
// the (-1)^j phase centre).
constexpr int kCols512 = 4;                  // columns per CTA: 256 threads, two CTAs per SM

__global__ void __launch_bounds__(64 * kCols512, 2) large512_cols_kernel(const float2 *__restrict__ H, int box_h,
                                                                       Batch bt, float *__restrict__ img, int add) {
    extern __shared__ float2 sm[];
    float2 *tw = sm;                                    // [kTwFloat2]
    float2 *bufs = sm + kTwFloat2;                      // [2 pols][kCols512 columns][kFftBuf]
    fill_fft512_tables(tw);
    const int c = threadIdx.x >> 6, tau = threadIdx.x & 63;
    const int cc = blockIdx.x, l0 = blockIdx.y * kCols512;
    float acc[4][8];
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[q][j] = 0.f;
    // input m (row tau + 64 m) of polarisation p of sample tt of this channel
    auto in = [&](int tt, int p, int m) -> float2 {
        const size_t f = ((size_t)cc * bt.tb + tt) * 2 + p;
        const int yy = tau + 64 * m;
        return yy < box_h ? H[(f * box_h + yy) * 512 + l0 + c] : make_float2(0.f, 0.f);
    };
    __syncthreads();
    for (int tt = 0; tt < bt.tb; tt++) {
        float2 x[8], yv[8];
#pragma unroll
        for (int m = 0; m < 8; m++) {
            x[m] = in(tt, 0, m);
            yv[m] = in(tt, 1, m);
        }
        fft512<false>(x, tau, bufs + c * kFftBuf, tw, [] { __syncthreads(); });
        fft512<false>(yv, tau, bufs + (kCols512 + c) * kFftBuf, tw, [] { __syncthreads(); });
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const float2 a = x[j], b = yv[j];
            acc[0][j] = fmaf(a.x, a.x, fmaf(a.y, a.y, acc[0][j]));
            acc[1][j] = fmaf(b.x, b.x, fmaf(b.y, b.y, acc[1][j]));
            acc[2][j] = fmaf(a.x, b.x, fmaf(a.y, b.y, acc[2][j]));      // Re X conj(Y)
            acc[3][j] = fmaf(a.y, b.x, fmaf(-a.x, b.y, acc[3][j]));     // Im X conj(Y)
        }
        __syncthreads();                                // exchange buffers free for the next sample
    }
    const int ch = bt.c0 + cc;
    const size_t NN = (size_t)512 * 512;
    const int ox = (l0 + c + 256) & 511;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        float *dst = img + ((size_t)ch * 4 + q) * NN + ox;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int oy = (tau + 64 * j + 256) & 511;
            float v = acc[q][j];
            if (add) v += dst[(size_t)oy * 512];
            dst[(size_t)oy * 512] = v;
        }
    }
}

// ------------------------------------------------------------------ N = 512, box <= 128 x 128
// A 512-point transform whose inputs vanish beyond the first 128 (a box of at
// most 128 cells along the transform) splits by output residue r = k mod 4:
//   F[4 k + r] = sum_{n < 128} (h[n] w512^(n r)) w128^(n k),  k < 128,
// four 128-point transforms of pre-twiddled inputs.  One warp computes one
// such 512-point transform, lane = 8 r + t.  With n = t + 8 m (m < 16) and
// k = k1 + 16 k2 (k1 < 16, k2 < 8), w128^(n k) = w128^(t k1) w8^(t k2)
// w16^(m k1): lane (r, t) takes the 16-point DFT over m of its 16
// pre-twiddled inputs and multiplies output k1 by w128^(t k1); after one
// exchange through shared memory (within the warp: no block barrier) lane
// (r, t) takes the 8-point DFTs over t of k1 = t and k1 = t + 8.  It ends with
// F[4 t + r + 32 h + 64 k2] in v[8 h + k2].  Exponent + throughout.
//
// Twiddle tables (built on the host in double precision, rounded once):
//   Pq[r kPr + 8 m + t] = w512^(r (t + 8 m)), Tq[8 k1 + t] = w128^(t k1).
// Pq's rows are kPr = 136 apart so that one instruction's 32 lanes touch two
// wavefronts; the exchange buffer of a warp, kXq float2 per transform, holds
// value k1 of lane (r, t) at r 152 + 9 k1 + t (writes and reads conflict-free).
constexpr int kPr = 136;
constexpr int kTwq = 4 * kPr + 128;          // float2: Pq, then Tq
constexpr int kXq = 3 * 152 + 15 * 9 + 8;    // float2 per transform's exchange buffer
constexpr size_t kHBytes = (size_t)64 << 20;     // row-pass output of a batch, N = 128, 256 (L2-resident)
constexpr size_t kH512Bytes = (size_t)1 << 30;   // each of the two row scratches at N = 512

// 16-point DFT, exponent +, natural order in and out: m = m1 + 4 m2,
// k = ka + 4 kb; 4-point DFTs over m2, twiddles w16^(m1 ka), 4-point DFTs
// over m1.
__device__ __forceinline__ void dft16(float2 (&a)[16]) {
    const float c8 = 0.92387953251128674f, s8 = 0.38268343236508978f, h = 0.70710678118654752f;
#pragma unroll
    for (int m1 = 0; m1 < 4; m1++) dft4(a[m1], a[m1 + 4], a[m1 + 8], a[m1 + 12]);   // a[m1 + 4 ka]
    a[5] = cmul(a[5], make_float2(c8, s8));                                         // w16^1
    a[9] = make_float2(h * (a[9].x - a[9].y), h * (a[9].x + a[9].y));               // w16^2
    a[13] = cmul(a[13], make_float2(s8, c8));                                       // w16^3
    a[6] = make_float2(h * (a[6].x - a[6].y), h * (a[6].x + a[6].y));               // w16^2
    a[10] = cmuli(a[10]);                                                           // w16^4
    a[14] = make_float2(-h * (a[14].x + a[14].y), h * (a[14].x - a[14].y));         // w16^6
    a[7] = cmul(a[7], make_float2(s8, c8));                                         // w16^3
    a[11] = make_float2(-h * (a[11].x + a[11].y), h * (a[11].x - a[11].y));         // w16^6
    a[15] = cmul(a[15], make_float2(-c8, -s8));                                     // w16^9
#pragma unroll
    for (int ka = 0; ka < 4; ka++) dft4(a[4 * ka], a[4 * ka + 1], a[4 * ka + 2], a[4 * ka + 3]);   // a[4 ka + kb]
    float2 o[16];
#pragma unroll
    for (int ka = 0; ka < 4; ka++)
#pragma unroll
        for (int kb = 0; kb < 4; kb++) o[ka + 4 * kb] = a[4 * ka + kb];
#pragma unroll
    for (int k = 0; k < 16; k++) a[k] = o[k];
}

// Two 512-point transforms (the two polarisations) by one warp, as above;
// xb: the warp's two exchange buffers (2 kXq float2), tw: Pq and Tq in shared
// memory.  Entry: x[m] = h_X[t + 8 m], y[m] = h_Y[t + 8 m].
__device__ __forceinline__ void fft512q2(float2 (&x)[16], float2 (&y)[16], int r, int t, float2 *xb,
                                         const float2 *tw) {
    const float2 *pr = tw + r * kPr + t;
#pragma unroll
    for (int m = 0; m < 16; m++) {
        const float2 w = pr[8 * m];
        x[m] = cmul(x[m], w);
        y[m] = cmul(y[m], w);
    }
    dft16(x);
    dft16(y);
    const float2 *tq = tw + 4 * kPr + t;
#pragma unroll
    for (int k = 1; k < 16; k++) {
        const float2 w = tq[8 * k];
        x[k] = cmul(x[k], w);
        y[k] = cmul(y[k], w);
    }
    float2 *wx = xb + r * 152 + t, *wy = wx + kXq;
#pragma unroll
    for (int k = 0; k < 16; k++) {
        wx[9 * k] = x[k];
        wy[9 * k] = y[k];
    }
    __syncwarp();
    const float2 *rx = xb + r * 152 + 9 * t, *ry = rx + kXq;
    float2 a0[8], a1[8], b0[8], b1[8];
#pragma unroll
    for (int s = 0; s < 8; s++) {
        a0[s] = rx[s];
        a1[s] = rx[72 + s];
        b0[s] = ry[s];
        b1[s] = ry[72 + s];
    }
    __syncwarp();                                        // the buffers are free again
    dft8(a0);
    dft8(a1);
    dft8(b0);
    dft8(b1);
#pragma unroll
    for (int k = 0; k < 8; k++) {
        x[k] = a0[k];
        x[8 + k] = a1[k];
        y[k] = b0[k];
        y[8 + k] = b1[k];
    }
}

__device__ __forceinline__ void load_twq(float2 *dst, const float2 *__restrict__ src) {
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    for (int i = threadIdx.x; i < kTwq / 2; i += blockDim.x) d4[i] = s4[i];
}

// Column pass, boxes of at most 128 rows: one warp per (image column l_x,
// channel of the batch), four adjacent columns per block.  For each sample
// the block copies the four columns of both pols (box_h rows of H, 32 bytes
// per row: whole L2 sectors) into shared memory asynchronously two samples
// ahead; each warp transforms its column along y and adds |F_X|^2, |F_Y|^2
// and F_X conj(F_Y) into 64 register accumulators (16 rows l_y per lane); at
// the end the column is read, added to and written once (output pixel
// shifted by N/2).  The staged rows are kRowQ float2 apart so that a warp's
// reads of rows t + 8 m hit distinct banks.
constexpr int kColsQ = 4;                     // columns (warps) per block
constexpr int kRowQ = 6;                      // float2 per staged row (4 used)
constexpr int kPfq = 3;                       // sample stages in flight
constexpr int kStageQ = 2 * 128 * kRowQ;      // float2 per stage (2 pols x 128 rows)

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait2() { asm volatile("cp.async.wait_group 2;\n" ::: "memory"); }

__global__ void __launch_bounds__(32 * kColsQ, 2) large512q_cols_kernel(const float2 *__restrict__ H, int box_h,
                                                                      const float2 *__restrict__ twq, Batch bt,
                                                                      float *__restrict__ img, int add) {
    extern __shared__ float4 smq[];
    float2 *tw = reinterpret_cast<float2 *>(smq);                 // [kTwq]
    float2 *pb = tw + kTwq;                                       // [kPfq][2 pols][128 rows][kRowQ]
    float2 *xb = pb + kPfq * kStageQ;                             // [kColsQ][2 kXq]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, r = lane >> 3, t = lane & 7;
    const int lx0 = blockIdx.x * kColsQ, lx = lx0 + warp, cc = blockIdx.y;
    xb += warp * 2 * kXq;
    load_twq(tw, twq);
    for (int i = threadIdx.x; i < kPfq * kStageQ; i += blockDim.x) pb[i] = make_float2(0.f, 0.f);
    __syncthreads();                                              // rows >= box_h stay zero
    auto issue = [&](int tt) {                                    // two 16-byte copies per (pol, row)
        const size_t f0 = ((size_t)cc * bt.tb + tt) * 2;
        float2 *dst = pb + (tt % kPfq) * kStageQ;
        for (int i = threadIdx.x; i < 2 * 128 * 2; i += blockDim.x) {
            const int u = i & 1, p = i >> 8, yy = (i >> 1) & 127;
            if (yy < box_h)
                cp_async16(dst + (p * 128 + yy) * kRowQ + 2 * u, H + (((f0 + p) * box_h + yy) * 512 + lx0 + 2 * u));
        }
    };
    float acc[4][16];
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
        for (int j = 0; j < 16; j++) acc[q][j] = 0.f;
    issue(0);
    cp_async_commit();
    if (bt.tb > 1) issue(1);
    cp_async_commit();
    for (int tt = 0; tt < bt.tb; tt++) {
        __syncthreads();                                          // the stage refilled next was read last sample
        if (tt + 2 < bt.tb) issue(tt + 2);
        cp_async_commit();
        cp_async_wait2();
        __syncthreads();                                          // sample tt's copies (every thread's) landed
        const float2 *src = pb + (tt % kPfq) * kStageQ + t * kRowQ + warp;
        float2 x[16], yv[16];
#pragma unroll
        for (int m = 0; m < 16; m++) {
            x[m] = src[8 * m * kRowQ];
            yv[m] = src[(128 + 8 * m) * kRowQ];
        }
        fft512q2(x, yv, r, t, xb, tw);
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const float2 a = x[j], b = yv[j];
            acc[0][j] = fmaf(a.x, a.x, fmaf(a.y, a.y, acc[0][j]));
            acc[1][j] = fmaf(b.x, b.x, fmaf(b.y, b.y, acc[1][j]));
            acc[2][j] = fmaf(a.x, b.x, fmaf(a.y, b.y, acc[2][j]));      // Re X conj(Y)
            acc[3][j] = fmaf(a.y, b.x, fmaf(-a.x, b.y, acc[3][j]));     // Im X conj(Y)
        }
    }
    const int ch = bt.c0 + cc;
    const size_t NN = (size_t)512 * 512;
    const int ox = (lx + 256) & 511;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        float *dst = img + ((size_t)ch * 4 + q) * NN + ox;
#pragma unroll
        for (int h = 0; h < 2; h++)
#pragma unroll
            for (int k2 = 0; k2 < 8; k2++) {
                const int oy = (4 * t + r + 32 * h + 64 * k2 + 256) & 511;
                float v = acc[q][8 * h + k2];
                if (add) v += dst[(size_t)oy * 512];
                dst[(size_t)oy * 512] = v;
            }
    }
}

}  // namespace

bool epic_large_supported(int grid_n) { return grid_n == 128 || grid_n == 256 || grid_n == 512; }

// N = 128, 256: the row-pass output of a batch (64 MB, kept in L2 between the
// two passes).  N = 512: two row scratches of 1 GB (the row pass of one batch
// overlaps the column pass of the previous one, through HBM) and the twiddle
// tables after them.
size_t epic_large_scratch_bytes(int grid_n, int box_h) {
    (void)box_h;
    return grid_n == 512 ? 2 * kH512Bytes + sizeof(float2) * (kTwq + kTwFloat2) : kHBytes;
}

// Pq and Tq (see the N = 512 transforms above) from FP64 sines and cosines.
hai_status epic_large_prepare(hai_layout *L) {
    if (L->grid_n != 512 || !L->d_large_scratch) return HAI_OK;
    std::vector<float2> tab(kTwq);
    auto w512 = [](long long j) {
        const double a = 2.0 * M_PI * (double)(j % 512) / 512.0;
        return make_float2((float)cos(a), (float)sin(a));
    };
    for (int r = 0; r < 4; r++)
        for (int m = 0; m < 16; m++)
            for (int t = 0; t < 8; t++) tab[r * kPr + 8 * m + t] = w512((long long)r * (t + 8 * m));
    for (int k1 = 0; k1 < 16; k1++)
        for (int t = 0; t < 8; t++) tab[4 * kPr + 8 * k1 + t] = w512(4ll * t * k1);
    // the radix-8 transforms' tables: w512^n, w512^(tau k), w64^(t1 k) (k = 1..7)
    tab.resize(kTwq + kTwFloat2);
    float2 *t8 = tab.data() + kTwq;
    for (int n = 0; n < 512; n++) t8[n] = w512(n);
    for (int i = 0; i < 7 * 64; i++) t8[512 + i] = w512((long long)(i & 63) * (1 + (i >> 6)));
    for (int i = 0; i < 7 * 8; i++) t8[512 + 7 * 64 + i] = w512(8ll * (i & 7) * (1 + (i >> 3)));
    cudaError_t e = cudaMemcpy(static_cast<uint8_t *>(L->d_large_scratch) + 2 * kH512Bytes, tab.data(),
                               sizeof(float2) * tab.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return hai_cuda_fail(e, "epic fp32 (large grid): twiddle tables");
    // the second stream and events that overlap the row pass of one batch with
    // the column pass of the previous one
    e = cudaStreamCreateWithFlags(&L->large_stream, cudaStreamNonBlocking);
    for (int i = 0; i < 5 && e == cudaSuccess; i++) e = cudaEventCreateWithFlags(&L->large_ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return hai_cuda_fail(e, "epic fp32 (large grid): stream");
    // per-cell table of the box when no cell holds more than one gather entry
    // (the row pass then reads element and weight in one 16-byte load)
    const int ncell = L->box_w * L->box_h;
    std::vector<int32_t> cstart(ncell + 1);
    e = cudaMemcpy(cstart.data(), L->d_cell_start, sizeof(int32_t) * (ncell + 1), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return hai_cuda_fail(e, "epic fp32 (large grid): gather table");
    for (int c = 0; c < ncell; c++)
        if (cstart[c + 1] - cstart[c] > 1) return HAI_OK;
    std::vector<int32_t> elem(std::max(1, L->nnz));
    std::vector<float2> w(std::max(1, L->nnz));
    if (L->nnz > 0) {
        e = cudaMemcpy(elem.data(), L->d_entry_elem, sizeof(int32_t) * L->nnz, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(w.data(), L->d_entry_w, sizeof(float2) * L->nnz, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return hai_cuda_fail(e, "epic fp32 (large grid): gather table");
    }
    std::vector<int4> cells(std::max(1, ncell));
    for (int c = 0; c < ncell; c++) {
        const bool has = cstart[c + 1] > cstart[c];
        const int k = cstart[c];
        int32_t wx = 0, wy = 0;
        if (has) {
            memcpy(&wx, &w[k].x, sizeof(wx));
            memcpy(&wy, &w[k].y, sizeof(wy));
        }
        cells[c] = has ? make_int4(elem[k], wx, wy, 0) : make_int4(-1, 0, 0, 0);
    }
    e = cudaMalloc(&L->d_large_cell, sizeof(int4) * cells.size());
    if (e == cudaSuccess) e = cudaMemcpy(L->d_large_cell, cells.data(), sizeof(int4) * cells.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return hai_cuda_fail(e, "epic fp32 (large grid): cell table");
    L->dev_bytes += sizeof(int4) * cells.size();
    return HAI_OK;
}

hai_status epic_large_launch(const hai_layout *L, const int8_t *volt, int C, int T, float *img, int accumulate,
                             cudaStream_t st) {
    const int N = L->grid_n, P = L->n_pol;
    if (!epic_large_supported(N) || !L->d_large_scratch)
        return hai_fail(HAI_ERR_UNSUPPORTED, "epic fp32: large-grid path needs N = 128, 256 or 512");
    int log2n = 0;
    while ((1 << log2n) < N) log2n++;
    const size_t field_bytes = sizeof(float2) * (size_t)L->box_h * N;
    const long long fields_cap = (long long)(kHBytes / field_bytes);
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
    if (N == 512 && P == 2) {
        // rows: register-resident radix-8 transforms, 8 rows per CTA, on the
        // layout's second stream into one of two row scratches, so that the
        // row pass of batch i overlaps the column pass of batch i - 1; columns:
        // the 4 x 128-point warp transforms for boxes of at most 128 rows, else
        // radix-8 as the rows.  Batches of 2 channels x as many samples as a
        // scratch holds (512 at a 128-row box): the column pass reads and
        // writes its image columns once per batch, and the two streams meet
        // once per batch.
        constexpr int kRpc = 8;
        constexpr int kCb = 2;
        const uint8_t *tabs = static_cast<const uint8_t *>(L->d_large_scratch) + 2 * kH512Bytes;
        const float2 *twq = reinterpret_cast<const float2 *>(tabs);
        const float2 *tw8 = twq + kTwq;
        const size_t rs_smem = sizeof(float2) * (kTwFloat2 + kRpc * (size_t)kFftBuf);
        const size_t cs_smem = sizeof(float2) * (kTwFloat2 + 2 * kCols512 * (size_t)kFftBuf);
        const size_t cq_smem = sizeof(float2) * (kTwq + (size_t)kPfq * kStageQ + (size_t)kColsQ * 2 * kXq);
        HAI_CUDA_TRY(hai_allow_dyn_smem(large512_rows_kernel<kRpc>, L->ctx->smem_optin));
        HAI_CUDA_TRY(hai_allow_dyn_smem(large512_cols_kernel, L->ctx->smem_optin));
        HAI_CUDA_TRY(hai_allow_dyn_smem(large512q_cols_kernel, L->ctx->smem_optin));
        cudaStream_t rst = L->large_stream;
        cudaEvent_t const *ev = L->large_ev;            // 0, 1: rows done (scratch 0, 1); 2, 3: columns done; 4: fork / join
        HAI_CUDA_TRY(cudaEventRecord(ev[4], st));
        HAI_CUDA_TRY(cudaStreamWaitEvent(rst, ev[4], 0));
        const int cb_max = std::min(C, kCb);
        const long long fields512 = (long long)(kH512Bytes / field_bytes);
        const int tb512 = (int)std::max<long long>(1, std::min<long long>(T, fields512 / ((long long)cb_max * P)));
        int i = 0;
        for (int t0 = 0; t0 < T; t0 += tb512) {
            const int tb = std::min(tb512, T - t0);
            for (int c0 = 0; c0 < C; c0 += cb_max, i++) {
                const int buf = i & 1;
                float2 *Hb = reinterpret_cast<float2 *>(static_cast<uint8_t *>(L->d_large_scratch) + buf * kH512Bytes);
                Batch bt;
                bt.c0 = c0;
                bt.cb = std::min(cb_max, C - c0);
                bt.t0 = t0;
                bt.tb = tb;
                if (i >= 2) HAI_CUDA_TRY(cudaStreamWaitEvent(rst, ev[2 + buf], 0));   // columns of batch i - 2 done
                large512_rows_kernel<kRpc><<<dim3(bt.cb * tb * P, (L->box_h + kRpc - 1) / kRpc), 64 * kRpc, rs_smem,
                                             rst>>>(volt, T, P, L->n_elem, L->box_w, L->box_h, L->d_cell_start,
                                                    L->d_entry_elem, L->d_entry_w,
                                                    static_cast<const int4 *>(L->d_large_cell), tw8, bt, Hb);
                HAI_CUDA_TRY(cudaEventRecord(ev[buf], rst));
                HAI_CUDA_TRY(cudaStreamWaitEvent(st, ev[buf], 0));
                const int add = (t0 > 0 || accumulate) ? 1 : 0;
                if (L->box_h <= 128)
                    large512q_cols_kernel<<<dim3(512 / kColsQ, bt.cb), 32 * kColsQ, cq_smem, st>>>(Hb, L->box_h, twq, bt,
                                                                                                   img, add);
                else
                    large512_cols_kernel<<<dim3(bt.cb, 512 / kCols512), 64 * kCols512, cs_smem, st>>>(Hb, L->box_h, bt,
                                                                                                     img, add);
                HAI_CUDA_TRY(cudaEventRecord(ev[2 + buf], st));
                prof_count(L->ctx, 2);
            }
        }
        // join: the caller's stream after the second stream's last work
        HAI_CUDA_TRY(cudaEventRecord(ev[4], rst));
        HAI_CUDA_TRY(cudaStreamWaitEvent(st, ev[4], 0));
        prof_end(L->ctx, pidx, st);
        HAI_CUDA_TRY(cudaGetLastError());
        return HAI_OK;
    }
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
