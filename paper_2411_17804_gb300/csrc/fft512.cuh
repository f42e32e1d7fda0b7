// Register-resident 512-point FFT building blocks (exponent +), shared by the
// FP32 large-grid EPIC kernels and the FFT correlator.
//
// A 512-point transform by 64 threads, each holding 8 points, in three
// radix-8 passes (512 = 8 x 8 x 8) with two exchanges through shared memory.
// Pass 1: thread tau takes x[tau + 64 m], m < 8, an 8-point DFT over m,
// twiddle w512^(tau k1); pass 2: thread (k1, t1) the 8 values of k1 at
// tau = t1 + 8 t2, an 8-point DFT over t2, twiddle w64^(t1 k2); pass 3: thread
// (k1, k2) the 8 values at t1, an 8-point DFT over t1.  Thread tau ends with
// X[tau + 64 j], j < 8 (natural order, stride 64).  The exchange layouts (rows
// 66 apart, then k1 74 + k2 9 + t1) serve every pass's accesses in two
// shared-memory wavefronts.
#pragma once

#include <cuda_runtime.h>

namespace hai_fft512 {

constexpr int kFftBuf = 589;                 // float2 per transform's exchange buffer

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }          // a * i

// 4-point DFT, exponent +: X_k = sum_m x_m i^(m k), natural order
__device__ __forceinline__ void dft4(float2 &x0, float2 &x1, float2 &x2, float2 &x3) {
    const float2 p = cadd(x0, x2), r = csub(x0, x2), q = cadd(x1, x3), s = cmuli(csub(x1, x3));
    x0 = cadd(p, q);
    x1 = cadd(r, s);
    x2 = csub(p, q);
    x3 = csub(r, s);
}

// 8-point DFT, exponent +, natural order in and out (decimation in frequency:
// the even outputs are the 4-point DFT of a_m + a_(m+4), the odd ones that of
// (a_m - a_(m+4)) w8^m)
__device__ __forceinline__ void dft8(float2 (&a)[8]) {
    const float h = 0.70710678118654752f;     // cos(pi / 4)
    float2 u0 = cadd(a[0], a[4]), u1 = cadd(a[1], a[5]), u2 = cadd(a[2], a[6]), u3 = cadd(a[3], a[7]);
    float2 v0 = csub(a[0], a[4]), v1 = csub(a[1], a[5]), v2 = csub(a[2], a[6]), v3 = csub(a[3], a[7]);
    v1 = make_float2(h * (v1.x - v1.y), h * (v1.x + v1.y));          // * e^(+i pi/4)
    v2 = cmuli(v2);                                                   // * e^(+i pi/2)
    v3 = make_float2(-h * (v3.x + v3.y), h * (v3.x - v3.y));         // * e^(+3i pi/4)
    dft4(u0, u1, u2, u3);
    dft4(v0, v1, v2, v3);
    a[0] = u0; a[2] = u1; a[4] = u2; a[6] = u3;
    a[1] = v0; a[3] = v1; a[5] = v2; a[7] = v3;
}

// The 8-point DFT when only a[0] and a[1] can be non-zero (the first pass of
// a transform whose non-zero inputs all lie in its first quarter).
__device__ __forceinline__ void dft8_first2(float2 (&a)[8]) {
    const float h = 0.70710678118654752f;
    const float2 u0 = a[0], u1 = a[1];
    const float2 v1 = make_float2(h * (u1.x - u1.y), h * (u1.x + u1.y));     // a1 * e^(+i pi/4)
    a[0] = cadd(u0, u1);
    a[2] = cadd(u0, cmuli(u1));
    a[4] = csub(u0, u1);
    a[6] = csub(u0, cmuli(u1));
    a[1] = cadd(u0, v1);
    a[3] = cadd(u0, cmuli(v1));
    a[5] = csub(u0, v1);
    a[7] = csub(u0, cmuli(v1));
}

// Twiddle tables of the 512-point transform in shared memory:
//   tw[n] = w512^n (n < 512), T1[(k - 1) 64 + tau] = w512^(tau k),
//   T2[(k - 1) 8 + t1] = w64^(t1 k) (k = 1..7): read by consecutive threads
//   without bank conflicts (T2 is a broadcast within groups of 8).
constexpr int kTwFloat2 = 512 + 7 * 64 + 7 * 8;

__device__ __forceinline__ void fill_fft512_tables(float2 *tw) {
    for (int k = threadIdx.x; k < 512; k += blockDim.x) {
        float s, c;
        sincospif((float)k / 256.0f, &s, &c);
        tw[k] = make_float2(c, s);
    }
    __syncthreads();
    float2 *T1 = tw + 512, *T2 = T1 + 7 * 64;
    for (int i = threadIdx.x; i < 7 * 64; i += blockDim.x) T1[i] = tw[((i & 63) * (1 + (i >> 6))) & 511];
    for (int i = threadIdx.x; i < 7 * 8; i += blockDim.x) T2[i] = tw[(8 * (i & 7) * (1 + (i >> 3))) & 511];
}

// One 512-point transform by the 64 threads of a group (tau = thread in the
// group), `buf` its exchange buffer, tw the tables above; ends with a[j] =
// X[tau + 64 j].  bar() synchronises every group of the CTA together.  Z2:
// the inputs a[2..7] are zero (skipped in the first pass).
template <bool Z2, typename Bar>
__device__ __forceinline__ void fft512(float2 (&a)[8], int tau, float2 *buf, const float2 *tw, Bar bar) {
    const float2 *T1 = tw + 512, *T2 = T1 + 7 * 64;
    if (Z2) dft8_first2(a);
    else dft8(a);
#pragma unroll
    for (int k = 1; k < 8; k++) a[k] = cmul(a[k], T1[(k - 1) * 64 + tau]);
#pragma unroll
    for (int k = 0; k < 8; k++) buf[k * 66 + tau] = a[k];
    bar();
    const int k1 = tau & 7, q = tau >> 3;
#pragma unroll
    for (int t2 = 0; t2 < 8; t2++) a[t2] = buf[k1 * 66 + q + 8 * t2];
    dft8(a);
#pragma unroll
    for (int k = 1; k < 8; k++) a[k] = cmul(a[k], T2[(k - 1) * 8 + q]);
    bar();
#pragma unroll
    for (int k2 = 0; k2 < 8; k2++) buf[k1 * 74 + k2 * 9 + q] = a[k2];
    bar();
#pragma unroll
    for (int t1 = 0; t1 < 8; t1++) a[t1] = buf[k1 * 74 + q * 9 + t1];
    dft8(a);
}

}  // namespace hai_fft512
