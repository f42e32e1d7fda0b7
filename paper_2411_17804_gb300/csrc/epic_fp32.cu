// EPIC direct imager, FP32 on CUDA cores (Eq. intra-station EPIC followed by
// the squaring and temporal sum of Eq. intra-station squaring), for grids of
// N = 16, 32, 64 (larger grids: epic_large.cu).
//
// In both kernels here one CTA sums a contiguous range of the flattened
// (channel, sample) index.  At N = 64 the 64-point lines are held in
// registers by groups of 8 lanes (epic64_kernel, described below); for
// N = 16 and 32, and as the fallback when that kernel's shared memory does not
// fit, epic_fp32_kernel does, per group of kSamples samples:
//   1. stages the int8 voltages of the group in shared memory;
//   2. row pass: one thread per (sample, pol, box row) gathers the gridded
//      row sum_a conj(W~) E_a from the layout's gather table and transforms
//      it along x with an N-point radix-2 FFT held in registers;
//   3. column pass: one thread per (sample, pol, column) transforms along y,
//      reading and writing its own column of the same shared buffer;
//   4. squaring: every thread owns N*N/256 pixels and adds F_X conj(F_Y)
//      products to register accumulators.
// Only the kernel's bounding box is transformed, placed at the grid origin.
// Shifting the input by (bx0, by0) multiplies F by exp(+2 pi i l.b / N), a
// phase common to both polarisations that cancels in every F_a conj(F_b);
// the (-1)^(jx+jy) phase-centre factor is an output shift by N/2.
#include <math.h>

#include <algorithm>

#include "fft512.cuh"
#include "hai_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kSamples = 2;        // samples per group
constexpr int kTwN = 64;           // twiddle table resolution

__constant__ float2 c_tw[kTwN / 2];   // exp(+2 pi i m / 64), m < 32

__host__ __device__ constexpr int bitrev(int i, int n) {
    int r = 0;
    for (int b = 1; b < n; b <<= 1) r = (r << 1) | ((i & b) ? 1 : 0);
    return r;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// In-register radix-2 decimation-in-time FFT, X[k] = sum_n x[n] e^{+2 pi i nk/N}.
template <int N>
__device__ __forceinline__ void fft_reg(float2 (&x)[N]) {
#pragma unroll
    for (int i = 0; i < N; i++) {
        const int j = bitrev(i, N);
        if (i < j) {
            float2 t = x[i];
            x[i] = x[j];
            x[j] = t;
        }
    }
#pragma unroll
    for (int len = 2; len <= N; len <<= 1) {
        const int half = len / 2;
#pragma unroll
        for (int k = 0; k < half; k++) {
#pragma unroll
            for (int s = 0; s < N; s += len) {
                float2 a = x[s + k], b = x[s + k + half], bw;
                if (k == 0) {
                    bw = b;
                } else if (4 * k == len) {
                    bw = make_float2(-b.y, b.x);               // times +i
                } else {
                    bw = cmul(b, c_tw[k * (kTwN / len)]);
                }
                x[s + k] = make_float2(a.x + bw.x, a.y + bw.y);
                x[s + k + half] = make_float2(a.x - bw.x, a.y - bw.y);
            }
        }
    }
}

template <int N, int P>
struct EpicSmem {
    static constexpr int NP = N + 1;                       // padded row stride
    static constexpr int kBuf = kSamples * P * N * NP;     // float2 count
};

// Gridded value of one cell: sum over the cell's gather entries.
__device__ __forceinline__ float2 grid_cell(int cell, const int32_t *__restrict__ cstart,
                                            const int32_t *__restrict__ celem,
                                            const float2 *__restrict__ cw, const char2 *e) {
    float2 acc = make_float2(0.f, 0.f);
    const int b = __ldg(cstart + cell), end = __ldg(cstart + cell + 1);
    for (int i = b; i < end; i++) {
        const int a = __ldg(celem + i);
        const float2 w = __ldg(cw + i);
        const char2 v = e[a];
        const float er = (float)v.x, ei = (float)v.y;
        acc.x = fmaf(w.x, er, fmaf(-w.y, ei, acc.x));
        acc.y = fmaf(w.x, ei, fmaf(w.y, er, acc.y));
    }
    return acc;
}

template <int N, int P>
__global__ void __launch_bounds__(kThreads, 1)
epic_fp32_kernel(const int8_t *__restrict__ volt, int C, int T, int ne, long long len,
                 int box_w, int box_h, const int32_t *__restrict__ cstart,
                 const int32_t *__restrict__ celem, const float2 *__restrict__ cw,
                 float *__restrict__ out, int direct, int accumulate) {
    constexpr int Q = (P == 2) ? 4 : 1;
    constexpr int NP = EpicSmem<N, P>::NP;
    constexpr int PIX = N * N / kThreads;
    static_assert(N * N % kThreads == 0, "pixels per thread");
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *buf = reinterpret_cast<float2 *>(smem);
    char2 *vs = reinterpret_cast<char2 *>(smem + sizeof(float2) * EpicSmem<N, P>::kBuf);

    const int tid = threadIdx.x;
    const long long total = (long long)C * T;
    const long long s0 = (long long)blockIdx.x * len;
    const long long s1 = min(total, s0 + len);
    const int sample_elems = P * ne;                 // char2 per sample

    float acc[PIX][Q];
#pragma unroll
    for (int m = 0; m < PIX; m++)
#pragma unroll
        for (int q = 0; q < Q; q++) acc[m][q] = 0.f;

    int seg = 0;
    int cur_c = (int)(s0 / T);
    auto flush = [&](int c, int sgm) {
        float *dst;
        if (direct) dst = out + (size_t)c * Q * N * N;
        else dst = out + ((size_t)blockIdx.x * 2 + sgm) * Q * N * N;
#pragma unroll
        for (int m = 0; m < PIX; m++) {
            const int pix = tid + m * kThreads;
#pragma unroll
            for (int q = 0; q < Q; q++) {
                float v = acc[m][q];
                if (direct && accumulate) v += dst[(size_t)q * N * N + pix];
                dst[(size_t)q * N * N + pix] = v;
                acc[m][q] = 0.f;
            }
        }
    };

    for (long long s = s0; s < s1;) {
        const int c = (int)(s / T);
        if (c != cur_c) {
            flush(cur_c, seg);
            seg++;
            cur_c = c;
        }
        const long long chan_end = (long long)(c + 1) * T;
        const int ng = (int)min((long long)kSamples, min(s1, chan_end) - s);

        // 1. stage voltages of the group (contiguous bytes)
        {
            const size_t nbytes = (size_t)ng * sample_elems * 2;
            const int8_t *src = volt + (size_t)s * sample_elems * 2;
            int8_t *dst = reinterpret_cast<int8_t *>(vs);
            if ((((uintptr_t)src) & 15) == 0 && (nbytes & 15) == 0) {
                const int4 *s4 = reinterpret_cast<const int4 *>(src);
                int4 *d4 = reinterpret_cast<int4 *>(dst);
                for (size_t i = tid; i < nbytes / 16; i += kThreads) d4[i] = __ldg(s4 + i);
            } else {
                for (size_t i = tid; i < nbytes; i += kThreads) dst[i] = src[i];
            }
        }
        __syncthreads();

        // 2. row pass: grid + FFT along x
        for (int task = tid; task < ng * P * box_h; task += kThreads) {
            const int g = task / (P * box_h);
            const int p = (task / box_h) % P;
            const int y = task % box_h;
            const char2 *e = vs + (size_t)(g * P + p) * ne;
            float2 x[N];
#pragma unroll
            for (int u = 0; u < N; u++)
                x[u] = (u < box_w) ? grid_cell(y * box_w + u, cstart, celem, cw, e) : make_float2(0.f, 0.f);
            fft_reg<N>(x);
            float2 *row = buf + (size_t)(g * P + p) * N * NP + (size_t)y * NP;
#pragma unroll
            for (int k = 0; k < N; k++) row[k] = x[k];
        }
        __syncthreads();

        // 3. column pass: FFT along y (rows >= box_h are zero)
        for (int task = tid; task < ng * P * N; task += kThreads) {
            const int gp = task / N;
            const int k = task % N;
            float2 *col = buf + (size_t)gp * N * NP + k;
            float2 x[N];
#pragma unroll
            for (int r = 0; r < N; r++) x[r] = (r < box_h) ? col[(size_t)r * NP] : make_float2(0.f, 0.f);
            fft_reg<N>(x);
#pragma unroll
            for (int r = 0; r < N; r++) col[(size_t)r * NP] = x[r];
        }
        __syncthreads();

        // 4. squaring and accumulation (pixel l reads F at l + N/2 mod N)
#pragma unroll
        for (int m = 0; m < PIX; m++) {
            const int pix = tid + m * kThreads;
            const int ly = pix / N, lx = pix % N;
            const int src = ((ly + N / 2) & (N - 1)) * NP + ((lx + N / 2) & (N - 1));
            for (int g = 0; g < ng; g++) {
                const float2 fx = buf[(size_t)(g * P) * N * NP + src];
                acc[m][0] = fmaf(fx.x, fx.x, fmaf(fx.y, fx.y, acc[m][0]));
                if (P == 2) {
                    const float2 fy = buf[(size_t)(g * P + 1) * N * NP + src];
                    acc[m][Q > 1 ? 1 : 0] = fmaf(fy.x, fy.x, fmaf(fy.y, fy.y, acc[m][Q > 1 ? 1 : 0]));
                    acc[m][Q > 2 ? 2 : 0] = fmaf(fx.x, fy.x, fmaf(fx.y, fy.y, acc[m][Q > 2 ? 2 : 0]));
                    acc[m][Q > 3 ? 3 : 0] = fmaf(fx.y, fy.x, fmaf(-fx.x, fy.y, acc[m][Q > 3 ? 3 : 0]));
                }
            }
        }
        __syncthreads();
        s += ng;
    }
    if (s1 > s0) flush(cur_c, seg);
}

// ------------------------------------------------------------------ N = 64
// The 64 x 64 grid with every 64-point line in registers: a group of 8 lanes
// per line, lane t holding points t + 8 m (m < 8).  With k = k1 + 8 k2,
// w64^((t + 8 m) k) = w64^(t k1) w8^(t k2) w8^(m k1): lane t takes the
// 8-point DFT over m (only m < 4 when the box spans at most 32 cells along
// the line), multiplies output k1 by w64^(t k1), and after one exchange
// through the group's shared scratch (within the warp) lane j takes the
// 8-point DFT over t of the values of k1 = j, ending with X[j + 8 k2] in
// a[k2].  Exponent + throughout.
//
// Per phase of one or two samples: row pass (a group per box row and sample,
// or per (box row, pol): gather, transform along x, row written to H), then
// column pass (a group per column, both pols, sample by sample: transform
// along y, then |F_X|^2, |F_Y|^2 and F_X conj(F_Y) of its 8 pixels into
// register accumulators).  The row pass of phase i and the column pass of
// phase i - 1 run together (H and the staged voltages double-buffered), so a
// phase costs one block barrier.
//
// Shared layouts, all accesses in the minimum two wavefronts per 8-byte
// access: H[sample][p][y][(k + 2 (y & 7)) & 63] with pol and sample planes
// 8 (mod 16) float2 apart (a half-warp writes one row of both samples, or of
// both pols, or rows y and y + 4 of one pol, and reads rows t + 8 m of two
// adjacent columns); the exchange scratch of a group holds value k of lane t
// at 9 k + t, groups 72 float2 (8 mod 16) apart, one pol at a time.
constexpr int k64Threads = 512;                  // 64 groups of 8 lanes
constexpr int k64Xs = 72;                        // float2 of exchange scratch per group (one pol at a time)

__device__ __forceinline__ void dft8_first4(float2 (&a)[8]) {
    // inputs a[4..7] zero: the even outputs are the 4-point DFT of a[0..3],
    // the odd ones that of a[m] w8^m
    const float h = 0.70710678118654752f;
    float2 v0 = a[0], v1 = a[1], v2 = a[2], v3 = a[3];
    v1 = make_float2(h * (v1.x - v1.y), h * (v1.x + v1.y));          // * e^(+i pi/4)
    v2 = hai_fft512::cmuli(v2);                                       // * e^(+i pi/2)
    v3 = make_float2(-h * (v3.x + v3.y), h * (v3.x - v3.y));         // * e^(+3i pi/4)
    float2 u0 = a[0], u1 = a[1], u2 = a[2], u3 = a[3];
    hai_fft512::dft4(u0, u1, u2, u3);
    hai_fft512::dft4(v0, v1, v2, v3);
    a[0] = u0; a[2] = u1; a[4] = u2; a[6] = u3;
    a[1] = v0; a[3] = v1; a[5] = v2; a[7] = v3;
}

__device__ __forceinline__ void cp_async16_64(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// Shared memory of the N = 64 kernel.  SP samples per phase (2 when the box
// is at most 32 rows and shared memory allows, else 1); sample si of a phase
// and pol p keep their H plane at si SO + p PO, SO = 8 (mod 16) too, so that
// a half-warp writing one row of two samples stays within two wavefronts.
// TS: the gather table (cell starts, then {element, conj(W~)} as int4 per
// entry) is copied into shared memory at the start.
template <int P, bool PX, bool PY, int SP, bool TS>
struct Epic64Smem {
    static constexpr int HR = PY ? 32 : 64;                  // rows of H
    static constexpr int PO = HR * 64 + 8;                   // pol plane stride (float2)
    static constexpr int SO = (P * PO + 15) / 16 * 16 + 8;   // sample stride
    static constexpr int HB = SP * SO;                        // one of the two H buffers
    static constexpr size_t fixed = sizeof(float2) * (2 * (size_t)HB + 64 * (size_t)k64Xs);
    __host__ __device__ static size_t vbuf(int ne) { return ((size_t)SP * P * ne * 2 + 15) / 16 * 16; }
    __host__ __device__ static size_t cbytes(int ncell) { return TS ? ((size_t)(ncell + 1) * 4 + 15) / 16 * 16 : 0; }
    __host__ __device__ static size_t bytes(int ne, int ncell, int nnz) {
        return fixed + 2 * vbuf(ne) + cbytes(ncell) + (TS ? (size_t)nnz * 16 : 0);
    }
};

// Same arguments and outputs as epic_fp32_kernel<64, P> (nnz = the table's
// entry count); PX / PY: the box spans at most 32 cells along x / y.  The
// int8 voltages of the next phase are copied into shared memory (16-byte
// cp.async when vec16) while the current one is imaged.
//
// Row tasks: warp w takes rows w and 31 - w (+ 32), so that the rows beyond a
// box of fewer than 32 spread over the four schedulers.  SP = 2: group g
// takes its row of sample g & 1 of the phase, both pols (one walk of the
// gather table for both); SP = 1, P = 2: pol g & 1; P = 1: rows g and g + 4
// paired in a half-warp.  The exchanges go one pol at a time.
template <int P, bool PX, bool PY, int SP, bool TS>
__global__ void __launch_bounds__(k64Threads, 1)
epic64_kernel(const int8_t *__restrict__ volt, int C, int T, int ne, long long len, int box_w, int box_h,
              const int32_t *__restrict__ cstart_g, const int32_t *__restrict__ celem,
              const float2 *__restrict__ cw, int nnz, float *__restrict__ out, int direct, int accumulate,
              int vec16) {
    constexpr int Q = (P == 2) ? 4 : 1;
    using S = Epic64Smem<P, PX, PY, SP, TS>;
    constexpr int PO = S::PO, SO = S::SO, HB = S::HB;
    constexpr int RP = (SP == 2) ? P : 1;                    // pols per row task
    constexpr int RR = (SP == 2 || P == 2) && !PY ? 2 : 1;   // row tasks per group
    static_assert(SP == 1 || PY, "two samples per phase need a box of at most 32 rows");
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *Hs = reinterpret_cast<float2 *>(smem);                        // [2][HB]
    float2 *xs = Hs + 2 * HB + (threadIdx.x >> 3) * k64Xs;                // this group's scratch
    unsigned char *vs = smem + S::fixed;                                  // [2][vstride]
    const int vbytes = P * ne * 2;                                        // one sample
    const int vstride = (int)S::vbuf(ne);
    const int ncell = box_w * box_h;
    int32_t *cs_s = reinterpret_cast<int32_t *>(vs + 2 * (size_t)vstride);
    int4 *ent_s = reinterpret_cast<int4 *>(reinterpret_cast<unsigned char *>(cs_s) + S::cbytes(ncell));

    const int tid = threadIdx.x, t = tid & 7, g = tid >> 3;
    const long long total = (long long)C * T;
    const long long s0 = (long long)blockIdx.x * len;
    const long long s1 = min(total, s0 + len);
    if (s0 >= s1) return;
    const int n = (int)(s1 - s0);
    const int nph = (n + SP - 1) / SP;

    if (TS) {
        for (int i = tid; i <= ncell; i += k64Threads) cs_s[i] = __ldg(cstart_g + i);
        for (int i = tid; i < nnz; i += k64Threads) {
            const float2 w = __ldg(cw + i);
            ent_s[i] = make_int4(__ldg(celem + i), __float_as_int(w.x), __float_as_int(w.y), 0);
        }
    }
    const int32_t *cstart = TS ? cs_s : cstart_g;

    // w64^(t k), k = 1..7, from the table of w64^m, m < 32
    float2 tw[8];
#pragma unroll
    for (int k = 1; k < 8; k++) {
        const int m = t * k;
        const float2 v = c_tw[m & 31];
        tw[k] = m < 32 ? v : make_float2(-v.x, -v.y);
    }

    auto load = [&](int ph, int b) {
        const int bytes = min(SP, n - SP * ph) * vbytes;
        const int8_t *src = volt + (size_t)(s0 + (long long)SP * ph) * vbytes;
        unsigned char *dst = vs + (size_t)b * vstride;
        if (vec16) {
            for (int i = tid; i < bytes / 16; i += k64Threads) cp_async16_64(dst + 16 * i, src + 16 * i);
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        } else {
            const char2 *s2 = reinterpret_cast<const char2 *>(src);
            char2 *d2 = reinterpret_cast<char2 *>(dst);
            for (int i = tid; i < bytes / 2; i += k64Threads) d2[i] = s2[i];
        }
    };

    float acc[8][Q];
#pragma unroll
    for (int k = 0; k < 8; k++)
#pragma unroll
        for (int q = 0; q < Q; q++) acc[k][q] = 0.f;
    const int col = g;                                   // column pass: column of this group
    int cur_c = (int)(s0 / T), seg = 0;
    auto flush = [&](int c, int sgm) {
        float *dst = direct ? out + (size_t)c * Q * 4096 : out + ((size_t)blockIdx.x * 2 + sgm) * Q * 4096;
        const int lx = (col + 32) & 63;
#pragma unroll
        for (int k2 = 0; k2 < 8; k2++) {
            const int pix = ((t + 8 * k2 + 32) & 63) * 64 + lx;
#pragma unroll
            for (int q = 0; q < Q; q++) {
                float v = acc[k2][q];
                if (direct && accumulate) v += dst[(size_t)q * 4096 + pix];
                dst[(size_t)q * 4096 + pix] = v;
                acc[k2][q] = 0.f;
            }
        }
    };
    // second half of a 64-point line: a[k1] (twiddled) of lane t in, X[t + 8 k2] in a[k2] out
    auto finish = [&](float2 (&a)[8]) {
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 8; k++) xs[9 * k + t] = a[k];
        __syncwarp();
#pragma unroll
        for (int u = 0; u < 8; u++) a[u] = xs[9 * t + u];
        hai_fft512::dft8(a);
    };

    load(0, 0);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    for (int it = 0; it <= nph; it++) {
        if (it + 1 < nph) load(it + 1, (it + 1) & 1);
        if (it < nph) {
            // row pass of phase it
            const unsigned char *V = vs + (size_t)(it & 1) * vstride;
            float2 *H = Hs + (size_t)(it & 1) * HB;
            const int ns = min(SP, n - SP * it);
#pragma unroll
            for (int r = 0; r < RR; r++) {
                int y, p0, si;
                const int w = g >> 2, yw = ((g & 2) ? 31 - w : w) + 32 * r;
                if (SP == 2) {
                    si = g & 1;
                    p0 = 0;
                    y = yw;
                } else if (P == 2) {
                    si = 0;
                    p0 = g & 1;
                    y = yw;
                } else {
                    si = 0;
                    p0 = 0;
                    y = (g & ~7) | ((g & 1) << 2) | ((g >> 1) & 3);
                }
                const bool live = y < box_h && si < ns;
                if (!__any_sync(0xffffffffu, live)) continue;             // warp-uniform
                float2 a[RP][8];
#pragma unroll
                for (int q = 0; q < RP; q++)
#pragma unroll
                    for (int m = 0; m < 8; m++) a[q][m] = make_float2(0.f, 0.f);
                if (live) {
                    const char2 *E = reinterpret_cast<const char2 *>(V + (size_t)si * vbytes) + (size_t)p0 * ne;
                    constexpr int MX = PX ? 4 : 8;
                    int cb[MX], ce[MX];                                   // the cells' entry ranges, loaded first
#pragma unroll
                    for (int m = 0; m < MX; m++) {
                        const int x = t + 8 * m;
                        cb[m] = ce[m] = 0;
                        if (x < box_w) {
                            cb[m] = cstart[y * box_w + x];
                            ce[m] = cstart[y * box_w + x + 1];
                        }
                    }
#pragma unroll
                    for (int m = 0; m < MX; m++) {
                        float2 acg[RP];
#pragma unroll
                        for (int q = 0; q < RP; q++) acg[q] = make_float2(0.f, 0.f);
                        for (int i = cb[m]; i < ce[m]; i++) {
                            int el;
                            float2 wv;                                    // conj(W~)
                            if (TS) {
                                const int4 d = ent_s[i];
                                el = d.x;
                                wv = make_float2(__int_as_float(d.y), __int_as_float(d.z));
                            } else {
                                el = __ldg(celem + i);
                                wv = __ldg(cw + i);
                            }
#pragma unroll
                            for (int q = 0; q < RP; q++) {
                                const char2 v = E[q * ne + el];
                                const float er = (float)v.x, ei = (float)v.y;
                                acg[q].x = fmaf(wv.x, er, fmaf(-wv.y, ei, acg[q].x));
                                acg[q].y = fmaf(wv.x, ei, fmaf(wv.y, er, acg[q].y));
                            }
                        }
#pragma unroll
                        for (int q = 0; q < RP; q++) a[q][m] = acg[q];
                    }
                }
#pragma unroll
                for (int q = 0; q < RP; q++) {
                    if (PX) dft8_first4(a[q]);
                    else hai_fft512::dft8(a[q]);
#pragma unroll
                    for (int k = 1; k < 8; k++) a[q][k] = hai_fft512::cmul(a[q][k], tw[k]);
                    finish(a[q]);
                }
                if (live) {
                    const int sw = 2 * (y & 7);
#pragma unroll
                    for (int q = 0; q < RP; q++) {
                        float2 *row = H + (size_t)si * SO + (size_t)(p0 + q) * PO + (size_t)y * 64;
#pragma unroll
                        for (int k2 = 0; k2 < 8; k2++) row[(t + 8 * k2 + sw) & 63] = a[q][k2];
                    }
                }
            }
        }
        if (it >= 1) {
            // column pass of phase it - 1, sample by sample
            const float2 *Hp = Hs + (size_t)((it - 1) & 1) * HB;
            const int ns = min(SP, n - SP * (it - 1));
            const int pos = (col + 2 * t) & 63;                           // row y = t + 8 m: y & 7 = t
#pragma unroll
            for (int si = 0; si < SP; si++) {
                if (si >= ns) break;                                      // CTA-uniform
                const int c = (int)((s0 + (long long)SP * (it - 1) + si) / T);
                if (c != cur_c) {
                    flush(cur_c, seg);
                    seg++;
                    cur_c = c;
                }
                const float2 *H = Hp + (size_t)si * SO;
                float2 f[P][8];
#pragma unroll
                for (int p = 0; p < P; p++) {
#pragma unroll
                    for (int m = 0; m < 8; m++) {
                        const int y = t + 8 * m;
                        f[p][m] = (m < (PY ? 4 : 8) && y < box_h) ? H[(size_t)p * PO + (size_t)y * 64 + pos]
                                                                  : make_float2(0.f, 0.f);
                    }
                    if (PY) dft8_first4(f[p]);
                    else hai_fft512::dft8(f[p]);
#pragma unroll
                    for (int k = 1; k < 8; k++) f[p][k] = hai_fft512::cmul(f[p][k], tw[k]);
                }
#pragma unroll
                for (int p = 0; p < P; p++) finish(f[p]);
#pragma unroll
                for (int k2 = 0; k2 < 8; k2++) {
                    const float2 fx = f[0][k2];
                    acc[k2][0] = fmaf(fx.x, fx.x, fmaf(fx.y, fx.y, acc[k2][0]));
                    if (P == 2) {
                        const float2 fy = f[P - 1][k2];
                        acc[k2][Q > 1 ? 1 : 0] = fmaf(fy.x, fy.x, fmaf(fy.y, fy.y, acc[k2][Q > 1 ? 1 : 0]));
                        acc[k2][Q > 2 ? 2 : 0] = fmaf(fx.x, fy.x, fmaf(fx.y, fy.y, acc[k2][Q > 2 ? 2 : 0]));
                        acc[k2][Q > 3 ? 3 : 0] = fmaf(fx.y, fy.x, fmaf(-fx.x, fy.y, acc[k2][Q > 3 ? 3 : 0]));
                    }
                }
            }
        }
        if (vec16) asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncthreads();
    }
    flush(cur_c, seg);
}

// img[c] = (accumulate ? img[c] : 0) + sum of the partials of channel c, in
// CTA order.  CTA b covers samples [b*len, (b+1)*len) of the flat index.
__global__ void epic_reduce_kernel(const float *__restrict__ part, float *__restrict__ img, int C,
                                   int T, long long len, int plane, int accumulate) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)C * plane) return;
    const int c = (int)(i / plane);
    const int off = (int)(i % plane);
    const int b0 = (int)(((long long)c * T) / len);
    const int b1 = (int)(((long long)(c + 1) * T - 1) / len);
    float s = 0.f;
    for (int b = b0; b <= b1; b++) {
        const int first = (int)(((long long)b * len) / T);
        const int sgm = c - first;
        s += part[((size_t)b * 2 + sgm) * plane + off];
    }
    img[i] = accumulate ? img[i] + s : s;
}

// The N = 64 kernel in the form the box and the shared memory allow:
// *launched = false if even the smallest form does not fit (the caller keeps
// the general kernel).
template <int P, bool PX, bool PY, int SP, bool TS>
void launch64_form(const int8_t *volt, int C, int T, int ne, const EpicSplit &sp, int box_w, int box_h,
                   const int32_t *cstart, const int32_t *celem, const float2 *cw, int nnz, float *dst,
                   int accumulate, size_t smem, cudaStream_t st) {
    const int vec16 = ((((uintptr_t)volt) & 15) == 0 && ((size_t)P * ne * 2) % 16 == 0) ? 1 : 0;
    epic64_kernel<P, PX, PY, SP, TS><<<sp.n_cta, k64Threads, smem, st>>>(
        volt, C, T, ne, sp.len, box_w, box_h, cstart, celem, cw, nnz, dst, sp.direct, accumulate, vec16);
}

template <int P, bool PX, bool PY, int SP, bool TS>
hai_status try64(const int8_t *volt, int C, int T, int ne, const EpicSplit &sp, int box_w, int box_h,
                 const int32_t *cstart, const int32_t *celem, const float2 *cw, int nnz, float *dst, int accumulate,
                 int smem_optin, cudaStream_t st, bool *launched) {
    const size_t smem = Epic64Smem<P, PX, PY, SP, TS>::bytes(ne, box_w * box_h, nnz);
    if (*launched || smem > (size_t)smem_optin) return HAI_OK;
    auto kern = epic64_kernel<P, PX, PY, SP, TS>;
    HAI_CUDA_TRY(hai_allow_dyn_smem(kern, smem_optin));
    launch64_form<P, PX, PY, SP, TS>(volt, C, T, ne, sp, box_w, box_h, cstart, celem, cw, nnz, dst, accumulate,
                                     smem, st);
    HAI_CUDA_TRY(cudaGetLastError());
    *launched = true;
    return HAI_OK;
}

// Forms in order of preference: two samples per phase (boxes of at most 32
// rows) with the table in shared memory, then without it; one sample with the
// table (taller boxes); one sample.  One pol: one sample, table in global
// memory.
template <int P, bool PX, bool PY>
hai_status launch64_box(const int8_t *volt, int C, int T, int ne, const EpicSplit &sp, int box_w, int box_h,
                        const int32_t *cstart, const int32_t *celem, const float2 *cw, int nnz, float *dst,
                        int accumulate, int smem_optin, cudaStream_t st, bool *launched) {
    *launched = false;
    if constexpr (P == 1) {       // one pol: the plain forms only
        return try64<P, PX, PY, 1, false>(volt, C, T, ne, sp, box_w, box_h, cstart, celem, cw, nnz, dst, accumulate,
                                          smem_optin, st, launched);
    } else {
#define HAI_TRY64(SPV, TSV)                                                                                    \
    {                                                                                                          \
        const hai_status s_ = try64<P, PX, PY, SPV, TSV>(volt, C, T, ne, sp, box_w, box_h, cstart, celem, cw,  \
                                                         nnz, dst, accumulate, smem_optin, st, launched);      \
        if (s_ != HAI_OK) return s_;                                                                           \
    }
        if constexpr (PY) {
            HAI_TRY64(2, true);
            HAI_TRY64(2, false);
        } else {
            HAI_TRY64(1, true);
        }
        HAI_TRY64(1, false);
#undef HAI_TRY64
        return HAI_OK;
    }
}

template <int P>
size_t epic64_bytes(int ne, int box_w, int box_h) {
    // the smallest form (one sample per phase, table in global memory)
    const bool px = box_w <= 32, py = box_h <= 32;
    if (px && py) return Epic64Smem<P, true, true, 1, false>::bytes(ne, 0, 0);
    if (px) return Epic64Smem<P, true, false, 1, false>::bytes(ne, 0, 0);
    if (py) return Epic64Smem<P, false, true, 1, false>::bytes(ne, 0, 0);
    return Epic64Smem<P, false, false, 1, false>::bytes(ne, 0, 0);
}

template <int P>
hai_status launch64(const int8_t *volt, int C, int T, int ne, const EpicSplit &sp, int box_w, int box_h,
                    const int32_t *cstart, const int32_t *celem, const float2 *cw, int nnz, float *dst,
                    int accumulate, int smem_optin, cudaStream_t st, bool *launched) {
    const bool px = box_w <= 32, py = box_h <= 32;
    if (px && py)
        return launch64_box<P, true, true>(volt, C, T, ne, sp, box_w, box_h, cstart, celem, cw, nnz, dst, accumulate,
                                           smem_optin, st, launched);
    if (px)
        return launch64_box<P, true, false>(volt, C, T, ne, sp, box_w, box_h, cstart, celem, cw, nnz, dst,
                                            accumulate, smem_optin, st, launched);
    if (py)
        return launch64_box<P, false, true>(volt, C, T, ne, sp, box_w, box_h, cstart, celem, cw, nnz, dst,
                                            accumulate, smem_optin, st, launched);
    return launch64_box<P, false, false>(volt, C, T, ne, sp, box_w, box_h, cstart, celem, cw, nnz, dst, accumulate,
                                         smem_optin, st, launched);
}

template <int N, int P>
hai_status launch_n(const hai_layout *L, const int8_t *volt, int C, int T, float *img, int accumulate,
                    cudaStream_t st) {
    if (N == 64) {
        const EpicSplit sp = epic_make_split(C, T, epic_fp32_target_ctas(L->ctx, N));
        if (!sp.direct && (size_t)sp.n_cta * 2 > L->partial_slots)
            return hai_fail(HAI_ERR_INVALID_ARG, "epic fp32: partial buffer too small");
        float *dst = sp.direct ? img : L->d_partials;
        bool launched = false;
        if (epic64_bytes<P>(L->n_elem, L->box_w, L->box_h) <= (size_t)L->ctx->smem_optin) {
            const int pidx = prof_begin(L->ctx, st);
            hai_status s = launch64<P>(volt, C, T, L->n_elem, sp, L->box_w, L->box_h, L->d_cell_start,
                                       L->d_entry_elem, L->d_entry_w, L->nnz, dst, accumulate, L->ctx->smem_optin,
                                       st, &launched);
            if (s != HAI_OK) return s;
            prof_end(L->ctx, pidx, st);
            prof_count(L->ctx, 1);
            if (!sp.direct) return epic_reduce_launch(L, sp, C, T, img, accumulate, st);
            return HAI_OK;
        }
    }
    const size_t smem = sizeof(float2) * EpicSmem<N, P>::kBuf +
                        ((size_t)kSamples * P * L->n_elem * 2 + 15) / 16 * 16;
    if (smem > (size_t)L->ctx->smem_optin)
        return hai_fail(HAI_ERR_UNSUPPORTED, "epic fp32: shared memory need exceeds the device limit");
    auto kern = epic_fp32_kernel<N, P>;
    HAI_CUDA_TRY(hai_allow_dyn_smem(kern, L->ctx->smem_optin));
    const EpicSplit sp = epic_make_split(C, T, epic_fp32_target_ctas(L->ctx, N));
    if (!sp.direct && (size_t)sp.n_cta * 2 > L->partial_slots)
        return hai_fail(HAI_ERR_INVALID_ARG, "epic fp32: partial buffer too small");
    float *dst = sp.direct ? img : L->d_partials;
    const int pidx = prof_begin(L->ctx, st);
    kern<<<sp.n_cta, kThreads, smem, st>>>(volt, C, T, L->n_elem, sp.len, L->box_w, L->box_h,
                                           L->d_cell_start, L->d_entry_elem, L->d_entry_w, dst,
                                           sp.direct, accumulate);
    prof_end(L->ctx, pidx, st);
    prof_count(L->ctx, 1);
    HAI_CUDA_TRY(cudaGetLastError());
    if (!sp.direct) return epic_reduce_launch(L, sp, C, T, img, accumulate, st);
    return HAI_OK;
}

}  // namespace

hai_status epic_fp32_init_tables(void) {
    float2 tw[kTwN / 2];
    for (int m = 0; m < kTwN / 2; m++) {
        const double ang = 2.0 * 3.14159265358979323846 * m / kTwN;
        tw[m] = make_float2((float)cos(ang), (float)sin(ang));
    }
    HAI_CUDA_TRY(cudaMemcpyToSymbol(c_tw, tw, sizeof(tw)));
    return HAI_OK;
}

int epic_fp32_target_ctas(const hai_ctx *ctx, int) { return ctx->num_sms; }

hai_status epic_reduce_launch(const hai_layout *L, const EpicSplit &sp, int C, int T, float *img,
                              int accumulate, cudaStream_t st) {
    const int Q = (L->n_pol == 2) ? 4 : 1;
    const int plane = Q * L->grid_n * L->grid_n;
    const long long n = (long long)C * plane;
    const int threads = 256;
    epic_reduce_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(
        L->d_partials, img, C, T, sp.len, plane, accumulate);
    prof_count(L->ctx, 1);
    HAI_CUDA_TRY(cudaGetLastError());
    return HAI_OK;
}

hai_status epic_fp32_launch(const hai_layout *L, const int8_t *volt, int C, int T, float *img,
                            int accumulate, cudaStream_t st) {
    const int n = L->grid_n, p = L->n_pol;
    if (n == 16) return p == 2 ? launch_n<16, 2>(L, volt, C, T, img, accumulate, st)
                               : launch_n<16, 1>(L, volt, C, T, img, accumulate, st);
    if (n == 32) return p == 2 ? launch_n<32, 2>(L, volt, C, T, img, accumulate, st)
                               : launch_n<32, 1>(L, volt, C, T, img, accumulate, st);
    if (n == 64) return p == 2 ? launch_n<64, 2>(L, volt, C, T, img, accumulate, st)
                               : launch_n<64, 1>(L, volt, C, T, img, accumulate, st);
    if (epic_large_supported(n)) return epic_large_launch(L, volt, C, T, img, accumulate, st);
    return hai_fail(HAI_ERR_UNSUPPORTED, "epic fp32: grid size");
}

// ============================================================================
// Allocation-free entry point.
//
// hai_layout_create reserves the gather table and the time-split partial
// images with cudaMalloc, so callers that must not allocate device memory
// cannot use hai_epic_image.  This entry point runs the same FP32 kernel with
// both kept in one fixed file-scope device array: the gather table is built
// on the host from the caller's layout description into a static host
// buffer and copied in on the caller's stream, and the partial images of the
// time split live after it.  Every call on a device shares the array (and
// the host buffer), which keeps the last call's contents; nothing in it has
// to start at zero, because each launch rewrites the table and every partial
// image slot it reads.  Calls that overlap on the GPU, or that come from two
// host threads at once, race on it.
// ============================================================================
namespace {

constexpr int kStaticMaxN = 64;                  // grid side
constexpr int kStaticMaxNnz = 102400;            // n_elem x K^2 gather entries
constexpr int kStaticMaxCells = kStaticMaxN * kStaticMaxN;
constexpr int kStaticCtas = 64;                  // CTAs of the time split
// cell starts | elements | (pad to 8 bytes) conj taps as float2, rounded to 16 bytes
constexpr size_t kStaticTableWords = ((size_t)(kStaticMaxCells + 1) + 3 * (size_t)kStaticMaxNnz + 1 + 3) & ~(size_t)3;
constexpr size_t kStaticPartialFloats = 2 * (size_t)kStaticCtas * 4 * kStaticMaxN * kStaticMaxN;
constexpr size_t kStaticFloats = kStaticTableWords + kStaticPartialFloats;   // 2,408,452 (9.2 MiB)
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) float g_epic_static_scratch[kStaticFloats];

// host side: device address of the array per device, and the host staging
// buffer of the gather table (cell starts | elements | conj taps)
static float *g_static_ptr[kStaticMaxDevices];
alignas(16) static int32_t g_static_host[kStaticTableWords];
static int32_t g_static_cursor[kStaticMaxCells];

// word offset of the float2 taps inside the table: 8-byte aligned
inline size_t static_taps_word(int ncell, int nnz) { return ((size_t)(ncell + 1) + nnz + 1) & ~(size_t)1; }

hai_status static_scratch(int device, float **out) {
    if (!g_static_ptr[device]) {
        // the host-side name of the array is only a stand-in: fetch the device
        // address once, with this device current; the FFT twiddles live in
        // constant memory that no context has filled yet on this path
        hai_status s = epic_fp32_init_tables();
        if (s != HAI_OK) return s;
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_epic_static_scratch);
        if (e != cudaSuccess) return hai_cuda_fail(e, "hai_epic_image_fp32_static: cudaGetSymbolAddress");
        g_static_ptr[device] = static_cast<float *>(p);
    }
    *out = g_static_ptr[device];
    return HAI_OK;
}

template <int N, int P>
hai_status launch_static(float *scratch, int ne, int box_w, int box_h, int ncell, int nnz, const int8_t *volt,
                         int C, int T, float *img, int accumulate, int sms, int smem_optin, cudaStream_t st) {
    const EpicSplit sp = epic_make_split(C, T, std::min(sms, kStaticCtas));
    const int32_t *cstart = reinterpret_cast<const int32_t *>(scratch);
    const int32_t *celem = cstart + (ncell + 1);
    const float2 *cw = reinterpret_cast<const float2 *>(cstart + static_taps_word(ncell, nnz));
    float *partials = scratch + kStaticTableWords;
    bool launched = false;
    if (N == 64) {
        hai_status s = launch64<P>(volt, C, T, ne, sp, box_w, box_h, cstart, celem, cw, nnz,
                                   sp.direct ? img : partials, accumulate, smem_optin, st, &launched);
        if (s != HAI_OK) return s;
    }
    if (!launched) {
        const size_t smem = sizeof(float2) * EpicSmem<N, P>::kBuf + ((size_t)kSamples * P * ne * 2 + 15) / 16 * 16;
        if (smem > (size_t)smem_optin)
            return hai_fail(HAI_ERR_UNSUPPORTED,
                            "hai_epic_image_fp32_static: shared memory need exceeds the device limit");
        auto kern = epic_fp32_kernel<N, P>;
        HAI_CUDA_TRY(hai_allow_dyn_smem(kern, smem_optin));
        kern<<<sp.n_cta, kThreads, smem, st>>>(volt, C, T, ne, sp.len, box_w, box_h, cstart, celem, cw,
                                               sp.direct ? img : partials, sp.direct, accumulate);
        HAI_CUDA_TRY(cudaGetLastError());
    }
    if (!sp.direct) {
        const int Q = (P == 2) ? 4 : 1;
        const int plane = Q * N * N;
        const long long n = (long long)C * plane;
        epic_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(partials, img, C, T, sp.len, plane,
                                                                          accumulate);
        HAI_CUDA_TRY(cudaGetLastError());
    }
    return HAI_OK;
}

}  // namespace

extern "C" hai_status hai_epic_image_fp32_static(int device, const hai_layout_desc *d, const int8_t *volt, int C,
                                                 int T, float *img, int accumulate, void *stream) {
    if (!d || !d->anchors || !d->taps) return hai_fail(HAI_ERR_INVALID_ARG, "hai_epic_image_fp32_static: NULL argument");
    if (device < 0 || device >= kStaticMaxDevices)
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_epic_image_fp32_static: device index out of range");
    if (d->n_elem <= 0 || d->ksize <= 0 || (d->n_pol != 1 && d->n_pol != 2) || C < 0 || T < 0 ||
        (accumulate != 0 && accumulate != 1))
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_epic_image_fp32_static: bad descriptor or size");
    const int n = d->grid_n, k = d->ksize, ne = d->n_elem;
    if (n != 16 && n != 32 && n != 64)
        return hai_fail(HAI_ERR_UNSUPPORTED, "hai_epic_image_fp32_static: grid_n must be 16, 32 or 64");
    if ((long long)ne * k * k > kStaticMaxNnz)
        return hai_fail(HAI_ERR_UNSUPPORTED, "hai_epic_image_fp32_static: n_elem * ksize^2 exceeds the static "
                                             "scratch maximum of 102400 gather entries");
    int bx0 = n, by0 = n, bx1 = 0, by1 = 0;
    for (int a = 0; a < ne; a++) {
        const int x0 = d->anchors[2 * a], y0 = d->anchors[2 * a + 1];
        if (x0 < 0 || y0 < 0 || (long)x0 + k > n || (long)y0 + k > n)
            return hai_fail(HAI_ERR_OFF_GRID, "hai_epic_image_fp32_static: a kernel tap lies outside the grid");
        bx0 = std::min(bx0, x0);
        by0 = std::min(by0, y0);
        bx1 = std::max(bx1, x0 + k);
        by1 = std::max(by1, y0 + k);
    }
    if (C == 0) return HAI_OK;
    if (!img || (T > 0 && !volt)) return hai_fail(HAI_ERR_INVALID_ARG, "hai_epic_image_fp32_static: NULL buffer");
    if ((((uintptr_t)volt) & 1) || (((uintptr_t)img) & 3))
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_epic_image_fp32_static: volt must be 2-byte and img 4-byte aligned");
    HAI_CUDA_TRY(cudaSetDevice(device));
    cudaStream_t st = (cudaStream_t)stream;
    const int Q = (d->n_pol == 2) ? 4 : 1;
    if (T == 0) {
        if (!accumulate) HAI_CUDA_TRY(cudaMemsetAsync(img, 0, sizeof(float) * (size_t)C * Q * n * n, st));
        return HAI_OK;
    }
    float *scratch = nullptr;
    hai_status s = static_scratch(device, &scratch);
    if (s != HAI_OK) return s;
    // gather table, same order as hai_layout_create: cells of the box row-major,
    // entries by element, weights conj(W~)
    const int box_w = bx1 - bx0, box_h = by1 - by0, ncell = box_w * box_h;
    const int nnz = ne * k * k;
    int32_t *cstart = g_static_host;
    int32_t *celem = cstart + (ncell + 1);
    float2 *cw = reinterpret_cast<float2 *>(cstart + static_taps_word(ncell, nnz));
    for (int i = 0; i <= ncell; i++) cstart[i] = 0;
    for (int a = 0; a < ne; a++)
        for (int v = 0; v < k; v++)
            for (int u = 0; u < k; u++) cstart[(d->anchors[2 * a + 1] + v - by0) * box_w + (d->anchors[2 * a] + u - bx0) + 1]++;
    for (int i = 0; i < ncell; i++) cstart[i + 1] += cstart[i];
    for (int i = 0; i < ncell; i++) g_static_cursor[i] = cstart[i];
    for (int a = 0; a < ne; a++)
        for (int v = 0; v < k; v++)
            for (int u = 0; u < k; u++) {
                const int cell = (d->anchors[2 * a + 1] + v - by0) * box_w + (d->anchors[2 * a] + u - bx0);
                const float *t = d->taps + (((size_t)a * k + v) * k + u) * 2;
                const int slot = g_static_cursor[cell]++;
                celem[slot] = a;
                cw[slot] = make_float2(t[0], -t[1]);
            }
    const size_t words = static_taps_word(ncell, nnz) + 2 * (size_t)nnz;
    HAI_CUDA_TRY(cudaMemcpyAsync(scratch, g_static_host, sizeof(int32_t) * words, cudaMemcpyHostToDevice, st));
    int sms = 0, optin = 0;
    HAI_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    HAI_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    const int p = d->n_pol;
#define HAI_STATIC_CASE(NN)                                                                                        \
    if (n == NN)                                                                                                   \
        return p == 2 ? launch_static<NN, 2>(scratch, ne, box_w, box_h, ncell, nnz, volt, C, T, img, accumulate, \
                                             sms, optin, st)                                                      \
                      : launch_static<NN, 1>(scratch, ne, box_w, box_h, ncell, nnz, volt, C, T, img, accumulate, \
                                             sms, optin, st);
    HAI_STATIC_CASE(16)
    HAI_STATIC_CASE(32)
    HAI_STATIC_CASE(64)
#undef HAI_STATIC_CASE
    return hai_fail(HAI_ERR_UNSUPPORTED, "hai_epic_image_fp32_static: grid size");
}
