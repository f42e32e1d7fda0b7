// Inter-station correlator beamforming (XBF, Eq. inter-station XBF) on tcgen05
// tensor cores.
//
// For beam k, channel c and polarisation pair (a, b) the image at the pixels
// sigma = s_k + (l - N/2) lambda / (N cell) is the direct sum over ordered
// station pairs (m, n), autos once, of V^{ab}_{mn} exp(+2 pi i sigma .
// (r_m - r_n) / lambda).  Pairing (m, n) with its mirror (n, m):
//   I[l] = sum over stored pairs m >= n of  P Phi[l] + Q conj(Phi[l]),
//   Phi[l] = exp(+2 pi i (l - N/2) . (r_m - r_n) / (N cell))   (geometry only)
//   P = V^{ab}_{mn} e,  Q = conj(V^{ba}_{mn} e),  e = exp(+2 pi i s_k . (r_m - r_n) / lambda)
// and for an auto P = V^{ab}_{mm}, Q = 0.  As real products
//   Re I = sum (P_r + Q_r) Phi_r + (Q_i - P_i) Phi_i
//   Im I = sum (P_i + Q_i) Phi_r + (P_r - Q_r) Phi_i
// so each image plane (XX, YY, Re XY, Im XY) is one row of a coefficient
// matrix A [rows][2B] and a whole cadence is one GEMM
//   img[rows][pixels] = A [rows][2B] x Phi^T [2B][pixels].
// Phi is built once per layout on the GPU (FP64 phase reduced to a fraction
// of a turn, then sincospi, stored fp16) and kept in HBM in the tensor cores'
// tile order, so each k-block of a tile is one contiguous bulk copy; A is
// rebuilt per call from the int32 visibilities with a power-of-two scale per
// image that keeps the fp16 values in range (undone in the epilogue).
//
// HAI_PREC_FP16_SPLIT: every value is split into an fp16 hi part and the fp16
// rounding remainder lo, and the K dimension is laid out three times,
// A' = [A_hi | A_hi | A_lo] against Phi' = [Phi_hi | Phi_lo | Phi_hi], so the
// same GEMM sums hi*hi + hi*lo + lo*hi (FP32-level accuracy, 3x the work).
//
// GEMM: one CTA per 128 x 256 output tile; a 4-stage pipeline of 48 KB bulk
// copies (A 128 x 64 and Phi 256 x 64, fp16); warp 0 streams, warp 1 issues
// tcgen05.mma (M = 128, N = 256, K = 16) into a 256-column TMEM accumulator,
// warps 4-7 write the tile.  Row blocks are the fastest grid index, so the
// CTAs running together share one Phi block, read from HBM once and served
// to the row blocks from L2.
#include <math.h>

#include <algorithm>
#include <vector>

#include "hai_internal.h"
#include "tc.cuh"

namespace {

constexpr int kTM = 128, kTN = 256, kTK = 64;
constexpr int kStages = 4;
constexpr uint32_t kABytes = kTM * kTK * 2;          // 16 KB
constexpr uint32_t kBBytes = kTN * kTK * 2;          // 32 KB
constexpr uint32_t kLBO = 128, kSBO = 1024;          // K-major: K-group and MN-group strides
constexpr uint32_t kIdesc = tc::idesc_f16(kTM, kTN, 0, 0);
constexpr int kThreads = 256;
constexpr size_t kSmem = (size_t)kStages * (kABytes + kBBytes);

__host__ __device__ __forceinline__ uint32_t tile_off(int row, int k) { return tc::off_kmajor(row, k, kLBO, kSBO); }

// Phi[pixel][(b, re/im)], 16 bytes (4 pairs) per thread
// split: K segments [Phi_hi | Phi_lo | Phi_hi] against [A_hi | A_hi | A_lo]
__global__ void xbf_phi_kernel(const double2 *__restrict__ duv, int B, int N, int log2n, int n_kblk, int split,
                               uint8_t *__restrict__ phi) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int groups = n_kblk * (kTK / 8);
    if (i >= (long long)N * N * groups) return;
    const int g = (int)(i % groups);
    const int p = (int)(i / groups);
    const double ox = (double)((p & (N - 1)) - N / 2), oy = (double)((p >> log2n) - N / 2);
    uint32_t h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int b = 4 * g + j;
        float c = 0.f, s = 0.f;
        if (b < B) {
            const double2 d = duv[b];
            const double t = (ox * d.x + oy * d.y) / (double)N;      // turns, FP64
            const float f = (float)(t - rint(t));                    // |f| <= 1/2
            sincospif(2.0f * f, &s, &c);
        }
        h[j] = tc::pack_half2(c, s);
        const float2 back = __half22float2(*reinterpret_cast<const __half2 *>(&h[j]));
        l[j] = tc::pack_half2(c - back.x, s - back.y);
    }
    const int nb = p / kTN, r = p % kTN, kb = g / (kTK / 8), kk = (g % (kTK / 8)) * 8;
    const int ktot = split ? 3 * n_kblk : n_kblk;
    uint8_t *base = phi + (size_t)nb * ktot * kBBytes + tile_off(r, kk);
    *reinterpret_cast<uint4 *>(base + (size_t)kb * kBBytes) = make_uint4(h[0], h[1], h[2], h[3]);
    if (split) {
        *reinterpret_cast<uint4 *>(base + (size_t)(n_kblk + kb) * kBBytes) = make_uint4(l[0], l[1], l[2], l[3]);
        *reinterpret_cast<uint4 *>(base + (size_t)(2 * n_kblk + kb) * kBBytes) = make_uint4(h[0], h[1], h[2], h[3]);
    }
}

// steering phasor e = exp(+2 pi i s_k . dr / lambda) per (beam, pair), FP64 phase
__global__ void xbf_steer_kernel(const double2 *__restrict__ dr, const double *__restrict__ dir, int K, int B,
                                 double inv_lambda, float2 *__restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)K * B) return;
    const int k = (int)(i / B), b = (int)(i % B);
    const double2 d = dr[b];
    const double turns = (dir[2 * k] * d.x + dir[2 * k + 1] * d.y) * inv_lambda;
    double s, c;
    sincospi(2.0 * (turns - rint(turns)), &s, &c);
    out[i] = make_float2((float)c, (float)s);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// the 8 coefficients (4 rows x (Phi_r, Phi_i)) of pair b of image img
__device__ __forceinline__ void pair_coefs(const int2 *__restrict__ v, int2 mn, float2 e, float (&o)[8]) {
    const long long bl = (long long)mn.x * (mn.x + 1) / 2 + mn.y;
    float2 V[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int2 x = v[bl * 4 + q];
        V[q] = make_float2((float)x.x, (float)x.y);
    }
    const bool autos = mn.x == mn.y;
    // P_ab, Q_ab for (a, b) = (0, 0), (1, 1), (0, 1)
    const int ab[3] = {0, 3, 1}, ba[3] = {0, 3, 2};
#pragma unroll
    for (int j = 0; j < 3; j++) {
        float2 P, Q;
        if (autos) {
            P = V[ab[j]];
            Q = make_float2(0.f, 0.f);
        } else {
            P = cmul(V[ab[j]], e);
            const float2 t = cmul(V[ba[j]], e);
            Q = make_float2(t.x, -t.y);
        }
        o[2 * j] = P.x + Q.x;                  // Re row: Phi_r coefficient
        o[2 * j + 1] = Q.y - P.y;              //         Phi_i coefficient
        if (j == 2) {
            o[6] = P.y + Q.y;                  // Im XY row
            o[7] = P.x - Q.x;
        }
    }
}

// one CTA per image (beam, channel): its 4 coefficient rows into the tiled A,
// scaled by 2^-e with e the smallest exponent that keeps every |value| <= 2^15
__global__ void __launch_bounds__(256) xbf_coef_kernel(const int32_t *__restrict__ vis, long long nbl,
                                                       const int2 *__restrict__ pairs,
                                                       const float2 *__restrict__ steer, int B, int C, int n_kblk,
                                                       int split, uint8_t *__restrict__ A,
                                                       float *__restrict__ scale) {
    __shared__ float red[8];
    const int img = blockIdx.x, k = img / C;
    const int2 *v = reinterpret_cast<const int2 *>(vis) + (size_t)img * nbl * 4;
    float mx = 0.f;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        float o[8];
        pair_coefs(v, pairs[b], steer[(size_t)k * B + b], o);
#pragma unroll
        for (int j = 0; j < 8; j++) mx = fmaxf(mx, fabsf(o[j]));
    }
    for (int off = 16; off; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) mx = fmaxf(mx, red[w]);
    int ex = 0;
    if (mx > 0.f) {
        frexpf(mx, &ex);                        // mx < 2^ex
        ex = max(0, ex - 15);
    }
    if (threadIdx.x == 0) scale[img] = ldexpf(1.0f, ex);
    const float sc = ldexpf(1.0f, -ex);
    const int row0 = img * 4;
    for (int b = threadIdx.x; b < n_kblk * (kTK / 2); b += blockDim.x) {
        float o[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (b < B) pair_coefs(v, pairs[b], steer[(size_t)k * B + b], o);
        const int kb = b / (kTK / 2), kk = 2 * (b % (kTK / 2));
        const int ktot = split ? 3 * n_kblk : n_kblk;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int r = row0 + j;
            uint8_t *dst = A + ((size_t)(r / kTM) * ktot + kb) * kABytes + tile_off(r % kTM, kk);
            const float x0 = o[2 * j] * sc, x1 = o[2 * j + 1] * sc;
            const uint32_t hi = tc::pack_half2(x0, x1);
            *reinterpret_cast<uint32_t *>(dst) = hi;
            if (split) {                        // segments [A_hi | A_hi | A_lo]
                const float2 back = __half22float2(*reinterpret_cast<const __half2 *>(&hi));
                *reinterpret_cast<uint32_t *>(dst + (size_t)n_kblk * kABytes) = hi;
                *reinterpret_cast<uint32_t *>(dst + (size_t)2 * n_kblk * kABytes) =
                    tc::pack_half2(x0 - back.x, x1 - back.y);
            }
        }
    }
}

struct GemmParams {
    const uint8_t *A, *phi;
    const float *scale;
    float *img;
    int n_kblk, M, npix, accumulate;
    unsigned *status;
};

__global__ void __launch_bounds__(kThreads, 1) xbf_gemm_kernel(const GemmParams p) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], accf;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mb = blockIdx.x, nb = blockIdx.y;
    if (tid == 0) {
        for (int s = 0; s < kStages; s++) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(&accf, 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc(&tslot, kTN);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tslot;
    auto sA = [&](int s) { return smem + (size_t)s * (kABytes + kBBytes); };
    auto sB = [&](int s) { return smem + (size_t)s * (kABytes + kBBytes) + kABytes; };
    const uint8_t *ablk = p.A + (size_t)mb * p.n_kblk * kABytes;
    const uint8_t *bblk = p.phi + (size_t)nb * p.n_kblk * kBBytes;
    if (warp == 0) {
        if (lane == 0)
            for (int kb = 0; kb < p.n_kblk; kb++) {
                const int s = kb % kStages;
                if (kb >= kStages) tc::mbar_wait(&empty[s], (uint32_t)(((kb / kStages) - 1) & 1), p.status);
                tc::mbar_arrive_expect_tx(&full[s], kABytes + kBBytes);
                tc::bulk_g2s(sA(s), ablk + (size_t)kb * kABytes, kABytes, &full[s]);
                tc::bulk_g2s(sB(s), bblk + (size_t)kb * kBBytes, kBBytes, &full[s]);
            }
    } else if (warp == 1) {
        if (lane == 0) {
            for (int kb = 0; kb < p.n_kblk; kb++) {
                const int s = kb % kStages;
                tc::mbar_wait(&full[s], (uint32_t)((kb / kStages) & 1), p.status);
                tc::fence_after();
                const uint32_t a = tc::smem_u32(sA(s)), b = tc::smem_u32(sB(s));
#pragma unroll
                for (int j = 0; j < kTK / 16; j++)
                    tc::mma_f16(tmem, tc::desc(a + j * 2 * kLBO, kLBO, kSBO), tc::desc(b + j * 2 * kLBO, kLBO, kSBO),
                                kIdesc, (kb > 0 || j > 0) ? 1u : 0u);
                tc::mma_commit(&empty[s]);
            }
            tc::mma_commit(&accf);
        }
    } else if (warp >= 4) {
        tc::mbar_wait(&accf, 0u, p.status);
        tc::fence_after();
        const int q = warp & 3;
        const int row = mb * kTM + q * 32 + lane;
        const float sc = row < p.M ? p.scale[row / 4] : 0.f;
#pragma unroll 1
        for (int ch = 0; ch < kTN / 32; ch++) {
            uint32_t r[32];
            tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ch * 32), r);
            tc::tmem_wait_ld();
            if (row < p.M) {
                float4 *dst = reinterpret_cast<float4 *>(p.img + (size_t)row * p.npix + (size_t)nb * kTN + ch * 32);
#pragma unroll
                for (int v = 0; v < 8; v++) {
                    float4 o = make_float4(__uint_as_float(r[4 * v]) * sc, __uint_as_float(r[4 * v + 1]) * sc,
                                           __uint_as_float(r[4 * v + 2]) * sc, __uint_as_float(r[4 * v + 3]) * sc);
                    if (p.accumulate) {
                        const float4 old = dst[v];
                        o.x += old.x;
                        o.y += old.y;
                        o.z += old.z;
                        o.w += old.w;
                    }
                    dst[v] = o;
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, kTN);
}

}  // namespace

struct hai_xbf_layout {
    hai_ctx *ctx = nullptr;
    int S = 0, N = 0, K = 0, pair_set = 0, max_images = 0, n_kblk = 0, n_mblk = 0, split = 0;
    long long B = 0, nbl = 0;
    int2 *d_pairs = nullptr;
    float2 *d_steer = nullptr;
    uint8_t *d_phi = nullptr;
    size_t phi_bytes = 0;
    uint8_t *d_coef = nullptr;
    size_t coef_bytes = 0;
    float *d_scale = nullptr;
};

static void xbf_free(hai_xbf_layout *L) {
    if (!L) return;
    cudaFree(L->d_pairs);
    cudaFree(L->d_steer);
    cudaFree(L->d_phi);
    cudaFree(L->d_coef);
    cudaFree(L->d_scale);
    delete L;
}

extern "C" hai_status hai_xbf_layout_create(hai_ctx *ctx, const hai_vis_layout_desc *d, int pair_set,
                                            int max_channels, hai_precision prec, hai_xbf_layout **out) {
    if (!ctx || !d || !out) return hai_fail(HAI_ERR_INVALID_ARG, "hai_xbf_layout_create: NULL argument");
    *out = nullptr;
    const int S = d->n_station, N = d->grid_n, K = d->n_dir;
    if (S <= 0 || !d->pos_m || !(d->lambda_m > 0) || !(d->cell_m > 0) || K <= 0 || N < 16 || N > 512 ||
        (N & (N - 1)) || (pair_set != 0 && pair_set != 1) || max_channels <= 0)
        return hai_fail(HAI_ERR_INVALID_ARG,
                        "hai_xbf_layout_create: bad descriptor (grid_n a power of two in 16..512), pair set or "
                        "channel count");
    if (d->n_pol != 2) return hai_fail(HAI_ERR_UNSUPPORTED, "hai_xbf_layout_create: station images need 2 pols");
    if (prec != HAI_PREC_FP16 && prec != HAI_PREC_FP16_SPLIT)
        return hai_fail(HAI_ERR_UNSUPPORTED, "hai_xbf_layout_create: precision must be FP16 or FP16_SPLIT");
    if ((long long)K * max_channels * 4 > (1ll << 30))
        return hai_fail(HAI_ERR_UNSUPPORTED, "hai_xbf_layout_create: too many images");
    if (hai_fault_injected("alloc")) return hai_fail(HAI_ERR_NO_MEMORY, "hai_xbf_layout_create: injected allocation failure");
    // the pair set, FP64 geometry on the host
    std::vector<int2> pairs;
    std::vector<double2> duv, dr;
    for (int m = 0; m < S; m++)
        for (int n = 0; n <= m; n++) {
            const double dx = d->pos_m[2 * m] - d->pos_m[2 * n], dy = d->pos_m[2 * m + 1] - d->pos_m[2 * n + 1];
            if (pair_set == 1 && (m == n || station_pair_kept(N, dx / d->cell_m, dy / d->cell_m))) continue;
            pairs.push_back(make_int2(m, n));
            duv.push_back(make_double2(dx / d->cell_m, dy / d->cell_m));
            dr.push_back(make_double2(dx, dy));
        }
    hai_xbf_layout *L = new hai_xbf_layout();
    L->ctx = ctx;
    L->S = S;
    L->N = N;
    L->K = K;
    L->pair_set = pair_set;
    L->max_images = K * max_channels;
    L->nbl = (long long)S * (S + 1) / 2;
    L->B = (long long)pairs.size();
    L->n_kblk = (int)((2 * L->B + kTK - 1) / kTK);
    L->n_mblk = (L->max_images * 4 + kTM - 1) / kTM;
    L->split = prec == HAI_PREC_FP16_SPLIT ? 1 : 0;
    const int nseg = L->split ? 3 : 1;
    const size_t npix = (size_t)N * N;
    L->phi_bytes = (size_t)nseg * L->n_kblk * kBBytes * (npix / kTN);
    L->coef_bytes = (size_t)nseg * L->n_kblk * kABytes * L->n_mblk;
    cudaError_t e = cudaSetDevice(ctx->device);
    double2 *d_duv = nullptr, *d_dr = nullptr;
    double *d_dir = nullptr;
    auto fail = [&](cudaError_t err) {
        cudaFree(d_duv);
        cudaFree(d_dr);
        cudaFree(d_dir);
        xbf_free(L);
        if (err == cudaErrorMemoryAllocation) return hai_cuda_fail(err, "hai_xbf_layout_create: allocation");
        return hai_cuda_fail(err, "hai_xbf_layout_create");
    };
    if (e != cudaSuccess) return fail(e);
    if (L->B > 0) {
        if ((e = cudaMalloc(&L->d_pairs, sizeof(int2) * L->B)) != cudaSuccess) return fail(e);
        if ((e = cudaMalloc(&L->d_steer, sizeof(float2) * L->B * K)) != cudaSuccess) return fail(e);
        if ((e = cudaMalloc(&L->d_phi, L->phi_bytes)) != cudaSuccess) return fail(e);
        if ((e = cudaMalloc(&L->d_coef, L->coef_bytes)) != cudaSuccess) return fail(e);
        if ((e = cudaMalloc(&d_duv, sizeof(double2) * L->B)) != cudaSuccess) return fail(e);
        if ((e = cudaMalloc(&d_dr, sizeof(double2) * L->B)) != cudaSuccess) return fail(e);
        if ((e = cudaMalloc(&d_dir, sizeof(double) * 2 * K)) != cudaSuccess) return fail(e);
        std::vector<double> dir(2 * (size_t)K, 0.0);
        if (d->dir) std::copy(d->dir, d->dir + 2 * (size_t)K, dir.begin());
        if ((e = cudaMemcpy(L->d_pairs, pairs.data(), sizeof(int2) * L->B, cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(e);
        if ((e = cudaMemcpy(d_duv, duv.data(), sizeof(double2) * L->B, cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(e);
        if ((e = cudaMemcpy(d_dr, dr.data(), sizeof(double2) * L->B, cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(e);
        if ((e = cudaMemcpy(d_dir, dir.data(), sizeof(double) * 2 * K, cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(e);
        if ((e = cudaMemset(L->d_coef, 0, L->coef_bytes)) != cudaSuccess) return fail(e);
        int log2n = 0;
        while ((1 << log2n) < N) log2n++;
        const long long nthr = (long long)npix * L->n_kblk * (kTK / 8);
        xbf_phi_kernel<<<(unsigned)((nthr + 255) / 256), 256>>>(d_duv, (int)L->B, N, log2n, L->n_kblk, L->split,
                                                              L->d_phi);
        const long long ns = (long long)K * L->B;
        xbf_steer_kernel<<<(unsigned)((ns + 255) / 256), 256>>>(d_dr, d_dir, K, (int)L->B, 1.0 / d->lambda_m,
                                                              L->d_steer);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e);
    }
    if ((e = cudaMalloc(&L->d_scale, sizeof(float) * L->max_images)) != cudaSuccess) return fail(e);
    cudaFree(d_duv);
    cudaFree(d_dr);
    cudaFree(d_dir);
    *out = L;
    return HAI_OK;
}

extern "C" void hai_xbf_layout_destroy(hai_xbf_layout *L) { xbf_free(L); }

extern "C" hai_status hai_xbf_layout_info(const hai_xbf_layout *L, long long *n_pairs, long long *device_bytes) {
    if (!L) return hai_fail(HAI_ERR_INVALID_ARG, "hai_xbf_layout_info: NULL layout");
    if (n_pairs) *n_pairs = L->B;
    if (device_bytes) *device_bytes = (long long)(L->phi_bytes + L->coef_bytes);
    return HAI_OK;
}

extern "C" hai_status hai_xbf_station_image(hai_ctx *ctx, const hai_xbf_layout *L, const int32_t *vis, int C,
                                            float *img, int accumulate, void *stream) {
    if (!ctx || !L) return hai_fail(HAI_ERR_INVALID_ARG, "hai_xbf_station_image: NULL ctx or layout");
    if (L->ctx != ctx) return hai_fail(HAI_ERR_INVALID_ARG, "hai_xbf_station_image: layout of another context");
    if (C < 0 || (long long)C * L->K > L->max_images || (accumulate != 0 && accumulate != 1))
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_xbf_station_image: channel count above the layout's maximum");
    if (C == 0) return HAI_OK;
    if (!vis || !img) return hai_fail(HAI_ERR_INVALID_ARG, "hai_xbf_station_image: NULL buffer");
    if (reinterpret_cast<uintptr_t>(img) & 15)
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_xbf_station_image: img must be 16-byte aligned");
    if (hai_fault_injected("launch")) return hai_fail(HAI_ERR_CUDA, "hai_xbf_station_image: injected launch failure");
    HAI_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int n_img = C * L->K, M = n_img * 4;
    const size_t npix = (size_t)L->N * L->N;
    if (L->B == 0) {                          // no pair in the set: the images are zero
        if (!accumulate) HAI_CUDA_TRY(cudaMemsetAsync(img, 0, sizeof(float) * M * npix, st));
        return HAI_OK;
    }
    HAI_CUDA_TRY(cudaFuncSetAttribute(xbf_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
    xbf_coef_kernel<<<n_img, 256, 0, st>>>(vis, L->nbl, L->d_pairs, L->d_steer, (int)L->B, C, L->n_kblk, L->split,
                                           L->d_coef, L->d_scale);
    GemmParams gp;
    gp.A = L->d_coef;
    gp.phi = L->d_phi;
    gp.scale = L->d_scale;
    gp.img = img;
    gp.n_kblk = (L->split ? 3 : 1) * L->n_kblk;
    gp.M = M;
    gp.npix = (int)npix;
    gp.accumulate = accumulate;
    gp.status = ctx->d_status;
    const int pidx = prof_begin(ctx, st);
    xbf_gemm_kernel<<<dim3((M + kTM - 1) / kTM, (unsigned)(npix / kTN)), kThreads, kSmem, st>>>(gp);
    prof_end(ctx, pidx, st);
    prof_count(ctx, 2);
    HAI_CUDA_TRY(cudaGetLastError());
    return HAI_OK;
}
