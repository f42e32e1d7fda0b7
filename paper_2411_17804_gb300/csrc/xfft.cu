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
// K_ab and the cells it lands on depend on the layout only.  On a layout's
// first call the host lists, per grid cell, the (pair, K_ab value, mirror)
// entries that land there; the imaging is then three kernels per batch of
// channels:
//   transpose: the visibilities to [pair][channel][pol pair] (float2), so
//              that one pair's values for every channel and product are
//              adjacent;
//   gather:    per cell, threads over (channel, product) sum the cell's
//              entries (no atomics; four partial sums combined in a fixed
//              order: deterministic) and store the cell with the (-1)^(dx+dy)
//              checkerboard;
//   FFT:       one CTA per (channel, product) grid: rows then columns,
//              radix-2 in shared memory, into the image planes.
#include <math.h>

#include <algorithm>
#include <vector>

#include "hai_internal.h"

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// products: XX = V^00, YY = V^11, XY = V^01; the mirror (b, a) of a stored
// pair uses V^00, V^11, V^10 (conjugated)
__constant__ int kProd[3] = {0, 3, 1};
__constant__ int kMProd[3] = {0, 3, 2};

// vis [C][nbl][PP] int2 -> vt [nbl][cb][PP] float2 for channels c0 .. c0+cb-1
__global__ void __launch_bounds__(256) xfft_transpose_kernel(const int32_t *__restrict__ vis, long long nbl, int PP,
                                                             int c0, int cb, float2 *__restrict__ vt) {
    const long long n = nbl * cb * PP;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int pp = (int)(i % PP);
        const long long r = i / PP;
        const int c = (int)(r % cb);
        const long long bl = r / cb;
        const int2 v = reinterpret_cast<const int2 *>(vis)[((size_t)(c0 + c) * nbl + bl) * PP + pp];
        vt[i] = make_float2((float)v.x, (float)v.y);
    }
}

// One block per cell; thread j = (channel c, product q), j = c np + q.  The
// cell's entries are taken four at a time into four partial sums (their loads
// independent), combined in a fixed order: deterministic.  grid [cb][np][N][N].
__global__ void __launch_bounds__(256) xfft_gather_kernel(const float2 *__restrict__ vt, const int32_t *__restrict__ cell_start,
                                                          const int32_t *__restrict__ ent, const float2 *__restrict__ kab,
                                                          int N, int cb, int np, int PP, float2 *__restrict__ grid) {
    const int nj = cb * np, NN = N * N;
    const int cell = blockIdx.x;
    const int dx = cell % N, dy = cell / N;
    const float sgn = ((dx + dy) & 1) ? -1.f : 1.f;
    const int q0 = cell_start[cell], q1 = cell_start[cell + 1];
    for (int j = threadIdx.x; j < nj; j += blockDim.x) {
        const int c = j / np, q = j - c * np;
        const int pd = np == 1 ? 0 : kProd[q], pm = np == 1 ? 0 : kMProd[q];
        float2 acc[4];
#pragma unroll
        for (int u = 0; u < 4; u++) acc[u] = make_float2(0.f, 0.f);
        int e = q0;
        for (; e + 4 <= q1; e += 4) {
            int32_t en[4];
            float2 kv[4], v[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                en[u] = ent[e + u];
                kv[u] = kab[e + u];
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const long long bl = en[u] & 0x7fffffff;
                v[u] = vt[(bl * cb + c) * PP + (en[u] < 0 ? pm : pd)];
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const float2 t = cmul(v[u], kv[u]);
                acc[u].x += t.x;
                acc[u].y += en[u] < 0 ? -t.y : t.y;
            }
        }
        for (; e < q1; e++) {
            const int32_t en = ent[e];
            const long long bl = en & 0x7fffffff;
            const float2 t = cmul(vt[(bl * cb + c) * PP + (en < 0 ? pm : pd)], kab[e]);
            acc[0].x += t.x;
            acc[0].y += en < 0 ? -t.y : t.y;
        }
        const float sx = (acc[0].x + acc[1].x) + (acc[2].x + acc[3].x);
        const float sy = (acc[0].y + acc[1].y) + (acc[2].y + acc[3].y);
        grid[((size_t)c * np + q) * NN + cell] = make_float2(sgn * sx, sgn * sy);
    }
}

// In-place radix-2 FFT (exponent +) of n points in bit-reversed order at
// x[0], x[s], ... by one warp; tw[k] = exp(+2 pi i k / n), k < n / 2.
__device__ void warp_fft(float2 *x, int s, int n, int log2n, const float2 *tw, int lane) {
    for (int lh = 0; lh < log2n; lh++) {
        const int half = 1 << lh, tshift = log2n - 1 - lh;
        for (int b = lane; b < n / 2; b += 32) {
            const int pos = b & (half - 1);
            const int i0 = ((b - pos) << 1) + pos, i1 = i0 + half;
            const float2 a = x[i0 * s];
            const float2 t = cmul(x[i1 * s], tw[pos << tshift]);
            x[i0 * s] = make_float2(a.x + t.x, a.y + t.y);
            x[i1 * s] = make_float2(a.x - t.x, a.y - t.y);
        }
        __syncwarp();
    }
}

// One CTA per (channel c, product q) grid: the grid lands bit-reversed along
// both axes in a padded shared tile, rows then columns are transformed in
// place, and the product goes to its image plane(s): q = 0 -> XX (real part),
// 1 -> YY (real part), 2 -> Re XY, Im XY.
__global__ void __launch_bounds__(256) xfft_fft_kernel(const float2 *__restrict__ grid, int N, int log2n, int np, int Q,
                                                       int c0, float *__restrict__ img, int accumulate) {
    extern __shared__ float2 sm[];
    const int S = N + 1;                 // padded row stride
    float2 *tw = sm + (size_t)N * S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const int c = blockIdx.x / np, q = blockIdx.x % np;
    const float2 *g = grid + (size_t)blockIdx.x * N * N;
    for (int k = threadIdx.x; k < N / 2; k += blockDim.x) {
        float s, co;
        sincospif((float)(2 * k) / (float)N, &s, &co);
        tw[k] = make_float2(co, s);
    }
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
        const int x = i % N, y = i / N;
        sm[(__brev(y) >> (32 - log2n)) * S + (__brev(x) >> (32 - log2n))] = g[i];
    }
    __syncthreads();
    for (int r = warp; r < N; r += nwarp) warp_fft(sm + (size_t)r * S, 1, N, log2n, tw, lane);
    __syncthreads();
    for (int col = warp; col < N; col += nwarp) warp_fft(sm + col, S, N, log2n, tw, lane);
    __syncthreads();
    const size_t NN = (size_t)N * N;
    float *out = img + ((size_t)(c0 + c) * Q) * NN;
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
        const float2 v = sm[(i / N) * S + (i % N)];
        if (q < 2) {
            float *o = out + (size_t)q * NN + i;
            *o = accumulate ? *o + v.x : v.x;
        } else {
            float *o = out + 2 * NN + i, *oi = out + 3 * NN + i;
            *o = accumulate ? *o + v.x : v.x;
            *oi = accumulate ? *oi + v.y : v.y;
        }
    }
}

}  // namespace

// The layout's per-cell gridding list, built once on the host (FP32 K_ab,
// summed in the order of the lag loops below) and kept with the layout.
static hai_status ensure_table(const hai_layout *L) {
    std::lock_guard<std::mutex> lock(L->xfft_mu);
    if (L->d_xcell) return HAI_OK;
    const int N = L->grid_n, K = L->ksize, ne = L->n_elem;
    // at most 2 (2K-1)^2 entries per stored pair, 12 bytes each on the device
    const double max_ent = (double)ne * (ne + 1) / 2 * 2.0 * (2 * K - 1) * (2 * K - 1);
    if (max_ent > 2.0e8)
        return hai_fail(HAI_ERR_UNSUPPORTED, "hai_xfft_image: the layout's gridding list would exceed 2e8 entries");
    const float2 *taps = reinterpret_cast<const float2 *>(L->h_taps.data());   // [ne][K][K], as given
    const int32_t *anc = L->h_anchors.data();
    struct Ent {
        int32_t cell, e;
        float2 k;
    };
    std::vector<Ent> ents;
    for (int a = 0, bl = 0; a < ne; a++)
        for (int b = 0; b <= a; b++, bl++) {
            const int dx0 = anc[2 * a] - anc[2 * b], dy0 = anc[2 * a + 1] - anc[2 * b + 1];
            const float2 *ta = taps + (size_t)a * K * K, *tb = taps + (size_t)b * K * K;
            for (int ey = -(K - 1); ey <= K - 1; ey++)
                for (int ex = -(K - 1); ex <= K - 1; ex++) {
                    // K_ab[e] = sum over tap pairs with (ua - ub, va - vb) = e of conj(w_a) w_b
                    float2 k = make_float2(0.f, 0.f);
                    for (int vb = std::max(0, -ey); vb < std::min(K, K - ey); vb++)
                        for (int ub = std::max(0, -ex); ub < std::min(K, K - ex); ub++) {
                            const float2 wa = ta[(vb + ey) * K + (ub + ex)], wb = tb[vb * K + ub];
                            k.x += wa.x * wb.x + wa.y * wb.y;
                            k.y += wa.x * wb.y - wa.y * wb.x;
                        }
                    if (k.x == 0.f && k.y == 0.f) continue;
                    const int dx = (((dx0 + ex) % N) + N) % N, dy = (((dy0 + ey) % N) + N) % N;
                    ents.push_back({dy * N + dx, bl, k});
                    if (a != b) ents.push_back({((N - dy) % N) * N + (N - dx) % N, (int32_t)((uint32_t)bl | 0x80000000u), k});
                }
        }
    std::vector<int32_t> start((size_t)N * N + 1, 0), ent(std::max<size_t>(1, ents.size()));
    std::vector<float2> kv(std::max<size_t>(1, ents.size()));
    for (const Ent &x : ents) start[x.cell + 1]++;
    for (int c = 0; c < N * N; c++) start[c + 1] += start[c];
    {
        std::vector<int32_t> fill(start.begin(), start.end() - 1);
        for (const Ent &x : ents) {
            ent[fill[x.cell]] = x.e;
            kv[fill[x.cell]++] = x.k;
        }
    }
    int32_t *d_start = nullptr, *d_ent = nullptr;
    float2 *d_k = nullptr;
    cudaError_t e = cudaMalloc(&d_start, sizeof(int32_t) * start.size());
    if (e == cudaSuccess) e = cudaMalloc(&d_ent, sizeof(int32_t) * ent.size());
    if (e == cudaSuccess) e = cudaMalloc(&d_k, sizeof(float2) * kv.size());
    if (e == cudaSuccess) e = cudaMemcpy(d_start, start.data(), sizeof(int32_t) * start.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_ent, ent.data(), sizeof(int32_t) * ent.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_k, kv.data(), sizeof(float2) * kv.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d_start);
        cudaFree(d_ent);
        cudaFree(d_k);
        return hai_cuda_fail(e, "hai_xfft_image: gridding list");
    }
    L->d_xent = d_ent;
    L->d_xk = d_k;
    L->d_xcell = d_start;
    L->dev_bytes += sizeof(int32_t) * (start.size() + ent.size()) + sizeof(float2) * kv.size();
    return HAI_OK;
}

extern "C" hai_status hai_xfft_image(hai_ctx *ctx, const hai_layout *L, const int32_t *vis, int C, float *img,
                                     int accumulate, void *stream) {
    if (!ctx || !L) return hai_fail(HAI_ERR_INVALID_ARG, "hai_xfft_image: NULL ctx or layout");
    if (L->ctx != ctx) return hai_fail(HAI_ERR_INVALID_ARG, "hai_xfft_image: layout of another context");
    if (C < 0 || (accumulate != 0 && accumulate != 1))
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_xfft_image: bad channel count or flag");
    const int N = L->grid_n;
    if (N != 16 && N != 32 && N != 64) return hai_fail(HAI_ERR_UNSUPPORTED, "hai_xfft_image: grid size");
    if (C == 0) return HAI_OK;
    if (!vis || !img) return hai_fail(HAI_ERR_INVALID_ARG, "hai_xfft_image: NULL buffer");
    if (hai_fault_injected("launch")) return hai_fail(HAI_ERR_CUDA, "hai_xfft_image: injected launch failure");
    HAI_CUDA_TRY(cudaSetDevice(ctx->device));
    const hai_status ts = ensure_table(L);
    if (ts != HAI_OK) return ts;
    const hai_status ws = hai_workspace(ctx);
    if (ws != HAI_OK) return ws;
    cudaStream_t st = (cudaStream_t)stream;
    const int P = L->n_pol, PP = P * P, np = (P == 2) ? 3 : 1, Q = (P == 2) ? 4 : 1;
    int log2n = 0;
    while ((1 << log2n) < N) log2n++;
    const long long nbl = (long long)L->n_elem * (L->n_elem + 1) / 2;
    // channels per batch: transposed visibilities and grids in the context's workspace
    const size_t per_chan = sizeof(float2) * ((size_t)nbl * PP + (size_t)np * N * N);
    const int cmax = (int)std::min<size_t>({(size_t)C, ctx->corr_ws_bytes / per_chan, (size_t)(256 / np) * 256});
    if (cmax < 1) return hai_fail(HAI_ERR_UNSUPPORTED, "hai_xfft_image: one channel exceeds the workspace");
    float2 *vt = static_cast<float2 *>(ctx->d_corr_ws);
    const size_t smem = sizeof(float2) * ((size_t)N * (N + 1) + N / 2);
    const int pidx = prof_begin(ctx, st);
    for (int c0 = 0; c0 < C; c0 += cmax) {
        const int cb = std::min(cmax, C - c0);
        float2 *grid = vt + (size_t)nbl * cb * PP;
        const long long n = nbl * cb * PP;
        xfft_transpose_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, 64LL * ctx->num_sms), 256, 0, st>>>(
            vis, nbl, PP, c0, cb, vt);
        xfft_gather_kernel<<<N * N, 256, 0, st>>>(vt, L->d_xcell, L->d_xent, L->d_xk, N, cb, np, PP, grid);
        xfft_fft_kernel<<<cb * np, 256, smem, st>>>(grid, N, log2n, np, Q, c0, img, accumulate);
        prof_count(ctx, 3);
    }
    prof_end(ctx, pidx, st);
    HAI_CUDA_TRY(cudaGetLastError());
    return HAI_OK;
}
