// Inter-station stage of the hierarchical array (Section 6, Eq. inter-station
// visibilities and Eq. inter-station XFFT).
//
// hai_beams_to_corr: station beams [S][C][T][K][P][2] int8 (the beamformer's
// output) -> correlator input [K][C][T][P][S][2] int8, so that hai_correlate
// with the (beam, channel) pairs as channels and the stations as elements
// gives V_mn(s_k) = sum_t E_m(s_k) conj(E_n(s_k)).
//
// hai_xfft_station_image: dirty images of those visibilities.  Every ordered
// station pair (m, n), autos included, is phased towards the beam direction,
// V~ = V exp(+2 pi i s_k.(r_m - r_n) / lambda), and gridded with a 2x2
// bilinear kernel at uv = (r_m - r_n) / cell; pairs whose 2x2 footprint (or
// its mirror's) leaves [-N/2, N/2 - 1]^2 are dropped and counted.  The steering
// phasors are computed once per (beam, pair) by an FP64 kernel at layout
// creation: the phase reaches ~10^5 rad on 65 km baselines, where FP32 would
// lose ~10^-2 rad; the FP64 phase is reduced to a fraction of a turn before
// sincospi and the phasor is stored in FP32.
//
// Both XX and YY grids are Hermitian (the mirror of a pair carries the
// conjugate), so their images are real and one complex FFT of G_XX + i G_YY
// gives XX in the real and YY in the imaginary part; XY needs its own complex
// grid.  The two complex grids are built in the caller's image planes
// [XX, YY, Re XY, Im XY] (as split re / im planes), which the FFT then
// transforms in place: no scratch memory.  Gridding runs in shared memory over
// tiles (<= 112 x 112 cells) of the window of uv cells that on-grid pairs
// touch, one CTA per (image, grid, tile) with the pairs binned to each tile on
// the host, and writes its cells with the (-1)^(u+v) checkerboard that puts
// the phase centre at pixel (N/2, N/2).  The FFTs read their twiddles from
// a shared-memory table.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "hai_internal.h"

namespace {

constexpr int kThreads = 512;
constexpr int kTileCells = 112;        // uv tile side: 2 x 112^2 floats = 98 KB of shared memory
constexpr int kTileSmall = 56;         // the smaller side, for layouts with many pairs per tile
constexpr size_t kTilePairsMin = 4096; // pairs per tile (average) that the smaller side needs

// Gridding record of one stored pair (m >= n): the 2x2 footprints of the pair
// and of its mirror, as window-relative cell of the lower corner and
// fractional offsets; du < 0 marks a dropped pair.
struct PairRec {
    int16_t du, dv, mu, mv;
    float fu, fv, mfu, mfv;
};

__device__ __forceinline__ void pair_of(long long bl, int &m, int &n) {
    int a = (int)((sqrt(8.0 * (double)bl + 1.0) - 1.0) * 0.5);
    while ((long long)(a + 1) * (a + 2) / 2 <= bl) a++;
    while ((long long)a * (a + 1) / 2 > bl) a--;
    m = a;
    n = (int)(bl - (long long)a * (a + 1) / 2);
}

// exp(+2 pi i s_k.(r_m - r_n) / lambda) for every (beam, stored pair), FP64.
__global__ void steering_kernel(const double *__restrict__ pos, const double *__restrict__ dir, int K,
                                long long nbl, double inv_lambda, float2 *__restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)K * nbl) return;
    const int k = (int)(i / nbl);
    const long long bl = i - (long long)k * nbl;
    int m, n;
    pair_of(bl, m, n);
    const double turns = (dir[2 * k] * (pos[2 * m] - pos[2 * n]) + dir[2 * k + 1] * (pos[2 * m + 1] - pos[2 * n + 1])) *
                         inv_lambda;
    const double frac = turns - rint(turns);          // |frac| <= 1/2: exact reduction in FP64
    double s, c;
    sincospi(2.0 * frac, &s, &c);
    out[i] = make_float2((float)c, (float)s);
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Adds the 2x2 footprint with lower corner (du, dv) (window cells) to the
// cells that fall inside this CTA's tile [tu0, tu0 + tw) x [tv0, tv0 + th)
// (tw, th: the tile's own extent; shared rows are tw apart).
__device__ __forceinline__ void add_footprint(float *wre, float *wim, int tu0, int tv0, int tw, int th, int du, int dv,
                                              float fu, float fv, float2 g) {
    const float w[4] = {(1.f - fu) * (1.f - fv), fu * (1.f - fv), (1.f - fu) * fv, fu * fv};
#pragma unroll
    for (int t = 0; t < 4; t++) {
        const int cu = du + (t & 1) - tu0, cv = dv + (t >> 1) - tv0;
        if (w[t] == 0.f || cu < 0 || cu >= tw || cv < 0 || cv >= th) continue;
        atomicAdd(&wre[cv * tw + cu], w[t] * g.x);
        atomicAdd(&wim[cv * tw + cu], w[t] * g.y);
    }
}

// One CTA per (image = (beam, channel), grid h, tile of the uv window):
// h = 0 builds G_XX + i G_YY into planes 0 / 1, h = 1 builds G_XY into
// planes 2 / 3.  The CTA grids the pairs binned to its tile, then writes its
// tile's cells with the checkerboard (the rest of the planes was zeroed).
__global__ void __launch_bounds__(kThreads) station_grid_kernel(
    const int32_t *__restrict__ vis, const PairRec *__restrict__ rec, const float2 *__restrict__ phasor,
    const int32_t *__restrict__ tile_start, const int32_t *__restrict__ tile_pairs, int C, long long nbl, int P,
    int N, int win_u0, int win_v0, int ww, int wh, int tw, int th, int ntx, float *__restrict__ img) {
    extern __shared__ float win[];     // [2][th][tw]: re, im
    const int image = blockIdx.x, h = blockIdx.y, tile = blockIdx.z;
    const int k = image / C;
    const int tu0 = (tile % ntx) * tw, tv0 = (tile / ntx) * th;
    const int tw_eff = min(tw, ww - tu0), th_eff = min(th, wh - tv0);
    float *wre = win, *wim = win + (size_t)tw * th;
    for (int i = threadIdx.x; i < 2 * tw * th; i += kThreads) win[i] = 0.f;
    __syncthreads();
    const int2 *v = reinterpret_cast<const int2 *>(vis) + (size_t)image * nbl * P * P;
    const float2 *ph = phasor + (size_t)k * nbl;
    for (int q = tile_start[tile] + threadIdx.x; q < tile_start[tile + 1]; q += kThreads) {
        const int bl = tile_pairs[q];
        const PairRec r = rec[bl];
        const float2 w = ph[bl];
        const int2 *vb = v + (size_t)bl * P * P;
        float2 g, gm;
        if (h == 0) {
            const int2 a = vb[0];
            const float2 xx = cmulf(make_float2((float)a.x, (float)a.y), w);
            float2 yy = make_float2(0.f, 0.f);
            if (P == 2) {
                const int2 b = vb[3];
                yy = cmulf(make_float2((float)b.x, (float)b.y), w);
            }
            g = make_float2(xx.x - yy.y, xx.y + yy.x);                  // XX + i YY
            gm = make_float2(xx.x + yy.y, -xx.y + yy.x);                // conj(XX) + i conj(YY)
        } else {
            const int2 a = vb[1], b = vb[2];
            g = cmulf(make_float2((float)a.x, (float)a.y), w);          // XY of (m, n)
            const float2 t = cmulf(make_float2((float)b.x, (float)b.y), w);
            gm = make_float2(t.x, -t.y);                                // XY of (n, m) = conj(YX~)
        }
        add_footprint(wre, wim, tu0, tv0, tw_eff, th_eff, r.du, r.dv, r.fu, r.fv, g);
        if (r.mu >= 0) add_footprint(wre, wim, tu0, tv0, tw_eff, th_eff, r.mu, r.mv, r.mfu, r.mfv, gm);
    }
    __syncthreads();
    float *pre = img + ((size_t)image * 4 + 2 * h) * N * N, *pim = pre + (size_t)N * N;
    for (int i = threadIdx.x; i < tw_eff * th_eff; i += kThreads) {
        const int cu = i % tw_eff, cv = i / tw_eff;
        const int u = win_u0 + tu0 + cu, v = win_v0 + tv0 + cv;
        const int x = (u + N) % N, y = (v + N) % N;
        const float sgn = ((u + v) & 1) ? -1.f : 1.f;
        pre[(size_t)y * N + x] = sgn * wre[cv * tw_eff + cu];     // rows tw_eff apart, as add_footprint wrote them
        pim[(size_t)y * N + x] = sgn * wim[cv * tw_eff + cu];
    }
}

// Twiddles exp(+2 pi i k / n), k < n / 2, into shared memory: sincospif of
// 2k / n, the same argument (exact in FP32 for power-of-two n) as pos / half
// of the butterfly that uses entry k.
__device__ __forceinline__ void load_twiddles(float2 *tw, int n) {
    for (int k = threadIdx.x; k < n / 2; k += blockDim.x) {
        float s, c;
        sincospif((float)(2 * k) / (float)n, &s, &c);
        tw[k] = make_float2(c, s);
    }
}

// In-place radix-2 FFT (exponent +) of n points held in bit-reversed order at
// x[0], x[stride], ... by one warp; tw as load_twiddles wrote it.
__device__ void warp_fft(float2 *x, int stride, int n, int log2n, const float2 *tw, int lane) {
    for (int lh = 0; lh < log2n; lh++) {
        const int half = 1 << lh, tshift = log2n - 1 - lh;       // twiddle of pos: tw[pos * n / (2 half)]
        for (int b = lane; b < n / 2; b += 32) {
            const int pos = b & (half - 1);
            const int i0 = ((b - pos) << 1) + pos, i1 = i0 + half;
            const float2 a = x[i0 * stride];
            const float2 t = cmulf(x[i1 * stride], tw[pos << tshift]);
            x[i0 * stride] = make_float2(a.x + t.x, a.y + t.y);
            x[i1 * stride] = make_float2(a.x - t.x, a.y - t.y);
        }
        __syncwarp();
    }
}

// Row pass: one warp per row of a plane pair (re plane, im plane).
__global__ void __launch_bounds__(kThreads) fft_rows_kernel(float *__restrict__ img, int N, int log2n) {
    extern __shared__ float2 rows[];   // [16][N], then the N / 2 twiddles
    float2 *tw = rows + (size_t)(kThreads / 32) * N;
    load_twiddles(tw, N);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pair = blockIdx.x;       // image * 2 + h
    const int y = blockIdx.y * (kThreads / 32) + warp;
    if (y >= N) return;
    float *pre = img + ((size_t)(pair >> 1) * 4 + 2 * (pair & 1)) * N * N + (size_t)y * N;
    float *pim = pre + (size_t)N * N;
    float2 *x = rows + (size_t)warp * N;
    // lane takes the N / 32 consecutive points j = E lane + k: their
    // bit-reversed slots for one k are a permutation of 32 adjacent entries,
    // so the stores are free of bank conflicts (j = lane + 32 k would put the
    // lanes 64 bytes apart)
    const int E = N / 32;
    if (E >= 4) {
        for (int k = 0; k < E; k += 4) {
            const int j = E * lane + k;
            const float4 r = *reinterpret_cast<const float4 *>(pre + j), m = *reinterpret_cast<const float4 *>(pim + j);
            x[__brev(j) >> (32 - log2n)] = make_float2(r.x, m.x);
            x[__brev(j + 1) >> (32 - log2n)] = make_float2(r.y, m.y);
            x[__brev(j + 2) >> (32 - log2n)] = make_float2(r.z, m.z);
            x[__brev(j + 3) >> (32 - log2n)] = make_float2(r.w, m.w);
        }
    } else {
        for (int j = lane; j < N; j += 32) x[__brev(j) >> (32 - log2n)] = make_float2(pre[j], pim[j]);
    }
    __syncwarp();
    warp_fft(x, 1, N, log2n, tw, lane);
    for (int j = lane; j < N; j += 32) {
        pre[j] = x[j].x;
        pim[j] = x[j].y;
    }
}

// Column pass: a CTA loads 32 columns of a plane pair and each warp
// transforms two of them.
__global__ void __launch_bounds__(kThreads) fft_cols_kernel(float *__restrict__ img, int N, int log2n) {
    extern __shared__ float2 tile[];   // [N][33], then the N / 2 twiddles
    float2 *tw = tile + (size_t)N * 33;
    load_twiddles(tw, N);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pair = blockIdx.x;
    const int x0 = blockIdx.y * 32;
    float *pre = img + ((size_t)(pair >> 1) * 4 + 2 * (pair & 1)) * N * N;
    float *pim = pre + (size_t)N * N;
    const int ncol = min(32, N - x0);
    for (int i = threadIdx.x; i < N * 32; i += kThreads) {
        const int y = i / 32, c = i % 32;
        if (c < ncol) tile[(__brev(y) >> (32 - log2n)) * 33 + c] = make_float2(pre[(size_t)y * N + x0 + c],
                                                                               pim[(size_t)y * N + x0 + c]);
    }
    __syncthreads();
    for (int c = warp; c < ncol; c += kThreads / 32) warp_fft(tile + c, 33, N, log2n, tw, lane);
    __syncthreads();
    for (int i = threadIdx.x; i < N * 32; i += kThreads) {
        const int y = i / 32, c = i % 32;
        if (c < ncol) {
            pre[(size_t)y * N + x0 + c] = tile[y * 33 + c].x;
            pim[(size_t)y * N + x0 + c] = tile[y * 33 + c].y;
        }
    }
}

// beams [S][C][T][K][P][2] -> [K][C][T][P][S][2]; one CTA per (c, t).  VEC:
// S and K P multiples of 8, 16-byte aligned buffers: every station's K P
// values and every output row move as 16-byte vectors through a shared slab
// [K P][Spad] (rows padded to keep 16-byte alignment).
template <bool VEC>
__global__ void __launch_bounds__(256) beams_to_corr_kernel(const char2 *__restrict__ in, int S, int C, int T, int KP,
                                                            int P, char2 *__restrict__ out) {
    extern __shared__ __align__(16) char2 slab[];
    const int Spad = VEC ? ((S + 7) & ~7) + 8 : S + 1;
    const long long ct = blockIdx.x;   // c * T + t
    const int c = (int)(ct / T), t = (int)(ct - (long long)c * T);
    if (VEC) {
        const int vpr = KP / 8;        // vectors per station segment
        for (int i = threadIdx.x; i < S * vpr; i += blockDim.x) {
            const int st = i / vpr, j0 = (i - st * vpr) * 8;
            const uint4 v = reinterpret_cast<const uint4 *>(in + ((size_t)st * C * T + ct) * KP)[i - st * vpr];
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 8; e++) {
                const uint32_t h = (w[e >> 1] >> (16 * (e & 1))) & 0xffffu;
                slab[(j0 + e) * Spad + st] = *reinterpret_cast<const char2 *>(&h);
            }
        }
    } else {
        for (int i = threadIdx.x; i < S * KP; i += blockDim.x) {
            const int st = i / KP, j = i - st * KP;
            slab[j * Spad + st] = in[((size_t)st * C * T + ct) * KP + j];
        }
    }
    __syncthreads();
    if (VEC) {
        const int vpr = S / 8;
        for (int i = threadIdx.x; i < KP * vpr; i += blockDim.x) {
            const int j = i / vpr, s0 = (i - j * vpr) * 8;   // j = (k, p)
            const int k = j / P, p = j - k * P;
            char2 *o = out + ((((size_t)k * C + c) * T + t) * P + p) * S + s0;
            *reinterpret_cast<uint4 *>(o) = *reinterpret_cast<const uint4 *>(slab + j * Spad + s0);
        }
    } else {
        for (int i = threadIdx.x; i < S * KP; i += blockDim.x) {
            const int j = i / S, st = i - j * S;     // j = (k, p)
            const int k = j / P, p = j - k * P;
            out[((((size_t)k * C + c) * T + t) * P + p) * S + st] = slab[j * Spad + st];
        }
    }
}

}  // namespace

struct hai_vis_layout {
    hai_ctx *ctx = nullptr;
    int S = 0, N = 0, P = 0, K = 0;
    long long nbl = 0;
    int win_u0 = 0, win_v0 = 0, ww = 0, wh = 0;
    int tw = 0, th = 0, ntx = 0, nty = 0;    // tiles of the window, one CTA each
    long long n_offgrid = 0;
    PairRec *d_rec = nullptr;
    float2 *d_phasor = nullptr;
    int32_t *d_tile_start = nullptr, *d_tile_pairs = nullptr;
};

void vis_layout_dims(const hai_vis_layout *L, int *S, int *N, int *K) {
    *S = L->S;
    *N = L->N;
    *K = L->K;
}

static void vis_layout_free(hai_vis_layout *L) {
    if (!L) return;
    cudaFree(L->d_rec);
    cudaFree(L->d_phasor);
    cudaFree(L->d_tile_start);
    cudaFree(L->d_tile_pairs);
    delete L;
}

extern "C" hai_status hai_vis_layout_create(hai_ctx *ctx, const hai_vis_layout_desc *d, hai_vis_layout **out) {
    if (!ctx || !d || !out) return hai_fail(HAI_ERR_INVALID_ARG, "hai_vis_layout_create: NULL argument");
    *out = nullptr;
    const int S = d->n_station, N = d->grid_n, K = d->n_dir;
    if (S <= 0 || !d->pos_m || !(d->lambda_m > 0) || !(d->cell_m > 0) || (d->n_pol != 1 && d->n_pol != 2) ||
        K <= 0 || N < 16 || N > 256 || (N & (N - 1)))
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_vis_layout_create: bad descriptor (grid_n a power of two in 16..256)");
    if (d->n_pol != 2) return hai_fail(HAI_ERR_UNSUPPORTED, "hai_vis_layout_create: station images need 2 pols");
    if (hai_fault_injected("alloc")) return hai_fail(HAI_ERR_NO_MEMORY, "hai_vis_layout_create: injected allocation failure");
    const long long nbl = (long long)S * (S + 1) / 2;
    // footprints in FP64 on the host: lower corner floor(uv) and fraction
    std::vector<PairRec> rec(nbl);
    std::vector<long> cu(nbl), cv(nbl), mcu(nbl), mcv(nbl);
    std::vector<float> fu(nbl), fv(nbl), mfu(nbl), mfv(nbl);
    std::vector<char> ok(nbl);
    long umin = N, vmin = N, umax = -N, vmax = -N;
    long long dropped = 0;
    for (int m = 0, bl = 0; m < S; m++)
        for (int n = 0; n <= m; n++, bl++) {
            const double du = (d->pos_m[2 * m] - d->pos_m[2 * n]) / d->cell_m;
            const double dv = (d->pos_m[2 * m + 1] - d->pos_m[2 * n + 1]) / d->cell_m;
            const double a = floor(du), b = floor(dv), ma = floor(-du), mb = floor(-dv);
            cu[bl] = (long)a;
            cv[bl] = (long)b;
            mcu[bl] = (long)ma;
            mcv[bl] = (long)mb;
            fu[bl] = (float)(du - a);
            fv[bl] = (float)(dv - b);
            mfu[bl] = (float)(-du - ma);
            mfv[bl] = (float)(-dv - mb);
            ok[bl] = station_pair_kept(N, du, dv);
            if (!ok[bl]) {
                dropped++;
                continue;
            }
            umin = std::min(umin, std::min(cu[bl], mcu[bl]));
            vmin = std::min(vmin, std::min(cv[bl], mcv[bl]));
            umax = std::max(umax, std::max(cu[bl], mcu[bl]) + 1);
            vmax = std::max(vmax, std::max(cv[bl], mcv[bl]) + 1);
        }
    hai_vis_layout *L = new hai_vis_layout();
    L->ctx = ctx;
    L->S = S;
    L->N = N;
    L->P = d->n_pol;
    L->K = K;
    L->nbl = nbl;
    L->n_offgrid = dropped;
    L->win_u0 = (int)umin;
    L->win_v0 = (int)vmin;
    L->ww = (int)(umax - umin + 1);
    L->wh = (int)(vmax - vmin + 1);
    for (int m = 0, bl = 0; m < S; m++)
        for (int n = 0; n <= m; n++, bl++) {
            PairRec &r = rec[bl];
            if (!ok[bl]) {
                r = PairRec{-1, -1, -1, -1, 0.f, 0.f, 0.f, 0.f};
                continue;
            }
            r.du = (int16_t)(cu[bl] - umin);
            r.dv = (int16_t)(cv[bl] - vmin);
            r.fu = fu[bl];
            r.fv = fv[bl];
            // an auto pair has no mirror
            r.mu = (int16_t)(m == n ? -1 : mcu[bl] - umin);
            r.mv = (int16_t)(mcv[bl] - vmin);
            r.mfu = mfu[bl];
            r.mfv = mfv[bl];
        }
    // tiles of at most side^2 cells (2 x 4 bytes each in shared memory); pairs
    // per tile: every tile that the pair's footprint or its mirror's touches.
    // The time follows the tiles that hold the densest cells (short
    // baselines near the window's centre): the smaller side spreads them over
    // more CTAs, which pays where the tiles stay well filled (measured: 512
    // stations in a 3 km core 6.1 -> 4.9 ms, 256 stations 0.91 -> 1.17 ms)
    std::vector<std::vector<int32_t>> lists;
    int ntile = 0;
    for (int side : {kTileSmall, kTileCells}) {
        L->ntx = (L->ww + side - 1) / side;
        L->nty = (L->wh + side - 1) / side;
        L->tw = (L->ww + L->ntx - 1) / L->ntx;
        L->th = (L->wh + L->nty - 1) / L->nty;
        ntile = L->ntx * L->nty;
        lists.assign(ntile, {});
        size_t binned = 0;
        for (long long bl = 0; bl < nbl; bl++) {
            const PairRec &r = rec[bl];
            if (r.du < 0) continue;
            int seen[8], ns = 0;
            auto touch = [&](int du, int dv) {
                for (int t = 0; t < 4; t++) {
                    const int tx = (du + (t & 1)) / L->tw, ty = (dv + (t >> 1)) / L->th;
                    const int id = ty * L->ntx + tx;
                    bool dup = false;
                    for (int j = 0; j < ns; j++) dup |= seen[j] == id;
                    if (!dup) seen[ns++] = id;
                }
            };
            touch(r.du, r.dv);
            if (r.mu >= 0) touch(r.mu, r.mv);
            for (int j = 0; j < ns; j++) lists[seen[j]].push_back((int32_t)bl);
            binned += ns;
        }
        if (side == kTileCells || binned >= kTilePairsMin * (size_t)ntile) break;
    }
    std::vector<int32_t> tstart(ntile + 1, 0), tpairs;
    for (int t = 0; t < ntile; t++) {
        tpairs.insert(tpairs.end(), lists[t].begin(), lists[t].end());
        tstart[t + 1] = (int32_t)tpairs.size();
    }
    double *d_pos = nullptr, *d_dir = nullptr;
    std::vector<double> dirs(2 * (size_t)K, 0.0);
    if (d->dir) std::copy(d->dir, d->dir + 2 * (size_t)K, dirs.begin());
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaMalloc(&L->d_rec, sizeof(PairRec) * nbl);
    if (e == cudaSuccess) e = cudaMemcpy(L->d_rec, rec.data(), sizeof(PairRec) * nbl, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&L->d_phasor, sizeof(float2) * (size_t)K * nbl);
    if (e == cudaSuccess) e = cudaMalloc(&L->d_tile_start, sizeof(int32_t) * tstart.size());
    if (e == cudaSuccess) e = cudaMalloc(&L->d_tile_pairs, sizeof(int32_t) * std::max<size_t>(1, tpairs.size()));
    if (e == cudaSuccess)
        e = cudaMemcpy(L->d_tile_start, tstart.data(), sizeof(int32_t) * tstart.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !tpairs.empty())
        e = cudaMemcpy(L->d_tile_pairs, tpairs.data(), sizeof(int32_t) * tpairs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&d_pos, sizeof(double) * 2 * S);
    if (e == cudaSuccess) e = cudaMalloc(&d_dir, sizeof(double) * 2 * K);
    if (e == cudaSuccess) e = cudaMemcpy(d_pos, d->pos_m, sizeof(double) * 2 * S, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_dir, dirs.data(), sizeof(double) * 2 * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const long long n = (long long)K * nbl;
        steering_kernel<<<(unsigned)((n + 255) / 256), 256>>>(d_pos, d_dir, K, nbl, 1.0 / d->lambda_m, L->d_phasor);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_pos);
    cudaFree(d_dir);
    if (e != cudaSuccess) {
        vis_layout_free(L);
        return hai_cuda_fail(e, "hai_vis_layout_create");
    }
    *out = L;
    return HAI_OK;
}

extern "C" void hai_vis_layout_destroy(hai_vis_layout *L) {
    if (!L) return;
    cudaSetDevice(L->ctx->device);
    vis_layout_free(L);
}

extern "C" hai_status hai_vis_layout_offgrid(const hai_vis_layout *L, long long *n_offgrid) {
    if (!L || !n_offgrid) return hai_fail(HAI_ERR_INVALID_ARG, "hai_vis_layout_offgrid: NULL argument");
    *n_offgrid = L->n_offgrid;
    return HAI_OK;
}

extern "C" hai_status hai_xfft_station_image(hai_ctx *ctx, const hai_vis_layout *L, const int32_t *vis, int C,
                                             float *img, void *stream) {
    if (!ctx || !L) return hai_fail(HAI_ERR_INVALID_ARG, "hai_xfft_station_image: NULL ctx or layout");
    if (L->ctx != ctx) return hai_fail(HAI_ERR_INVALID_ARG, "hai_xfft_station_image: layout of another context");
    if (C < 0) return hai_fail(HAI_ERR_INVALID_ARG, "hai_xfft_station_image: negative channel count");
    if (C == 0) return HAI_OK;
    if (!vis || !img) return hai_fail(HAI_ERR_INVALID_ARG, "hai_xfft_station_image: NULL buffer");
    if (hai_fault_injected("launch")) return hai_fail(HAI_ERR_CUDA, "hai_xfft_station_image: injected launch failure");
    HAI_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int N = L->N, images = L->K * C;
    int log2n = 0;
    while ((1 << log2n) < N) log2n++;
    const size_t win_bytes = (size_t)2 * L->tw * L->th * sizeof(float);
    HAI_CUDA_TRY(hai_allow_dyn_smem(station_grid_kernel, ctx->smem_optin));
    if ((long long)images * 2 > 0x7fffffffll) return hai_fail(HAI_ERR_UNSUPPORTED, "hai_xfft_station_image: too many images");
    // cells outside the window stay zero; the tiles write the rest
    HAI_CUDA_TRY(cudaMemsetAsync(img, 0, sizeof(float) * (size_t)images * 4 * N * N, st));
    const int pidx = prof_begin(ctx, st);
    station_grid_kernel<<<dim3(images, 2, L->ntx * L->nty), kThreads, win_bytes, st>>>(
        vis, L->d_rec, L->d_phasor, L->d_tile_start, L->d_tile_pairs, C, L->nbl, L->P, N, L->win_u0, L->win_v0, L->ww,
        L->wh, L->tw, L->th, L->ntx, img);
    prof_end(ctx, pidx, st);
    HAI_CUDA_TRY(cudaGetLastError());
    const int rows_per_cta = kThreads / 32;
    fft_rows_kernel<<<dim3(images * 2, (N + rows_per_cta - 1) / rows_per_cta), kThreads,
                      sizeof(float2) * (rows_per_cta * N + N / 2), st>>>(img, N, log2n);
    HAI_CUDA_TRY(cudaGetLastError());
    const size_t tile = sizeof(float2) * ((size_t)N * 33 + N / 2);
    HAI_CUDA_TRY(hai_allow_dyn_smem(fft_cols_kernel, ctx->smem_optin));
    fft_cols_kernel<<<dim3(images * 2, (N + 31) / 32), kThreads, tile, st>>>(img, N, log2n);
    prof_count(ctx, 3);
    HAI_CUDA_TRY(cudaGetLastError());
    return HAI_OK;
}

extern "C" hai_status hai_beams_to_corr(hai_ctx *ctx, const int8_t *beams, int S, int C, int T, int K, int P,
                                        int8_t *out, void *stream) {
    if (!ctx) return hai_fail(HAI_ERR_INVALID_ARG, "hai_beams_to_corr: NULL ctx");
    if (S <= 0 || C < 0 || T < 0 || K <= 0 || (P != 1 && P != 2))
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_beams_to_corr: bad sizes");
    if ((long long)C * T == 0) return HAI_OK;
    if (!beams || !out) return hai_fail(HAI_ERR_INVALID_ARG, "hai_beams_to_corr: NULL buffer");
    const bool vec = S % 8 == 0 && (K * P) % 8 == 0 && (((uintptr_t)beams | (uintptr_t)out) & 15) == 0;
    const size_t smem = sizeof(char2) * (size_t)K * P * (vec ? ((S + 7) & ~7) + 8 : S + 1);
    if (smem > 48 * 1024) return hai_fail(HAI_ERR_UNSUPPORTED, "hai_beams_to_corr: S x K x P too large for one tile");
    if ((long long)C * T > 0x7fffffffll) return hai_fail(HAI_ERR_UNSUPPORTED, "hai_beams_to_corr: too many samples");
    HAI_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned grid = (unsigned)((long long)C * T);
    const char2 *in = reinterpret_cast<const char2 *>(beams);
    char2 *o = reinterpret_cast<char2 *>(out);
    if (vec)
        beams_to_corr_kernel<true><<<grid, 256, smem, st>>>(in, S, C, T, K * P, P, o);
    else
        beams_to_corr_kernel<false><<<grid, 256, smem, st>>>(in, S, C, T, K * P, P, o);
    prof_count(ctx, 1);
    HAI_CUDA_TRY(cudaGetLastError());
    return HAI_OK;
}
