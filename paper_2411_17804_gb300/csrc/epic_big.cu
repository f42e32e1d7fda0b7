// EPIC on tcgen05 tensor cores for large grids (N = 256, 512): Eq.
// intra-station EPIC, then the squaring and temporal sum of Eq. intra-station
// squaring, FP16 operands and FP32 accumulation.
//
// The 2D DFT of the kernel's bounding box (<= N/2 x N/2 cells, at the
// transform's origin; the shift by the box corner is a phase common to both
// polarisations and cancels in every product) is two dense complex products
// with W'[j][l] = (-1)^j exp(+2 pi i l j / N) (the (-1)^j puts the phase
// centre at pixel N/2), written as real GEMMs.  A grid of 512^2 does not fit
// one SM, so the stages run as three kernels per batch of (channel, sample)
// pairs, through HBM:
//   grid:   every field (channel, sample, pol) gathered into its box (FP32
//           sums of conj(W~) E, stored fp16; one thread per cell and 8
//           fields), K-major in the tensor cores' tile order:
//           A1[field][y block][k block] = 128 rows y x 64 (x, re/im);
//   stage1: H[y][l_x] = sum_x G[y][x] W'[x][l_x]: persistent CTAs over
//           (field, y block, 128-wide l_x block) tiles, bulk copies of A1 and
//           the constant DFT operand, tcgen05.mma M = 128, N = 256 (re, im of
//           128 l_x), accumulator double-buffered in TMEM; the epilogue stores
//           H as fp16, transposed, into the stage-2 operand layout:
//           A2[channel, sample][64-wide l_x block][k block] = MN-major tiles
//           of 128 rows (l_x, pol) x 64 (y, re/im);
//   stage2: F[l_y][l_x] = sum_y W'[y][l_y] H[y][l_x] for a 64 x 64 pixel
//           tile of one channel: persistent CTAs over (channel, l_x block,
//           l_y block), the tile's DFT operand resident in shared memory, the
//           A2 tiles of each sample streamed by bulk copies, M = 128 (l_x,
//           pol), N = 128 (re, im of 64 l_y); the epilogue adds |F_X|^2,
//           |F_Y|^2 and F_X conj(F_Y) of the pixel tile into registers over
//           the samples and writes the tile once per item.
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "hai_internal.h"
#include "tc.cuh"

namespace {

constexpr uint32_t kKBytes = 128;        // K-major: K-group stride
constexpr uint32_t kKMN = 1024;          // K-major: MN-group stride (64-deep k block)
constexpr uint32_t kMKs = 2048;          // MN-major (128 rows): K-group stride
constexpr uint32_t kMMN = 128;           // MN-major: MN-group stride
constexpr uint32_t kTile16 = 16384;      // 128 rows x 64 K fp16
constexpr uint32_t kTile32 = 32768;      // 256 rows x 64 K fp16
constexpr int kS1Stages = 4;
constexpr uint32_t kIdesc1 = tc::idesc_f16(128, 256, 0, 0);
constexpr uint32_t kIdesc2 = tc::idesc_f16(128, 128, 1, 0);

struct BigGeo {
    int N, P, bx, by;            // grid, pols, box (cells)
    int kb1;                     // k blocks of stage 1: 2 bx_pad / 64
    int yb;                      // y blocks of 128 rows: by_pad / 128
    int kb2;                     // k blocks of stage 2: 2 by_pad / 64
    int lb1;                     // 128-wide l_x blocks: N / 128
    int lb2;                     // 64-wide l blocks: N / 64
};

// ------------------------------------------------------------------ grid
// one thread per (cell of the padded box, row-major; group of kGridFields
// fields): the cell's entries are read once for the group and the fields'
// voltage loads are independent, so they are in flight together.  Fields of
// the batch are f = (c T + t - b0) P + pol.
constexpr int kGridFields = 8;

__global__ void __launch_bounds__(256) big_grid_kernel(const int8_t *__restrict__ volt, int ne,
                                                       const int32_t *__restrict__ cell_start,
                                                       const int32_t *__restrict__ entry_elem,
                                                       const float2 *__restrict__ entry_w, BigGeo g, long long b0,
                                                       long long nfield, uint8_t *__restrict__ a1) {
    const int bxp = g.kb1 * 32, byp = g.yb * 128;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= bxp * byp) return;
    const int x = i % bxp, y = i / bxp;
    const long long f0 = (long long)blockIdx.y * kGridFields;
    const int nf = (int)(nfield - f0 < kGridFields ? nfield - f0 : kGridFields);
    int k0 = 0, k1 = 0;
    if (x < g.bx && y < g.by) {
        k0 = cell_start[y * g.bx + x];
        k1 = cell_start[y * g.bx + x + 1];
    }
    // voltages of field f: volt + ((b0 P + f) ne) char2
    const char2 *E = reinterpret_cast<const char2 *>(volt) + (size_t)(b0 * g.P + f0) * ne;
    float2 acc[kGridFields];
#pragma unroll
    for (int j = 0; j < kGridFields; j++) acc[j] = make_float2(0.f, 0.f);
    for (int k = k0; k < k1; k++) {
        const int e = entry_elem[k];
        const float2 w = entry_w[k];                           // conj(W~)
        char2 v[kGridFields];
#pragma unroll
        for (int j = 0; j < kGridFields; j++) v[j] = j < nf ? E[(size_t)j * ne + e] : make_char2(0, 0);
#pragma unroll
        for (int j = 0; j < kGridFields; j++) {
            acc[j].x = fmaf(w.x, (float)v[j].x, fmaf(-w.y, (float)v[j].y, acc[j].x));
            acc[j].y = fmaf(w.x, (float)v[j].y, fmaf(w.y, (float)v[j].x, acc[j].y));
        }
    }
    const int k = 2 * x;
    const size_t field_bytes = (size_t)g.yb * g.kb1 * kTile16;
    uint8_t *dst = a1 + (size_t)f0 * field_bytes + ((size_t)(y / 128) * g.kb1 + k / 64) * kTile16 +
                   tc::off_kmajor(y % 128, k % 64, kKBytes, kKMN);
#pragma unroll
    for (int j = 0; j < kGridFields; j++)
        if (j < nf) *reinterpret_cast<uint32_t *>(dst + (size_t)j * field_bytes) = tc::pack_half2(acc[j].x, acc[j].y);
}

// ------------------------------------------------------------------ stage 1
struct S1Params {
    const uint8_t *a1, *b1;
    uint8_t *a2;
    BigGeo g;
    long long b0, nfield;        // batch start (c T + t) and fields in the batch
    long long ntiles;
    unsigned *status;
};

__global__ void __launch_bounds__(384, 1) big_s1_kernel(const S1Params p) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[kS1Stages], empty[kS1Stages], dfull[2], dempty[2];
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const BigGeo g = p.g;
    if (tid == 0) {
        for (int s = 0; s < kS1Stages; s++) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&dfull[b], 1);
            tc::mbar_init(&dempty[b], 256);
        }
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc(&tslot, 512);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tslot;
    auto sA = [&](int s) { return smem + (size_t)s * (kTile16 + kTile32); };
    auto sB = [&](int s) { return smem + (size_t)s * (kTile16 + kTile32) + kTile16; };
    const int per_field = g.yb * g.lb1;
    if (warp == 0) {
        if (lane == 0) {
            long long gs = 0;
            for (long long tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x) {
                const long long f = tile / per_field;
                const int r = (int)(tile % per_field), ybk = r / g.lb1, lb = r % g.lb1;
                const uint8_t *ab = p.a1 + ((size_t)f * g.yb + ybk) * g.kb1 * kTile16;
                const uint8_t *bb = p.b1 + (size_t)lb * g.kb1 * kTile32;
                for (int kb = 0; kb < g.kb1; kb++, gs++) {
                    const int s = (int)(gs % kS1Stages);
                    if (gs >= kS1Stages) tc::mbar_wait(&empty[s], (uint32_t)(((gs / kS1Stages) - 1) & 1), p.status);
                    tc::mbar_arrive_expect_tx(&full[s], kTile16 + kTile32);
                    tc::bulk_g2s(sA(s), ab + (size_t)kb * kTile16, kTile16, &full[s]);
                    tc::bulk_g2s(sB(s), bb + (size_t)kb * kTile32, kTile32, &full[s]);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            long long gs = 0, gt = 0;
            for (long long tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x, gt++) {
                const int b = (int)(gt & 1);
                if (gt >= 2) tc::mbar_wait(&dempty[b], (uint32_t)(((gt >> 1) - 1) & 1), p.status);
                tc::fence_after();
                const uint32_t d = tmem + (uint32_t)b * 256u;
                for (int kb = 0; kb < g.kb1; kb++, gs++) {
                    const int s = (int)(gs % kS1Stages);
                    tc::mbar_wait(&full[s], (uint32_t)((gs / kS1Stages) & 1), p.status);
                    tc::fence_after();
                    const uint32_t a = tc::smem_u32(sA(s)), bq = tc::smem_u32(sB(s));
#pragma unroll
                    for (int j = 0; j < 4; j++)
                        tc::mma_f16(d, tc::desc(a + j * 2 * kKBytes, kKBytes, kKMN),
                                    tc::desc(bq + j * 2 * kKBytes, kKBytes, kKMN), kIdesc1, (kb > 0 || j > 0) ? 1u : 0u);
                    tc::mma_commit(&empty[s]);
                }
                tc::mma_commit(&dfull[b]);
            }
        }
    } else if (warp >= 4) {
        // epilogue, warps 4-11: thread = row y of the tile and one half (h) of
        // its 128 (re, im) values -> the stage-2 operand rows (l_x, pol), K
        // index 2 y + re/im
        const int q = warp & 3, row = q * 32 + lane, h = (warp - 4) >> 2;
        long long gt = 0;
        for (long long tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x, gt++) {
            const int b = (int)(gt & 1);
            const long long f = tile / per_field;
            const int r = (int)(tile % per_field), ybk = r / g.lb1, lb = r % g.lb1;
            const int pol = (int)(f % g.P);
            const long long ct = f / g.P;                       // (c, t) in the batch
            const int y = ybk * 128 + row;
            const int kr = 2 * y, kb2 = kr / 64, kk = kr % 64;  // K of the real part; imag at kk + 1
            tc::mbar_wait(&dfull[b], (uint32_t)((gt >> 1) & 1), p.status);
            tc::fence_after();
#pragma unroll 1
            for (int ch = 4 * h; ch < 4 * h + 4; ch++) {       // 16 l_x values per chunk
                uint32_t rr[16], ri[16];
                tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)b * 256u + (uint32_t)(16 * ch), rr);
                tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)b * 256u + 128u + (uint32_t)(16 * ch), ri);
                tc::tmem_wait_ld();
                const int lx = lb * 128 + 16 * ch;             // first l_x of the chunk
                const int lxb = lx / 64, lx64 = lx % 64;
                uint8_t *tile2 = p.a2 + (((size_t)ct * g.lb2 + lxb) * g.kb2 + kb2) * kTile16;
                // rows (l_x, pol): m = (l_x >> 4) 32 + pol 16 + (l_x & 15)
                const int m0 = (lx64 >> 4) * 32 + pol * 16;
#pragma unroll
                for (int half = 0; half < 2; half++) {          // 8 l_x -> one 16-byte run per K value
                    uint32_t hr[4], hi[4];
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        hr[e] = tc::pack_half2(__uint_as_float(rr[8 * half + 2 * e]), __uint_as_float(rr[8 * half + 2 * e + 1]));
                        hi[e] = tc::pack_half2(__uint_as_float(ri[8 * half + 2 * e]), __uint_as_float(ri[8 * half + 2 * e + 1]));
                    }
                    const int m = m0 + 8 * half;
                    *reinterpret_cast<uint4 *>(tile2 + tc::off_mnmajor(m, kk, kMKs, kMMN)) =
                        make_uint4(hr[0], hr[1], hr[2], hr[3]);
                    *reinterpret_cast<uint4 *>(tile2 + tc::off_mnmajor(m, kk + 1, kMKs, kMMN)) =
                        make_uint4(hi[0], hi[1], hi[2], hi[3]);
                }
            }
            tc::fence_before();
            tc::mbar_arrive(&dempty[b]);
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------------ stage 2
struct S2Params {
    const uint8_t *a2, *b2;
    float *img;
    BigGeo g;
    long long b0, b1;            // batch range of c T + t
    int T, c_first, n_items;     // items: (channel - c_first, l_x block, l_y block)
    int accumulate;
    unsigned *status;
};

constexpr int kS2Threads = 384;             // warp 0 loads, warp 1 MMA, warps 4-11 epilogue
constexpr int kS2Kb = 4;                    // k blocks of stage 2 (boxes <= 128 rows: 2 x 128 / 64)
constexpr int kS2Epi = 256;

__global__ void __launch_bounds__(kS2Threads, 1) big_s2_kernel(const S2Params p) {
    extern __shared__ __align__(1024) uint8_t smem[];
    // sdone[b]: every MMA of the sample in A buffer / accumulator b has completed
    // (one commit per sample: the loader may refill A buffer b, the epilogue
    // may read accumulator b)
    __shared__ __align__(8) uint64_t bfull, afull[2], sdone[2], dempty[2];
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const BigGeo g = p.g;
    const uint32_t abytes = (uint32_t)g.kb2 * kTile16;     // one sample's A2 for a 64-wide l_x block
    uint8_t *sB = smem;                                      // [kb2][16 KB]
    auto sA = [&](int s) { return smem + abytes + (size_t)s * abytes; };
    if (tid == 0) {
        tc::mbar_init(&bfull, 1);
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&afull[b], 1);
            tc::mbar_init(&sdone[b], 1);
            tc::mbar_init(&dempty[b], kS2Epi);
        }
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc(&tslot, 256);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tslot;
    const int per_chan = g.lb2 * g.lb2;
    // samples of channel c in the batch
    auto trange = [&](int c, int &t0, int &t1) {
        const long long lo = (long long)c * p.T, hi = lo + p.T;
        t0 = (int)(max(p.b0, lo) - lo);
        t1 = (int)(min(p.b1, hi) - lo);
    };
    if (warp == 0) {
        if (lane == 0) {
            long long gs = 0;
            int cur_lyb = -1;
            uint32_t bphase = 0;
            for (int it = blockIdx.x; it < p.n_items; it += gridDim.x) {
                const int c = p.c_first + it / per_chan, r = it % per_chan, lxb = r / g.lb2, lyb = r % g.lb2;
                if (lyb != cur_lyb) {
                    // the previous item's MMAs have all completed once its last A stage is released
                    if (gs > 0) tc::mbar_wait(&sdone[(gs - 1) & 1], (uint32_t)(((gs - 1) >> 1) & 1), p.status);
                    tc::mbar_arrive_expect_tx(&bfull, abytes);
                    tc::bulk_g2s(sB, p.b2 + (size_t)lyb * abytes, abytes, &bfull);
                    cur_lyb = lyb;
                    bphase++;
                }
                int t0, t1;
                trange(c, t0, t1);
                for (int t = t0; t < t1; t++, gs++) {
                    const int s = (int)(gs & 1);
                    if (gs >= 2) tc::mbar_wait(&sdone[s], (uint32_t)(((gs >> 1) - 1) & 1), p.status);
                    const long long ct = (long long)c * p.T + t - p.b0;
                    tc::mbar_arrive_expect_tx(&afull[s], abytes);
                    tc::bulk_g2s(sA(s), p.a2 + ((size_t)ct * g.lb2 + lxb) * abytes, abytes, &afull[s]);
                }
            }
        }
    } else if (warp == 1) {
        // one thread issues 16 MMAs per sample (4 k blocks x 4), one commit;
        // descriptors advance by additions to their 14-bit address field
        if (lane == 0) {
            long long gs = 0;
            int cur_lyb = -1;
            uint32_t bph = 0;
            const uint64_t db0 = tc::desc(tc::smem_u32(sB), kKBytes, kKMN);
            const uint64_t da0 = tc::desc(tc::smem_u32(sA(0)), kMKs, kMMN);
            const uint64_t kBufD = abytes >> 4, kKbD = kTile16 >> 4, kStepA = (2 * kMKs) >> 4, kStepB = (2 * kKBytes) >> 4;
            for (int it = blockIdx.x; it < p.n_items; it += gridDim.x) {
                const int c = p.c_first + it / per_chan, r = it % per_chan, lyb = r % g.lb2;
                if (lyb != cur_lyb) {
                    tc::mbar_wait(&bfull, bph & 1, p.status);
                    bph++;
                    cur_lyb = lyb;
                }
                int t0, t1;
                trange(c, t0, t1);
                for (int t = t0; t < t1; t++, gs++) {
                    const int s = (int)(gs & 1);
                    const uint32_t ph = (uint32_t)((gs >> 1) & 1);
                    if (gs >= 2) tc::mbar_wait(&dempty[s], ph ^ 1u, p.status);
                    tc::mbar_wait(&afull[s], ph, p.status);
                    tc::fence_after();
                    const uint64_t da = da0 + (uint64_t)s * kBufD;
                    const uint32_t d = tmem + (uint32_t)s * 128u;
#pragma unroll
                    for (int kb = 0; kb < kS2Kb; kb++)
#pragma unroll
                        for (int j = 0; j < 4; j++)
                            tc::mma_f16(d, da + kb * kKbD + j * kStepA, db0 + kb * kKbD + j * kStepB, kIdesc2,
                                        (kb > 0 || j > 0) ? 1u : 0u);
                    tc::mma_commit(&sdone[s]);
                }
            }
        }
    } else if (warp >= 4) {
        // epilogue: the N = 64 tile epilogue of the small-grid kernel: thread
        // row m = (l_x, pol), half h of the 64 l_y
        const int q = warp & 3, h = (warp - 4) >> 2;
        const int m = 32 * q + lane;
        const int pol = (m >> 4) & 1, kx = (m >> 5) * 16 + (m & 15);
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        constexpr int kLy = 32;
        const size_t NN = (size_t)g.N * g.N;
        float2 acc_a[kLy / 2], acc_x[kLy / 2];
        long long gs = 0;
        for (int it = blockIdx.x; it < p.n_items; it += gridDim.x) {
            const int c = p.c_first + it / per_chan, r = it % per_chan, lxb = r / g.lb2, lyb = r % g.lb2;
#pragma unroll
            for (int t = 0; t < kLy / 2; t++) acc_a[t] = acc_x[t] = make_float2(0.f, 0.f);
            int t0, t1;
            trange(c, t0, t1);
            for (int t = t0; t < t1; t++, gs++) {
                const int s = (int)(gs & 1);
                tc::mbar_wait(&sdone[s], (uint32_t)((gs >> 1) & 1), p.status);
                tc::fence_after();
#pragma unroll
                for (int cc = 0; cc < 2; cc++) {
                    const uint32_t col = (uint32_t)s * 128u + (uint32_t)(kLy * h + 16 * cc);
                    uint32_t rr[16], ri[16];
                    tc::tmem_ld16(tmem + lane_base + col, rr);
                    tc::tmem_ld16(tmem + lane_base + col + 64, ri);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int k = 0; k < 16; k += 2) {
                        const float2 fr = make_float2(__uint_as_float(rr[k]), __uint_as_float(rr[k + 1]));
                        const float2 fi = make_float2(__uint_as_float(ri[k]), __uint_as_float(ri[k + 1]));
                        float2 &a = acc_a[(16 * cc + k) >> 1];
                        a = __ffma2_rn(fr, fr, __ffma2_rn(fi, fi, a));
                    }
#pragma unroll
                    for (int k = 0; k < 8; k++) {
                        const float e_r = __uint_as_float(rr[2 * k]), e_i = __uint_as_float(ri[2 * k]);
                        const float o_r = __uint_as_float(rr[2 * k + 1]), o_i = __uint_as_float(ri[2 * k + 1]);
                        const float mr = pol ? o_r : e_r, mi = pol ? o_i : e_i;
                        const float sr = __shfl_xor_sync(0xffffffffu, pol ? e_r : o_r, 16);
                        const float si = __shfl_xor_sync(0xffffffffu, pol ? e_i : o_i, 16);
                        float2 &a = acc_x[8 * cc + k];
                        a = __ffma2_rn(make_float2(mr, mi), make_float2(sr, sr),
                                       __ffma2_rn(make_float2(mi, -mr), make_float2(si, si), a));
                    }
                }
                tc::fence_before();
                tc::mbar_arrive(&dempty[s]);
            }
            // write the pixel tile (image planes XX, YY, Re XY, Im XY of channel c)
            const bool add = p.accumulate || t0 > 0;
            float *dst = p.img + (size_t)c * 4 * NN;
            const int px = lxb * 64 + kx;
#pragma unroll
            for (int t = 0; t < kLy; t++) {
                const size_t idx = pol * NN + (size_t)(lyb * 64 + kLy * h + t) * g.N + px;
                float v = (t & 1) ? acc_a[t >> 1].y : acc_a[t >> 1].x;
                if (add) v += dst[idx];
                dst[idx] = v;
            }
            const float sgn = pol ? -1.f : 1.f;
#pragma unroll
            for (int t = 0; t < kLy / 2; t++) {
                const int ly = kLy * h + 16 * (t >> 3) + 2 * (t & 7) + pol;
                const size_t idx = 2 * NN + (size_t)(lyb * 64 + ly) * g.N + px;
                float vr = acc_x[t].x, vi = sgn * acc_x[t].y;
                if (add) {
                    vr += dst[idx];
                    vi += dst[idx + NN];
                }
                dst[idx] = vr;
                dst[idx + NN] = vi;
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

BigGeo big_geo(const hai_layout *L) {
    BigGeo g;
    g.N = L->grid_n;
    g.P = L->n_pol;
    g.bx = L->box_w;
    g.by = L->box_h;
    g.kb1 = (2 * g.bx + 63) / 64;
    g.yb = (g.by + 127) / 128;
    g.kb2 = g.yb * 4;                                // 2 * by_pad / 64
    g.lb1 = g.N / 128;
    g.lb2 = g.N / 64;
    return g;
}

// W'[j][l] = (-1)^j exp(+2 pi i l j / N), FP64, as the K-major operand rows
// (c_out, l) over K = (j, c_in): [[Wr, -Wi], [Wi, Wr]]
void dft_operand(int N, int jpad, int lblock, std::vector<uint16_t> &out) {
    const int kb = 2 * jpad / 64, nblk = N / lblock;
    const uint32_t tile = (uint32_t)(2 * lblock) * 128u;     // rows x 64 K fp16
    out.assign((size_t)nblk * kb * tile / 2, 0);
    for (int b = 0; b < nblk; b++)
        for (int co = 0; co < 2; co++)
            for (int li = 0; li < lblock; li++) {
                const int l = b * lblock + li, row = co * lblock + li;
                for (int j = 0; j < jpad; j++) {
                    const double ang = 2.0 * M_PI * (double)(((long long)l * j) % N) / (double)N;
                    const double sg = (j & 1) ? -1.0 : 1.0;
                    const double wr = sg * cos(ang), wi = sg * sin(ang);
                    for (int ci = 0; ci < 2; ci++) {
                        const double v = co == 0 ? (ci == 0 ? wr : -wi) : (ci == 0 ? wi : wr);
                        const int k = 2 * j + ci;
                        const size_t off = ((size_t)b * kb + k / 64) * tile + tc::off_kmajor(row, k % 64, kKBytes, kKMN);
                        const __half h = __float2half_rn((float)v);
                        out[off / 2] = *reinterpret_cast<const uint16_t *>(&h);
                    }
                }
            }
}

}  // namespace

bool epic_big_supported(const hai_layout *L) {
    return (L->grid_n == 256 || L->grid_n == 512) && L->n_pol == 2 && L->box_w <= L->grid_n / 2 &&
           L->box_h <= std::min(128, L->grid_n / 2);
}

// Per layout: the two DFT operands and the batch scratch (A1 and A2).
hai_status epic_big_prepare(hai_layout *L) {
    if (!epic_big_supported(L)) return HAI_OK;
    const BigGeo g = big_geo(L);
    std::vector<uint16_t> b1, b2;
    dft_operand(g.N, g.kb1 * 32, 128, b1);
    dft_operand(g.N, g.yb * 128, 64, b2);
    const size_t per_ct = (size_t)g.P * g.yb * g.kb1 * kTile16 + (size_t)g.lb2 * g.kb2 * kTile16;
    const size_t budget = (size_t)512 << 20;
    L->big_batch = (long long)std::max<size_t>(1, budget / per_ct);
    const size_t a1 = (size_t)L->big_batch * g.P * g.yb * g.kb1 * kTile16;
    const size_t a2 = (size_t)L->big_batch * g.lb2 * g.kb2 * kTile16;
    cudaError_t e = cudaMalloc(&L->d_big, b1.size() * 2 + b2.size() * 2 + a1 + a2);
    if (e != cudaSuccess) return hai_cuda_fail(e, "epic fp16 (large grid): scratch");
    uint8_t *base = static_cast<uint8_t *>(L->d_big);
    L->big_b1 = base;
    L->big_b2 = base + b1.size() * 2;
    L->big_a1 = base + b1.size() * 2 + b2.size() * 2;
    L->big_a2 = static_cast<uint8_t *>(L->big_a1) + a1;
    e = cudaMemcpy(L->big_b1, b1.data(), b1.size() * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L->big_b2, b2.data(), b2.size() * 2, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return hai_cuda_fail(e, "epic fp16 (large grid): DFT operands");
    return HAI_OK;
}

hai_status epic_big_launch(const hai_layout *L, const int8_t *volt, int C, int T, float *img, int accumulate,
                           cudaStream_t st) {
    if (!epic_big_supported(L) || !L->d_big)
        return hai_fail(HAI_ERR_UNSUPPORTED, "epic fp16: large-grid tensor path needs N = 256 or 512, 2 pols, "
                                             "a box <= N/2");
    hai_ctx *ctx = L->ctx;
    const BigGeo g = big_geo(L);
    if (g.kb2 != kS2Kb) return hai_fail(HAI_ERR_UNSUPPORTED, "epic fp16 (large grid): box taller than 128 cells");
    const size_t s1_smem = (size_t)kS1Stages * (kTile16 + kTile32);
    const size_t s2_smem = (size_t)3 * g.kb2 * kTile16;
    if (s1_smem > (size_t)ctx->smem_optin - 2048 || s2_smem > (size_t)ctx->smem_optin - 2048)
        return hai_fail(HAI_ERR_UNSUPPORTED, "epic fp16 (large grid): shared memory");
    HAI_CUDA_TRY(cudaFuncSetAttribute(big_s1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1_smem));
    HAI_CUDA_TRY(cudaFuncSetAttribute(big_s2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s2_smem));
    const long long total = (long long)C * T;
    const int pidx = prof_begin(ctx, st);
    for (long long b0 = 0; b0 < total; b0 += L->big_batch) {
        const long long b1 = std::min(total, b0 + L->big_batch);
        const long long nfield = (b1 - b0) * g.P;
        const int ncell = (g.kb1 * 32) * (g.yb * 128);
        big_grid_kernel<<<dim3((ncell + 255) / 256, (unsigned)((nfield + kGridFields - 1) / kGridFields)), 256, 0,
                          st>>>(volt, L->n_elem, L->d_cell_start, L->d_entry_elem, L->d_entry_w, g, b0, nfield,
                                static_cast<uint8_t *>(L->big_a1));
        S1Params p1;
        p1.a1 = static_cast<const uint8_t *>(L->big_a1);
        p1.b1 = static_cast<const uint8_t *>(L->big_b1);
        p1.a2 = static_cast<uint8_t *>(L->big_a2);
        p1.g = g;
        p1.b0 = b0;
        p1.nfield = nfield;
        p1.ntiles = nfield * g.yb * g.lb1;
        p1.status = ctx->d_status;
        big_s1_kernel<<<(unsigned)std::min<long long>(p1.ntiles, ctx->num_sms), 384, s1_smem, st>>>(p1);
        S2Params p2;
        p2.a2 = static_cast<const uint8_t *>(L->big_a2);
        p2.b2 = static_cast<const uint8_t *>(L->big_b2);
        p2.img = img;
        p2.g = g;
        p2.b0 = b0;
        p2.b1 = b1;
        p2.T = T;
        p2.c_first = (int)(b0 / T);
        const int c_last = (int)((b1 - 1) / T);
        p2.n_items = (c_last - p2.c_first + 1) * g.lb2 * g.lb2;
        p2.accumulate = accumulate;
        p2.status = ctx->d_status;
        big_s2_kernel<<<(unsigned)std::min(p2.n_items, ctx->num_sms), kS2Threads, s2_smem, st>>>(p2);
        prof_count(ctx, 3);
    }
    prof_end(ctx, pidx, st);
    HAI_CUDA_TRY(cudaGetLastError());
    return HAI_OK;
}
