// EPIC on tcgen05 tensor cores for large grids (N = 256, 512): Eq.
// intra-station EPIC, then the squaring and temporal sum of Eq. intra-station
// squaring, with 16-bit operands (FP16 or BF16, optionally split into hi + lo
// parts whose products hi*hi + hi*lo + lo*hi reach ~FP32 accuracy) and FP32
// accumulation.
//
// The 2D DFT of the kernel's bounding box (<= N/2 x N/2 cells, at the
// transform's origin; the shift by the box corner is a phase common to both
// polarisations and cancels in every product) is two dense complex products
// with W'[j][l] = (-1)^j exp(+2 pi i l j / N) (the (-1)^j puts the phase
// centre at pixel N/2), written as real GEMMs.  A grid of 512^2 does not fit
// one SM, so the stages run as kernels per batch through an HBM scratch.  A
// batch is a block of samples [t0, t1) of every channel, so that a long
// cadence of few channels still gives stage 2 work for every SM:
//   grid:   every field (channel, sample, pol) gathered into its box (FP32
//           sums of conj(W~) E, stored as 16-bit (hi, lo) values; one thread per
//           cell and 8 fields), K-major in the tensor cores' tile order:
//           A1[field][k block] = 128 rows y x 64 (x, re/im);
//   stage1: H[y][l_x] = sum_x G[y][x] W'[x][l_x]: persistent CTAs over
//           contiguous ranges of (l_x block, field) tiles, the l_x block's DFT
//           operand resident in shared memory, A1 streamed by bulk copies,
//           tcgen05.mma M = 128 (y), N = 2 W1 (re, im of W1 l_x), accumulator
//           double-buffered in TMEM; the epilogue stores H (16-bit),
//           transposed, into the stage-2 operand:
//           A2[channel, sample][64-wide l_x block][k block] = MN-major tiles
//           of 128 rows (l_x, pol) x 64 (y, re/im);
//   stage2: F[l_y][l_x] = sum_y W'[y][l_y] H[y][l_x] for a 64 x W2 pixel
//           tile of one channel: an item is (l_y block, channel, l_x block);
//           persistent CTAs take contiguous ranges of (item, sample) units, so
//           every CTA gets the same number of samples; the l_y block's DFT
//           operand stays resident while the CTA's items share it, A2 is
//           streamed per k block, M = 128 (l_x, pol), N = 2 W2 (re, im of W2
//           l_y); sixteen epilogue warps add |F_X|^2, |F_Y|^2 and F_X conj(F_Y)
//           into registers over the samples.  The CTA holding an item's first
//           sample writes (or adds to) the image tile; a CTA whose range begins
//           inside an item writes its partial tile to its own slot, and
//   fixup:  adds the slots of every split item to the image in CTA order
//           (deterministic: the same order on every run).
// W1 = W2 = 128 (MMA N = 256) for plain operands, 64 (N = 128) for split ones
// (the hi and lo DFT operands then fit shared memory together).
#include <cuda_bf16.h>
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
constexpr uint32_t kTile16 = 16384;      // 128 rows x 64 K x 2 bytes
constexpr int kKb2 = 4;                  // k blocks of stage 2 (box rows padded to 128: 2 x 128 / 64)
constexpr int kMaxKb1 = 4;               // k blocks of stage 1 (box <= 128 columns)

struct BigGeo {
    int N, P, bx, by;            // grid, pols, box (cells)
    int kb1;                     // k blocks of stage 1: 2 bx_pad / 64
    int lb2;                     // 64-wide l_x blocks: N / 64
};

// Per-variant constants of the two GEMM kernels.
template <bool SP>
struct Var {
    static constexpr int W = SP ? 64 : 128;             // l values per tile (both stages)
    static constexpr int NM = 2 * W;                     // MMA N (re, im)
    static constexpr int Parts = SP ? 2 : 1;             // operand parts (hi, lo)
    static constexpr uint32_t BTile = (uint32_t)NM * 128u;   // one k block of a DFT operand part
    static constexpr int S1Stages = SP ? 3 : 4;
    static constexpr int S2Stages = SP ? 3 : 6;
    static constexpr uint32_t AStage = kTile16 * Parts;      // one k block of A (all parts)
    static constexpr uint32_t S1Smem = (uint32_t)kMaxKb1 * BTile * Parts + S1Stages * AStage;
    static constexpr uint32_t S2Smem = (uint32_t)kKb2 * BTile * Parts + S2Stages * AStage;
    static constexpr uint32_t TmemCols = 2 * NM;         // double-buffered accumulator
    static constexpr int Ly = W / 4;                     // l_y per stage-2 epilogue thread
    static constexpr int SlotFloats = 4 * W * 64;        // one partial pixel tile
};

// ------------------------------------------------------------------ grid
// one thread per (cell of the padded box, row-major; group of kGridFields
// fields): the cell's entries are read once for the group and the fields'
// voltage loads are independent, so they are in flight together.  Field f of
// the batch is (c, t0 + s, pol) with f = (c tb + s) P + pol.
constexpr int kGridFields = 8;

template <bool BF, bool SP>
__global__ void __launch_bounds__(256) big_grid_kernel(const int8_t *__restrict__ volt, int ne, int T,
                                                       const int32_t *__restrict__ cell_start,
                                                       const int32_t *__restrict__ entry_elem,
                                                       const float2 *__restrict__ entry_w, BigGeo g, int t0,
                                                       int tb, long long nfield, uint8_t *__restrict__ a1,
                                                       uint8_t *__restrict__ a1lo) {
    const int bxp = g.kb1 * 32, byp = 128;
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
    const char2 *E[kGridFields];
#pragma unroll
    for (int j = 0; j < kGridFields; j++) {
        const long long f = f0 + (j < nf ? j : 0);
        const long long ct = f / g.P;
        const int pol = (int)(f % g.P);
        const long long c = ct / tb, t = t0 + ct % tb;
        E[j] = reinterpret_cast<const char2 *>(volt) + ((c * T + t) * g.P + pol) * (long long)ne;
    }
    float2 acc[kGridFields];
#pragma unroll
    for (int j = 0; j < kGridFields; j++) acc[j] = make_float2(0.f, 0.f);
    for (int k = k0; k < k1; k++) {
        const int e = entry_elem[k];
        const float2 w = entry_w[k];                           // conj(W~)
        char2 v[kGridFields];
#pragma unroll
        for (int j = 0; j < kGridFields; j++) v[j] = j < nf ? E[j][e] : make_char2(0, 0);
#pragma unroll
        for (int j = 0; j < kGridFields; j++) {
            acc[j].x = fmaf(w.x, (float)v[j].x, fmaf(-w.y, (float)v[j].y, acc[j].x));
            acc[j].y = fmaf(w.x, (float)v[j].y, fmaf(w.y, (float)v[j].x, acc[j].y));
        }
    }
    const int k = 2 * x;
    const size_t field_bytes = (size_t)g.kb1 * kTile16;
    const size_t off = (size_t)f0 * field_bytes + (size_t)(k / 64) * kTile16 + tc::off_kmajor(y, k % 64, kKBytes, kKMN);
#pragma unroll
    for (int j = 0; j < kGridFields; j++)
        if (j < nf) {
            if constexpr (SP) {
                uint32_t hi, lo;
                tc::pack2_split<BF>(acc[j].x, acc[j].y, hi, lo);
                *reinterpret_cast<uint32_t *>(a1 + off + (size_t)j * field_bytes) = hi;
                *reinterpret_cast<uint32_t *>(a1lo + off + (size_t)j * field_bytes) = lo;
            } else {
                *reinterpret_cast<uint32_t *>(a1 + off + (size_t)j * field_bytes) = tc::pack2<BF>(acc[j].x, acc[j].y);
            }
        }
}

// The same gridding with the voltages staged in shared memory: one CTA per
// kGridFb consecutive fields (both polarisations of a sample) loads their N_e
// complex int8 voltages with 16-byte loads, then every thread builds whole
// 16-byte runs of A1 (4 cells of one row: 8 values) for each field, eight
// consecutive threads covering the 128 contiguous bytes of one k group of 8
// rows.  The 4 cells' gather entries are contiguous in the table, read four at
// a time with independent loads and shared by the CTA's fields.  Used when the
// fields fit (kGridSmemMax bytes).
constexpr int kGridThreads = 512;
constexpr int kGridSmemMax = 96 * 1024;
constexpr int kGridFb = 2;

// 32-bit words of one field's voltages in shared memory: ne words hold the
// 2 ne bytes twice over (one word per element pair, rounded up), plus 2 pad
// words per 32; kept even so that 8-byte stores stay aligned.
__host__ __device__ __forceinline__ int gridw_padded(int ne) {
    const int w = (ne + 1) / 2;
    return ((w + 2 * ((w + 31) >> 5)) + 1) & ~1;
}

template <bool BF, bool SP>
__global__ void __launch_bounds__(kGridThreads) big_grid_smem_kernel(
    const int8_t *__restrict__ volt, int ne, int T, const int32_t *__restrict__ cell_start,
    const int32_t *__restrict__ entry_elem, const float2 *__restrict__ entry_w, BigGeo g, int t0, int tb,
    long long nfield, uint8_t *__restrict__ a1, uint8_t *__restrict__ a1lo) {
    // voltages in shared memory with 2 pad words after every 32 (word w at
    // w + 2 (w >> 5)): rows of a lattice 64 words apart then fall on
    // different banks
    extern __shared__ __align__(16) uint32_t sw[];          // [kGridFb][padded words]
    const long long f0 = (long long)blockIdx.x * kGridFb;
    const int nf = (int)(nfield - f0 < kGridFb ? nfield - f0 : kGridFb);
    const int nwp = gridw_padded(ne);
    for (int j = 0; j < nf; j++) {
        const long long f = f0 + j;
        const long long ct = f / g.P;
        const int pol = (int)(f % g.P);
        const long long c = ct / tb, t = t0 + ct % tb;
        const int8_t *src = volt + ((c * T + t) * g.P + pol) * (long long)ne * 2;
        uint32_t *dst = sw + (size_t)j * nwp;
        if ((reinterpret_cast<uintptr_t>(src) & 7) == 0 && (ne & 3) == 0) {
            // 8-byte loads (two words), eight in flight per thread
            const uint2 *s2 = reinterpret_cast<const uint2 *>(src);
            const int n2 = ne / 4;
            for (int i0 = threadIdx.x; i0 < n2; i0 += 8 * kGridThreads) {
                uint2 v[8];
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    const int i = i0 + u * kGridThreads;
                    v[u] = i < n2 ? __ldg(s2 + i) : make_uint2(0u, 0u);
                }
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    const int i = i0 + u * kGridThreads;
                    if (i < n2) {
                        const int w = 2 * i;
                        *reinterpret_cast<uint2 *>(dst + w + 2 * (w >> 5)) = v[u];
                    }
                }
            }
        } else {
            const char2 *s2 = reinterpret_cast<const char2 *>(src);
            char2 *d2 = reinterpret_cast<char2 *>(dst);
            for (int e = threadIdx.x; e < ne; e += blockDim.x) {
                const int w = e >> 1;
                d2[2 * (w + 2 * (w >> 5)) + (e & 1)] = s2[e];
            }
        }
    }
    __syncthreads();
    const char2 *sv = reinterpret_cast<const char2 *>(sw);
    const int nkg = g.kb1 * 8;                       // k groups (4 cells each) per row
    const int nchunk = 128 * nkg;
    const size_t field_bytes = (size_t)g.kb1 * kTile16;
    for (int q = threadIdx.x; q < nchunk; q += blockDim.x) {
        const int y = (q & 7) + 8 * (q / (8 * nkg)), kg = (q >> 3) % nkg;
        const int x0 = 4 * kg;
        float2 acc[kGridFb][4];
#pragma unroll
        for (int j = 0; j < kGridFb; j++)
#pragma unroll
            for (int i = 0; i < 4; i++) acc[j][i] = make_float2(0.f, 0.f);
        if (y < g.by && x0 < g.bx) {
            // entries of cells x0 .. x0+3 (those inside the box): [cs[0], cs[4])
            const int cell0 = y * g.bx + x0;
            int cs[5];
#pragma unroll
            for (int i = 0; i < 5; i++) cs[i] = cell_start[cell0 + min(i, g.bx - x0)];
            for (int k = cs[0]; k < cs[4]; k += 4) {
                int e[4];
                float2 w[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const bool ok = k + u < cs[4];
                    e[u] = ok ? entry_elem[k + u] : 0;
                    w[u] = ok ? entry_w[k + u] : make_float2(0.f, 0.f);     // conj(W~); 0 past the end
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int kk = k + u;
                    const int ci = (kk >= cs[1]) + (kk >= cs[2]) + (kk >= cs[3]);
#pragma unroll
                    const int wd = e[u] >> 1;
                    const int pe = 2 * (wd + 2 * (wd >> 5)) + (e[u] & 1);   // padded char2 index
#pragma unroll
                    for (int j = 0; j < kGridFb; j++) {
                        const char2 v = sv[(size_t)j * 2 * nwp + pe];
#pragma unroll
                        for (int i = 0; i < 4; i++)
                            if (i == ci) {
                                acc[j][i].x = fmaf(w[u].x, (float)v.x, fmaf(-w[u].y, (float)v.y, acc[j][i].x));
                                acc[j][i].y = fmaf(w[u].x, (float)v.y, fmaf(w[u].y, (float)v.x, acc[j][i].y));
                            }
                    }
                }
            }
        }
        const size_t off = (size_t)(kg >> 3) * kTile16 + (size_t)(y >> 3) * kKMN + (size_t)(kg & 7) * kKBytes +
                           (size_t)(y & 7) * 16;
#pragma unroll
        for (int j = 0; j < kGridFb; j++) {
            if (j >= nf) break;
            uint8_t *dst = a1 + (size_t)(f0 + j) * field_bytes + off;
            if constexpr (SP) {
                uint4 hi, lo;
                tc::pack2_split<BF>(acc[j][0].x, acc[j][0].y, hi.x, lo.x);
                tc::pack2_split<BF>(acc[j][1].x, acc[j][1].y, hi.y, lo.y);
                tc::pack2_split<BF>(acc[j][2].x, acc[j][2].y, hi.z, lo.z);
                tc::pack2_split<BF>(acc[j][3].x, acc[j][3].y, hi.w, lo.w);
                *reinterpret_cast<uint4 *>(dst) = hi;
                *reinterpret_cast<uint4 *>(a1lo + (size_t)(f0 + j) * field_bytes + off) = lo;
            } else {
                *reinterpret_cast<uint4 *>(dst) =
                    make_uint4(tc::pack2<BF>(acc[j][0].x, acc[j][0].y), tc::pack2<BF>(acc[j][1].x, acc[j][1].y),
                               tc::pack2<BF>(acc[j][2].x, acc[j][2].y), tc::pack2<BF>(acc[j][3].x, acc[j][3].y));
            }
        }
    }
}

// Gridding for layouts whose cells each hold at most one gather entry (a
// lattice of elements on cells, 1 x 1 taps): a dense per-cell table of the
// padded box (element or -1, conj(W~)) replaces the CSR walk, so a 4-cell run
// is three vector loads with no dependent chain.  Voltages staged as above.
template <bool BF, bool SP>
__global__ void __launch_bounds__(kGridThreads) big_grid_dense_kernel(
    const int8_t *__restrict__ volt, int ne, int T, const int4 *__restrict__ cell_elem,
    const float4 *__restrict__ cell_w, BigGeo g, int t0, int tb, long long nfield, uint8_t *__restrict__ a1,
    uint8_t *__restrict__ a1lo) {
    extern __shared__ __align__(16) uint32_t sw[];          // [kGridFb][padded words]
    const long long f0 = (long long)blockIdx.x * kGridFb;
    const int nf = (int)(nfield - f0 < kGridFb ? nfield - f0 : kGridFb);
    const int nwp = gridw_padded(ne);
    for (int j = 0; j < nf; j++) {
        const long long f = f0 + j;
        const long long ct = f / g.P;
        const int pol = (int)(f % g.P);
        const long long c = ct / tb, t = t0 + ct % tb;
        const int8_t *src = volt + ((c * T + t) * g.P + pol) * (long long)ne * 2;
        uint32_t *dst = sw + (size_t)j * nwp;
        if ((reinterpret_cast<uintptr_t>(src) & 7) == 0 && (ne & 3) == 0) {
            const uint2 *s2 = reinterpret_cast<const uint2 *>(src);
            const int n2 = ne / 4;
            for (int i0 = threadIdx.x; i0 < n2; i0 += 8 * kGridThreads) {
                uint2 v[8];
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    const int i = i0 + u * kGridThreads;
                    v[u] = i < n2 ? __ldg(s2 + i) : make_uint2(0u, 0u);
                }
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    const int i = i0 + u * kGridThreads;
                    if (i < n2) {
                        const int w = 2 * i;
                        *reinterpret_cast<uint2 *>(dst + w + 2 * (w >> 5)) = v[u];
                    }
                }
            }
        } else {
            const char2 *s2 = reinterpret_cast<const char2 *>(src);
            char2 *d2 = reinterpret_cast<char2 *>(dst);
            for (int e = threadIdx.x; e < ne; e += blockDim.x) {
                const int w = e >> 1;
                d2[2 * (w + 2 * (w >> 5)) + (e & 1)] = s2[e];
            }
        }
    }
    __syncthreads();
    const char2 *sv = reinterpret_cast<const char2 *>(sw);
    const int nkg = g.kb1 * 8;
    const int nchunk = 128 * nkg;
    const size_t field_bytes = (size_t)g.kb1 * kTile16;
    for (int q = threadIdx.x; q < nchunk; q += blockDim.x) {
        const int y = (q & 7) + 8 * (q / (8 * nkg)), kg = (q >> 3) % nkg;
        // the table is stored in this loop's run order q (4 cells 4 kg .. 4 kg + 3
        // of row y): a warp reads it contiguously
        const int4 el = cell_elem[q];
        const float4 w01 = cell_w[2 * q], w23 = cell_w[2 * q + 1];
        const int ev[4] = {el.x, el.y, el.z, el.w};
        const float2 wv[4] = {make_float2(w01.x, w01.y), make_float2(w01.z, w01.w), make_float2(w23.x, w23.y),
                              make_float2(w23.z, w23.w)};
        const size_t off = (size_t)(kg >> 3) * kTile16 + (size_t)(y >> 3) * kKMN + (size_t)(kg & 7) * kKBytes +
                           (size_t)(y & 7) * 16;
#pragma unroll
        for (int j = 0; j < kGridFb; j++) {
            if (j >= nf) break;
            float2 acc[4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                acc[i] = make_float2(0.f, 0.f);
                if (ev[i] >= 0) {
                    const int wd = ev[i] >> 1;
                    const char2 v = sv[(size_t)j * 2 * nwp + 2 * (wd + 2 * (wd >> 5)) + (ev[i] & 1)];
                    acc[i].x = fmaf(wv[i].x, (float)v.x, -wv[i].y * (float)v.y);
                    acc[i].y = fmaf(wv[i].x, (float)v.y, wv[i].y * (float)v.x);
                }
            }
            uint8_t *dst = a1 + (size_t)(f0 + j) * field_bytes + off;
            if constexpr (SP) {
                uint4 hi, lo;
                tc::pack2_split<BF>(acc[0].x, acc[0].y, hi.x, lo.x);
                tc::pack2_split<BF>(acc[1].x, acc[1].y, hi.y, lo.y);
                tc::pack2_split<BF>(acc[2].x, acc[2].y, hi.z, lo.z);
                tc::pack2_split<BF>(acc[3].x, acc[3].y, hi.w, lo.w);
                *reinterpret_cast<uint4 *>(dst) = hi;
                *reinterpret_cast<uint4 *>(a1lo + (size_t)(f0 + j) * field_bytes + off) = lo;
            } else {
                *reinterpret_cast<uint4 *>(dst) =
                    make_uint4(tc::pack2<BF>(acc[0].x, acc[0].y), tc::pack2<BF>(acc[1].x, acc[1].y),
                               tc::pack2<BF>(acc[2].x, acc[2].y), tc::pack2<BF>(acc[3].x, acc[3].y));
            }
        }
    }
}

// ------------------------------------------------------------------ stage 1
struct S1Params {
    const uint8_t *a1, *a1lo;    // A1 (hi, lo)
    const uint8_t *b1, *b1lo;    // DFT operand (hi, lo): [l_x block][k block] tiles
    uint8_t *a2, *a2lo;          // stage-2 operand (hi, lo)
    BigGeo g;
    long long nfield;            // fields in the batch
    long long ntiles;            // (l_x block, field) tiles
    unsigned *status;
};

constexpr int kS1Threads = 640;             // warp 0 loads, warp 1 MMA, warps 4-19 epilogue

template <bool BF, bool SP>
__global__ void __launch_bounds__(kS1Threads, 1) big_s1_kernel(const S1Params p) {
    using V = Var<SP>;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[V::S1Stages], empty[V::S1Stages], dfull[2], dempty[2], bfull;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const BigGeo g = p.g;
    constexpr uint32_t kIdesc = tc::idesc_f16_as(BF, 128, V::NM, 0, 0);
    const uint32_t bpart = (uint32_t)g.kb1 * V::BTile;                 // one DFT operand part of a block
    uint8_t *sB = smem;                                                 // [part][kb1][BTile]
    uint8_t *sA0 = smem + (size_t)kMaxKb1 * V::BTile * V::Parts;       // ring [stage][part][16 KB]
    if (tid == 0) {
        for (int s = 0; s < V::S1Stages; s++) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&dfull[b], 1);
            tc::mbar_init(&dempty[b], 16);              // one arrival per epilogue warp
        }
        tc::mbar_init(&bfull, 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc(&tslot, V::TmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tslot;
    const int lbs = g.N / V::W;
    const long long nf = p.nfield;
    // contiguous tile range of this CTA; tiles are (l_x block, field), field fastest
    const long long r0 = p.ntiles * blockIdx.x / gridDim.x, r1 = p.ntiles * (blockIdx.x + 1) / gridDim.x;
    if (warp == 0) {
        if (lane == 0) {
            long long gs = 0;
            int cur_lb = -1;
            for (long long tile = r0; tile < r1; tile++) {
                const int lb = (int)(tile / nf);
                const long long f = tile % nf;
                if (lb != cur_lb) {
                    // every MMA reading the old operand has completed once the
                    // previous tile's accumulator is full
                    const long long gt = tile - r0;
                    if (gt > 0) tc::mbar_wait(&dfull[(gt - 1) & 1], (uint32_t)(((gt - 1) >> 1) & 1), p.status);
                    tc::mbar_arrive_expect_tx(&bfull, bpart * V::Parts);
                    for (int part = 0; part < V::Parts; part++) {
                        const uint8_t *src = (part ? p.b1lo : p.b1) + (size_t)lb * bpart;
                        tc::bulk_g2s(sB + (size_t)part * kMaxKb1 * V::BTile, src, bpart, &bfull);
                    }
                    cur_lb = lb;
                }
                if (tile + 2 < r1) {                      // A1 of the tile two ahead into L2
                    const size_t pre = (size_t)((tile + 2) % nf) * g.kb1 * kTile16;
                    tc::bulk_prefetch_l2(p.a1 + pre, (uint32_t)g.kb1 * kTile16);
                    if constexpr (SP) tc::bulk_prefetch_l2(p.a1lo + pre, (uint32_t)g.kb1 * kTile16);
                }
                for (int kb = 0; kb < g.kb1; kb++, gs++) {
                    const int s = (int)(gs % V::S1Stages);
                    if (gs >= V::S1Stages)
                        tc::mbar_wait(&empty[s], (uint32_t)(((gs / V::S1Stages) - 1) & 1), p.status);
                    tc::mbar_arrive_expect_tx(&full[s], V::AStage);
                    const size_t off = ((size_t)f * g.kb1 + kb) * kTile16;
                    tc::bulk_g2s(sA0 + (size_t)s * V::AStage, p.a1 + off, kTile16, &full[s]);
                    if constexpr (SP) tc::bulk_g2s(sA0 + (size_t)s * V::AStage + kTile16, p.a1lo + off, kTile16, &full[s]);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            long long gs = 0;
            int cur_lb = -1;
            uint32_t bph = 0;
            for (long long tile = r0; tile < r1; tile++) {
                const long long gt = tile - r0;
                const int lb = (int)(tile / nf);
                if (lb != cur_lb) {
                    tc::mbar_wait(&bfull, bph & 1, p.status);
                    bph++;
                    cur_lb = lb;
                }
                const int b = (int)(gt & 1);
                if (gt >= 2) tc::mbar_wait(&dempty[b], (uint32_t)(((gt >> 1) - 1) & 1), p.status);
                tc::fence_after();
                const uint32_t d = tmem + (uint32_t)b * V::NM;
                for (int kb = 0; kb < g.kb1; kb++, gs++) {
                    const int s = (int)(gs % V::S1Stages);
                    // bulk-copied stage: no tcgen05 fence needed (see stage 2)
                    tc::mbar_wait(&full[s], (uint32_t)((gs / V::S1Stages) & 1), p.status);
                    const uint32_t a = tc::smem_u32(sA0 + (size_t)s * V::AStage);
                    const uint32_t bq = tc::smem_u32(sB + (size_t)kb * V::BTile);
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const uint32_t acc0 = (kb > 0 || j > 0) ? 1u : 0u;
                        const uint64_t da = tc::desc(a + j * 2 * kKBytes, kKBytes, kKMN);
                        const uint64_t db = tc::desc(bq + j * 2 * kKBytes, kKBytes, kKMN);
                        tc::mma_f16(d, da, db, kIdesc, acc0);
                        if constexpr (SP) {
                            const uint64_t dal = tc::desc(a + kTile16 + j * 2 * kKBytes, kKBytes, kKMN);
                            const uint64_t dbl = tc::desc(bq + kMaxKb1 * V::BTile + j * 2 * kKBytes, kKBytes, kKMN);
                            tc::mma_f16(d, da, dbl, kIdesc, 1u);
                            tc::mma_f16(d, dal, db, kIdesc, 1u);
                        }
                    }
                    tc::mma_commit(&empty[s]);
                }
                tc::mma_commit(&dfull[b]);
            }
        }
    } else if (warp >= 4) {
        // epilogue, warps 4-19: thread = row y of the tile and one quarter (h)
        // of its W1 l_x -> the stage-2 operand rows (l_x, pol), K index 2 y +
        // re/im
        const int q = warp & 3, y = q * 32 + lane, h = (warp - 4) >> 2;
        const int kb2 = (2 * y) / 64, kk = (2 * y) % 64;   // K of the real part; imag at kk + 1
        constexpr int kChunks = V::W / 64;                   // 16 l_x per chunk, per quarter
        long long gt = 0;
        for (long long tile = r0; tile < r1; tile++, gt++) {
            const int b = (int)(gt & 1);
            const int lb = (int)(tile / nf);
            const long long f = tile % nf;
            const int pol = (int)(f % g.P);
            const long long ct = f / g.P;                       // (c, s) of the batch
            // one lane of the warp waits, the warp follows (the wait's result
            // reaches the others through the warp barrier)
            if (lane == 0) tc::mbar_wait(&dfull[b], (uint32_t)((gt >> 1) & 1), p.status);
            __syncwarp();
            tc::fence_after();
#pragma unroll 1
            for (int ch = kChunks * h; ch < kChunks * h + kChunks; ch++) {
                uint32_t rr[16], ri[16];
                const uint32_t t0 = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)b * V::NM + (uint32_t)(16 * ch);
                tc::tmem_ld16(t0, rr);
                tc::tmem_ld16(t0 + V::W, ri);
                tc::tmem_wait_ld();
                const int lx = lb * V::W + 16 * ch;             // first l_x of the chunk
                const int lxb = lx / 64, lx64 = lx % 64;
                const size_t toff = (((size_t)ct * g.lb2 + lxb) * kKb2 + kb2) * kTile16;
                // rows (l_x, pol): m = (l_x >> 4) 32 + pol 16 + (l_x & 15)
                const int m0 = (lx64 >> 4) * 32 + pol * 16;
#pragma unroll
                for (int half = 0; half < 2; half++) {          // 8 l_x -> one 16-byte run per K value
                    uint32_t hr[4], hi[4], lr[4], li[4];
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const float a0 = __uint_as_float(rr[8 * half + 2 * e]), a1v = __uint_as_float(rr[8 * half + 2 * e + 1]);
                        const float b0 = __uint_as_float(ri[8 * half + 2 * e]), b1v = __uint_as_float(ri[8 * half + 2 * e + 1]);
                        if constexpr (SP) {
                            tc::pack2_split<BF>(a0, a1v, hr[e], lr[e]);
                            tc::pack2_split<BF>(b0, b1v, hi[e], li[e]);
                        } else {
                            hr[e] = tc::pack2<BF>(a0, a1v);
                            hi[e] = tc::pack2<BF>(b0, b1v);
                        }
                    }
                    // K values kk (re) and kk + 1 (im) are adjacent 16-byte rows of
                    // the MN-major tile (kk even): one 32-byte store
                    const int m = m0 + 8 * half;
                    const size_t o_r = toff + tc::off_mnmajor(m, kk, kMKs, kMMN);
                    tc::st_global_v8(p.a2 + o_r, make_uint4(hr[0], hr[1], hr[2], hr[3]), make_uint4(hi[0], hi[1], hi[2], hi[3]));
                    if constexpr (SP)
                        tc::st_global_v8(p.a2lo + o_r, make_uint4(lr[0], lr[1], lr[2], lr[3]),
                                         make_uint4(li[0], li[1], li[2], li[3]));
                }
            }
            // one arrival per warp once all its lanes' TMEM reads are done
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&dempty[b]);
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, V::TmemCols);
}

// ------------------------------------------------------------------ stage 2
struct S2Params {
    const uint8_t *a2, *a2lo;    // stage-2 operand (hi, lo) of the batch
    const uint8_t *b2, *b2lo;    // DFT operand (hi, lo): [l_y block][k block] tiles
    float *img;
    float *slots;                // one partial pixel tile per CTA
    BigGeo g;
    int C, tb;                   // channels, samples of the batch
    long long units;             // items x tb
    int add;                     // 1: the head part adds to the image (accumulate or a later batch)
    unsigned *status;
};

constexpr int kAhead = 4;                   // samples of L2 prefetch ahead of the stage-2 loads

// Unit range of CTA k of G over U units: [U k / G, U (k + 1) / G).
__host__ __device__ __forceinline__ long long unit_start(long long U, int G, int k) { return U * k / G; }

template <bool BF, bool SP>
__global__ void __launch_bounds__(576, 1) big_s2_kernel(const S2Params p) {
    using V = Var<SP>;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t bfull, afull[V::S2Stages], aempty[V::S2Stages], dfull[2], dempty[2];
    __shared__ uint32_t tslot;
    constexpr int kEpi = 512;                               // 16 epilogue warps
    constexpr uint32_t kIdesc = tc::idesc_f16_as(BF, 128, V::NM, 1, 0);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const BigGeo g = p.g;
    uint8_t *sB = smem;                                                  // [part][kb2][BTile]
    uint8_t *sA0 = smem + (size_t)kKb2 * V::BTile * V::Parts;           // ring [stage][part][16 KB]
    if (tid == 0) {
        tc::mbar_init(&bfull, 1);
        for (int s = 0; s < V::S2Stages; s++) {
            tc::mbar_init(&afull[s], 1);
            tc::mbar_init(&aempty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&dfull[b], 1);
            tc::mbar_init(&dempty[b], kEpi / 32);       // one arrival per epilogue warp
        }
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc(&tslot, V::TmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tslot;
    const int per_lyb = p.C * g.lb2;                       // items per l_y block
    const int tb = p.tb;
    const long long u0 = unit_start(p.units, gridDim.x, blockIdx.x);
    const long long u1 = unit_start(p.units, gridDim.x, blockIdx.x + 1);
    const uint32_t bbytes = (uint32_t)kKb2 * V::BTile;     // one DFT operand part of an l_y block
    if (warp == 0) {
        if (lane == 0) {
            long long gs = 0, gk = 0;                      // samples and k blocks loaded
            int cur_lyb = -1;
            for (long long u = u0; u < u1;) {
                const long long it = u / tb;
                const int s0 = (int)(u % tb), s1 = (int)std::min<long long>(tb, s0 + (u1 - u));
                const int lyb = (int)(it / per_lyb), rem = (int)(it % per_lyb), c = rem / g.lb2, lxb = rem % g.lb2;
                if (lyb != cur_lyb) {
                    // every MMA reading the old operand has completed once the
                    // last sample's accumulator is full
                    if (gs > 0) tc::mbar_wait(&dfull[(gs - 1) & 1], (uint32_t)(((gs - 1) >> 1) & 1), p.status);
                    tc::mbar_arrive_expect_tx(&bfull, bbytes * V::Parts);
                    for (int part = 0; part < V::Parts; part++)
                        tc::bulk_g2s(sB + (size_t)part * bbytes, (part ? p.b2lo : p.b2) + (size_t)lyb * bbytes, bbytes,
                                     &bfull);
                    cur_lyb = lyb;
                }
                for (int s = s0; s < s1; s++, gs++) {
                    const size_t base = (((size_t)c * tb + s) * g.lb2 + lxb) * kKb2 * kTile16;
                    // the operand of a sample kAhead ahead into L2 (the ring holds ~1.5 samples)
                    if (s + kAhead < s1) {
                        const size_t pre = base + (size_t)kAhead * g.lb2 * kKb2 * kTile16;
                        tc::bulk_prefetch_l2(p.a2 + pre, kKb2 * kTile16);
                        if constexpr (SP) tc::bulk_prefetch_l2(p.a2lo + pre, kKb2 * kTile16);
                    }
                    for (int kb = 0; kb < kKb2; kb++, gk++) {
                        const int st = (int)(gk % V::S2Stages);
                        if (gk >= V::S2Stages)
                            tc::mbar_wait(&aempty[st], (uint32_t)(((gk / V::S2Stages) - 1) & 1), p.status);
                        tc::mbar_arrive_expect_tx(&afull[st], V::AStage);
                        tc::bulk_g2s(sA0 + (size_t)st * V::AStage, p.a2 + base + (size_t)kb * kTile16, kTile16, &afull[st]);
                        if constexpr (SP)
                            tc::bulk_g2s(sA0 + (size_t)st * V::AStage + kTile16, p.a2lo + base + (size_t)kb * kTile16,
                                         kTile16, &afull[st]);
                    }
                }
                u += s1 - s0;
            }
        }
    } else if (warp == 1) {
        // one thread issues the MMAs: per k block 4 K-steps (x 3 products when
        // split), one commit per k block (frees the A stage) and one per sample
        // (fills the accumulator)
        if (lane == 0) {
            long long gs = 0, gk = 0;
            int cur_lyb = -1;
            uint32_t bph = 0;
            const uint32_t sb0 = tc::smem_u32(sB), sa0 = tc::smem_u32(sA0);
            for (long long u = u0; u < u1;) {
                const long long it = u / tb;
                const int s0 = (int)(u % tb), s1 = (int)std::min<long long>(tb, s0 + (u1 - u));
                const int lyb = (int)(it / per_lyb);
                if (lyb != cur_lyb) {
                    tc::mbar_wait(&bfull, bph & 1, p.status);
                    bph++;
                    cur_lyb = lyb;
                }
                for (int s = s0; s < s1; s++, gs++) {
                    const int b = (int)(gs & 1);
                    if (gs >= 2) tc::mbar_wait(&dempty[b], (uint32_t)(((gs >> 1) - 1) & 1), p.status);
                    tc::fence_after();
                    const uint32_t d = tmem + (uint32_t)b * V::NM;
                    for (int kb = 0; kb < kKb2; kb++, gk++) {
                        const int st = (int)(gk % V::S2Stages);
                        // a stage filled by bulk copies (async proxy, completed on the
                        // mbarrier) needs no tcgen05 fence before the MMAs read it; the
                        // fence above orders them after the epilogue's TMEM reads
                        tc::mbar_wait(&afull[st], (uint32_t)((gk / V::S2Stages) & 1), p.status);
                        const uint32_t a = sa0 + (uint32_t)st * V::AStage;
                        const uint32_t bq = sb0 + (uint32_t)kb * V::BTile;
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            const uint32_t acc0 = (kb > 0 || j > 0) ? 1u : 0u;
                            const uint64_t da = tc::desc(a + j * 2 * kMKs, kMKs, kMMN);
                            const uint64_t db = tc::desc(bq + j * 2 * kKBytes, kKBytes, kKMN);
                            tc::mma_f16(d, da, db, kIdesc, acc0);
                            if constexpr (SP) {
                                const uint64_t dal = tc::desc(a + kTile16 + j * 2 * kMKs, kMKs, kMMN);
                                const uint64_t dbl = tc::desc(bq + bbytes + j * 2 * kKBytes, kKBytes, kKMN);
                                tc::mma_f16(d, da, dbl, kIdesc, 1u);
                                tc::mma_f16(d, dal, db, kIdesc, 1u);
                            }
                        }
                        tc::mma_commit(&aempty[st]);
                    }
                    tc::mma_commit(&dfull[b]);
                }
                u += s1 - s0;
            }
        }
    } else if (warp >= 2) {
        // epilogue, warps 2-17: thread row m = (l_x, pol) of TMEM lane
        // quadrant q, group h of Ly l_y values
        const int ew = warp - 2, q = warp & 3, h = ew >> 2;
        const int m = 32 * q + lane;
        const int pol = (m >> 4) & 1, kx = (m >> 5) * 16 + (m & 15);
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        constexpr int kLy = V::Ly;
        const size_t NN = (size_t)g.N * g.N;
        float2 acc_a[kLy / 2], acc_x[kLy / 2];
        long long gs = 0;
        for (long long u = u0; u < u1;) {
            const long long it = u / tb;
            const int s0 = (int)(u % tb), s1 = (int)std::min<long long>(tb, s0 + (u1 - u));
            const int lyb = (int)(it / per_lyb), rem = (int)(it % per_lyb), c = rem / g.lb2, lxb = rem % g.lb2;
#pragma unroll
            for (int t = 0; t < kLy / 2; t++) acc_a[t] = acc_x[t] = make_float2(0.f, 0.f);
            for (int s = s0; s < s1; s++, gs++) {
                const int b = (int)(gs & 1);
                if (lane == 0) tc::mbar_wait(&dfull[b], (uint32_t)((gs >> 1) & 1), p.status);
                __syncwarp();
                tc::fence_after();
                // 8 l_y at a time (re and im: 16 registers): the pixel pairs
                // (2k, 2k + 1) of the cross term stay inside each group
#pragma unroll
                for (int g8 = 0; g8 < kLy / 8; g8++) {
                    const uint32_t col = (uint32_t)b * V::NM + (uint32_t)(kLy * h + 8 * g8);
                    uint32_t rr[8], ri[8];
                    tc::tmem_ld8(tmem + lane_base + col, rr);
                    tc::tmem_ld8(tmem + lane_base + col + V::W, ri);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int k = 0; k < 8; k += 2) {
                        const float2 fr = make_float2(__uint_as_float(rr[k]), __uint_as_float(rr[k + 1]));
                        const float2 fi = make_float2(__uint_as_float(ri[k]), __uint_as_float(ri[k + 1]));
                        float2 &a = acc_a[(8 * g8 + k) >> 1];
                        a = __ffma2_rn(fr, fr, __ffma2_rn(fi, fi, a));
                    }
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        const float e_r = __uint_as_float(rr[2 * k]), e_i = __uint_as_float(ri[2 * k]);
                        const float o_r = __uint_as_float(rr[2 * k + 1]), o_i = __uint_as_float(ri[2 * k + 1]);
                        const float mr = pol ? o_r : e_r, mi = pol ? o_i : e_i;
                        const float sr = __shfl_xor_sync(0xffffffffu, pol ? e_r : o_r, 16);
                        const float si = __shfl_xor_sync(0xffffffffu, pol ? e_i : o_i, 16);
                        float2 &a = acc_x[4 * g8 + k];
                        a = __ffma2_rn(make_float2(mr, mi), make_float2(sr, sr),
                                       __ffma2_rn(make_float2(mi, -mr), make_float2(si, si), a));
                    }
                }
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&dempty[b]);
            }
            // the part's pixel tile: planes XX, YY, Re XY, Im XY of channel c,
            // to the image (the item's first sample is here) or to this CTA's slot
            const bool head = s0 == 0;
            float *dst;
            size_t rs, ps;
            bool add;
            if (head) {
                dst = p.img + (size_t)c * 4 * NN + (size_t)lyb * V::W * g.N + (size_t)lxb * 64;
                rs = g.N;
                ps = NN;
                add = p.add != 0;
            } else {
                dst = p.slots + (size_t)blockIdx.x * V::SlotFloats;
                rs = 64;
                ps = (size_t)V::W * 64;
                add = false;
            }
#pragma unroll
            for (int t = 0; t < kLy; t++) {
                float *d = dst + pol * ps + (size_t)(kLy * h + t) * rs + kx;
                float v = (t & 1) ? acc_a[t >> 1].y : acc_a[t >> 1].x;
                if (add) v += *d;
                *d = v;
            }
            const float sgn = pol ? -1.f : 1.f;
#pragma unroll
            for (int t = 0; t < kLy / 2; t++) {
                const int ly = kLy * h + 16 * (t >> 3) + 2 * (t & 7) + pol;
                float *d = dst + 2 * ps + (size_t)ly * rs + kx;
                float vr = acc_x[t].x, vi = sgn * acc_x[t].y;
                if (add) {
                    vr += d[0];
                    vi += d[ps];
                }
                d[0] = vr;
                d[ps] = vi;
            }
            u += s1 - s0;
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, V::TmemCols);
}

// ------------------------------------------------------------------ fixup
// Block (k, slice): if CTA k's range begins inside an item and CTA k - 1's
// range does not begin inside the same item, CTA k is that item's first
// partial: add the slots of k, k + 1, ... (every CTA whose range begins inside
// the item) to the item's image tile, in CTA order.  Each of kFixSlices blocks
// takes a slice of the tile, four elements per thread with independent loads.
constexpr int kFixSlices = 32;

template <int W>
__global__ void __launch_bounds__(256) big_fixup_kernel(const float *__restrict__ slots, float *__restrict__ img,
                                                        BigGeo g, int C, int tb, long long units, int G) {
    const int k = blockIdx.x;
    auto tail_item = [&](int j) -> long long {            // item whose middle CTA j's range begins in, or -1
        if (j <= 0 || j >= G) return -1;
        const long long a = unit_start(units, G, j), b = unit_start(units, G, j + 1);
        return (a < b && a % tb != 0) ? a / tb : -1;
    };
    const long long it = tail_item(k);
    if (it < 0 || tail_item(k - 1) == it) return;
    int k1 = k + 1;
    while (tail_item(k1) == it) k1++;
    const int per_lyb = C * g.lb2;
    const int lyb = (int)(it / per_lyb), rem = (int)(it % per_lyb), c = rem / g.lb2, lxb = rem % g.lb2;
    const size_t NN = (size_t)g.N * g.N;
    constexpr int kSlot = 4 * W * 64, kPer = kSlot / kFixSlices;      // elements per block
    static_assert(kPer == 4 * 256 || kPer == 2 * 256, "slice = 2 or 4 elements per thread");
    constexpr int kE = kPer / 256;
    float *dst = img + (size_t)c * 4 * NN + (size_t)lyb * W * g.N + (size_t)lxb * 64;
    size_t di[kE];
    float s[kE], v[kE];
#pragma unroll
    for (int i = 0; i < kE; i++) {
        const int e = blockIdx.y * kPer + i * 256 + threadIdx.x;
        const int plane = e / (W * 64), r = e % (W * 64), ly = r / 64, lx = r % 64;
        di[i] = plane * NN + (size_t)ly * g.N + lx;
        v[i] = dst[di[i]];
        s[i] = 0.f;
    }
    for (int j = k; j < k1; j++)
#pragma unroll
        for (int i = 0; i < kE; i++) s[i] += slots[(size_t)j * kSlot + blockIdx.y * kPer + i * 256 + threadIdx.x];
#pragma unroll
    for (int i = 0; i < kE; i++) dst[di[i]] = v[i] + s[i];
}

BigGeo big_geo(const hai_layout *L) {
    BigGeo g;
    g.N = L->grid_n;
    g.P = L->n_pol;
    g.bx = L->box_w;
    g.by = L->box_h;
    g.kb1 = (2 * g.bx + 63) / 64;
    g.lb2 = g.N / 64;
    return g;
}

// W'[j][l] = (-1)^j exp(+2 pi i l j / N), FP64, as the K-major operand rows
// (c_out, l) over K = (j, c_in): [[Wr, -Wi], [Wi, Wr]], in blocks of `lblock`
// l values, rounded to FP16 or BF16 (part 0) or the remainder after that
// rounding rounded again (part 1, the lo part of the split operand).
template <typename H>
uint16_t bits16(H h) {
    return *reinterpret_cast<const uint16_t *>(&h);
}

void dft_operand(int N, int jpad, int lblock, bool bf16, int part, std::vector<uint16_t> &out) {
    const int kb = 2 * jpad / 64, nblk = N / lblock;
    const uint32_t tile = (uint32_t)(2 * lblock) * 128u;     // rows x 64 K x 2 bytes
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
                        uint16_t h, r;
                        if (bf16) {
                            const __nv_bfloat16 hi = __float2bfloat16_rn((float)v);
                            h = bits16(hi);
                            r = bits16(__float2bfloat16_rn((float)(v - (double)__bfloat162float(hi))));
                        } else {
                            const __half hi = __float2half_rn((float)v);
                            h = bits16(hi);
                            r = bits16(__float2half_rn((float)(v - (double)__half2float(hi))));
                        }
                        out[off / 2] = part ? r : h;
                    }
                }
            }
}

// Index of the (bf16, split) variant: 0 fp16, 1 bf16, 2 fp16 split, 3 bf16 split.
int variant(hai_precision prec) {
    switch (prec) {
        case HAI_PREC_FP16: return 0;
        case HAI_PREC_BF16: return 1;
        case HAI_PREC_FP16_SPLIT: return 2;
        case HAI_PREC_BF16_SPLIT: return 3;
        default: return -1;
    }
}

template <bool BF, bool SP>
hai_status launch_variant(const hai_layout *L, const int8_t *volt, int C, int T, float *img, int accumulate,
                          cudaStream_t st) {
    using V = Var<SP>;
    hai_ctx *ctx = L->ctx;
    const BigGeo g = big_geo(L);
    const int vi = (BF ? 1 : 0) + (SP ? 2 : 0);
    if (V::S1Smem > (uint32_t)ctx->smem_optin - 1024 || V::S2Smem > (uint32_t)ctx->smem_optin - 1024)
        return hai_fail(HAI_ERR_UNSUPPORTED, "epic tensor cores (large grid): shared memory");
    HAI_CUDA_TRY(hai_allow_dyn_smem(big_grid_smem_kernel<BF, SP>, ctx->smem_optin));
    HAI_CUDA_TRY(hai_allow_dyn_smem(big_grid_dense_kernel<BF, SP>, ctx->smem_optin));
    HAI_CUDA_TRY(hai_allow_dyn_smem(big_s1_kernel<BF, SP>, ctx->smem_optin));
    HAI_CUDA_TRY(hai_allow_dyn_smem(big_s2_kernel<BF, SP>, ctx->smem_optin));
    // the scratch holds big_batch (channel, sample) pairs of plain operands,
    // half as many split ones: channels in chunks of at most that many, and
    // per chunk batches of as many samples of every channel as fit
    const long long pairs = std::max<long long>(1, L->big_batch / V::Parts);
    int cb_max = (int)std::min<long long>(C, pairs);
    if (L->big_chunk > 0) cb_max = std::min(cb_max, L->big_chunk);          // the autotuner's choice
    const size_t a1_bytes = (size_t)L->big_batch * g.P * g.kb1 * kTile16;   // plain capacity of A1 (hi + lo when split)
    uint8_t *a1 = static_cast<uint8_t *>(L->big_a1), *a2 = static_cast<uint8_t *>(L->big_a2);
    const size_t a1_half = a1_bytes / 2, a2_half = (size_t)L->big_batch * g.lb2 * kKb2 * kTile16 / 2;
    uint8_t *a1lo = SP ? a1 + a1_half : nullptr, *a2lo = SP ? a2 + a2_half : nullptr;
    const int G1 = ctx->num_sms, G2 = ctx->num_sms;
    int launches = 0;
    // the fixup of a batch runs on the layout's second stream beside the next
    // batch's gridding and stage 1; the next stage 2 (which rewrites the
    // slots and adds to the image tiles) and the return wait for it
    bool fix_pending = false;
    const size_t NN = (size_t)g.N * g.N;
    for (int c0 = 0; c0 < C; c0 += cb_max) {
    const int Cc = std::min(cb_max, C - c0);
    const int8_t *vc = volt + (size_t)c0 * T * g.P * L->n_elem * 2;
    float *ic = img + (size_t)c0 * 4 * NN;
    const int tb_max = (int)std::max<long long>(1, std::min<long long>(T, pairs / Cc));
    for (int t0 = 0; t0 < T; t0 += tb_max) {
        const int tb = std::min(tb_max, T - t0);
        const long long nfield = (long long)Cc * tb * g.P;
        const int ncell = (g.kb1 * 32) * 128;
        const size_t vbytes = (size_t)kGridFb * 4 * gridw_padded(L->n_elem);
        if (vbytes <= (size_t)kGridSmemMax && L->big_cell)
            big_grid_dense_kernel<BF, SP><<<(unsigned)((nfield + kGridFb - 1) / kGridFb), kGridThreads, vbytes, st>>>(
                vc, L->n_elem, T, static_cast<const int4 *>(L->big_cell),
                reinterpret_cast<const float4 *>(static_cast<const uint8_t *>(L->big_cell) + L->big_cell_w_off), g, t0,
                tb, nfield, a1, a1lo);
        else if (vbytes <= (size_t)kGridSmemMax)
            big_grid_smem_kernel<BF, SP><<<(unsigned)((nfield + kGridFb - 1) / kGridFb), kGridThreads, vbytes, st>>>(
                vc, L->n_elem, T, L->d_cell_start, L->d_entry_elem, L->d_entry_w, g, t0, tb, nfield, a1, a1lo);
        else
            big_grid_kernel<BF, SP><<<dim3((ncell + 255) / 256, (unsigned)((nfield + kGridFields - 1) / kGridFields)),
                                      256, 0, st>>>(vc, L->n_elem, T, L->d_cell_start, L->d_entry_elem, L->d_entry_w, g,
                                                    t0, tb, nfield, a1, a1lo);
        S1Params p1;
        p1.a1 = a1;
        p1.a1lo = a1lo;
        p1.b1 = static_cast<const uint8_t *>(L->big_b1[vi][0]);
        p1.b1lo = static_cast<const uint8_t *>(L->big_b1[vi][1]);
        p1.a2 = a2;
        p1.a2lo = a2lo;
        p1.g = g;
        p1.nfield = nfield;
        p1.ntiles = nfield * (g.N / V::W);
        p1.status = ctx->d_status;
        big_s1_kernel<BF, SP><<<(unsigned)std::min<long long>(p1.ntiles, G1), kS1Threads, V::S1Smem, st>>>(p1);
        S2Params p2;
        p2.a2 = a2;
        p2.a2lo = a2lo;
        p2.b2 = static_cast<const uint8_t *>(L->big_b2[vi][0]);
        p2.b2lo = static_cast<const uint8_t *>(L->big_b2[vi][1]);
        p2.img = ic;
        p2.slots = static_cast<float *>(L->big_slots);
        p2.g = g;
        p2.C = Cc;
        p2.tb = tb;
        const long long items = (long long)(g.N / V::W) * Cc * g.lb2;
        p2.units = items * tb;
        p2.add = (accumulate || t0 > 0) ? 1 : 0;
        p2.status = ctx->d_status;
        const int G = (int)std::min<long long>(p2.units, G2);
        if (fix_pending) HAI_CUDA_TRY(cudaStreamWaitEvent(st, L->big_ev[1], 0));
        // the profiled (dominant) kernel of this path: every stage-2 launch
        const int pidx = prof_begin(ctx, st);
        big_s2_kernel<BF, SP><<<(unsigned)G, 576, V::S2Smem, st>>>(p2);
        prof_end(ctx, pidx, st);
        launches += 3;
        // items split between CTAs: their later parts were left in the slots
        bool split_items = false;
        for (int k = 1; k < G && !split_items; k++) {
            const long long a = unit_start(p2.units, G, k), b = unit_start(p2.units, G, k + 1);
            split_items = a < b && a % tb != 0;
        }
        if (split_items) {
            HAI_CUDA_TRY(cudaEventRecord(L->big_ev[0], st));
            HAI_CUDA_TRY(cudaStreamWaitEvent(L->big_stream, L->big_ev[0], 0));
            big_fixup_kernel<V::W><<<dim3((unsigned)G, kFixSlices), 256, 0, L->big_stream>>>(p2.slots, ic, g, Cc, tb,
                                                                                          p2.units, G);
            HAI_CUDA_TRY(cudaEventRecord(L->big_ev[1], L->big_stream));
            fix_pending = true;
            launches++;
        }
    }
    }
    if (fix_pending) HAI_CUDA_TRY(cudaStreamWaitEvent(st, L->big_ev[1], 0));
    prof_count(ctx, launches);
    HAI_CUDA_TRY(cudaGetLastError());
    return HAI_OK;
}

}  // namespace

// N = 128 runs here only with split operands (the 4-CTA cluster kernel
// holds one operand copy in shared memory); its box (<= 64 rows) is padded
// to the 128 rows of stage 2's K like every other box.
bool epic_big_supported(const hai_layout *L) {
    return (L->grid_n == 128 || L->grid_n == 256 || L->grid_n == 512) && L->n_pol == 2 &&
           L->box_w <= L->grid_n / 2 && L->box_h <= std::min(128, L->grid_n / 2);
}

bool epic_big_used(const hai_layout *L, hai_precision prec) {
    if (!epic_big_supported(L) || !L->d_big || prec == HAI_PREC_FP32) return false;
    return L->grid_n >= 256 || prec == HAI_PREC_FP16_SPLIT || prec == HAI_PREC_BF16_SPLIT;
}

// Per layout: the DFT operands of every variant (plain W = 128 blocks, split
// hi and lo W = 64 blocks, FP16 and BF16; at N = 128 the split ones only),
// the batch scratch (A1 and A2) and the partial-tile slots.
hai_status epic_big_prepare(hai_layout *L) {
    if (!epic_big_supported(L)) return HAI_OK;
    const BigGeo g = big_geo(L);
    const bool split_only = g.N == 128;
    std::vector<std::vector<uint16_t>> ops;          // [variant][stage][part]
    size_t op_bytes = 0;
    for (int vi = 0; vi < 4; vi++) {
        const bool bf = vi & 1, sp = vi >= 2;
        const int w = sp ? 64 : 128;
        for (int stage = 0; stage < 2; stage++)
            for (int part = 0; part < 2; part++) {
                ops.emplace_back();
                if ((part && !sp) || (split_only && !sp)) continue;
                dft_operand(g.N, stage == 0 ? g.kb1 * 32 : 128, w, bf, part, ops.back());
                op_bytes += (ops.back().size() * 2 + 1023) & ~(size_t)1023;
            }
    }
    // dense per-cell table of the padded box (128 rows x kb1 * 32 cells) when
    // every cell holds at most one gather entry
    std::vector<int32_t> cstart(g.bx * g.by + 1);
    std::vector<int32_t> celem;
    std::vector<float2> cw;
    bool dense = true;
    {
        cudaError_t e0 = cudaMemcpy(cstart.data(), L->d_cell_start, sizeof(int32_t) * cstart.size(), cudaMemcpyDeviceToHost);
        if (e0 != cudaSuccess) return hai_cuda_fail(e0, "epic tensor cores (large grid): gather table");
        for (int i = 0; i < g.bx * g.by && dense; i++) dense = cstart[i + 1] - cstart[i] <= 1;
        if (dense && L->nnz > 0) {
            celem.resize(L->nnz);
            cw.resize(L->nnz);
            e0 = cudaMemcpy(celem.data(), L->d_entry_elem, sizeof(int32_t) * L->nnz, cudaMemcpyDeviceToHost);
            if (e0 == cudaSuccess) e0 = cudaMemcpy(cw.data(), L->d_entry_w, sizeof(float2) * L->nnz, cudaMemcpyDeviceToHost);
            if (e0 != cudaSuccess) return hai_cuda_fail(e0, "epic tensor cores (large grid): gather table");
        }
    }
    const int bxp = g.kb1 * 32, ncellp = bxp * 128;
    std::vector<int32_t> dense_elem;
    std::vector<float2> dense_w;
    if (dense) {
        // in the gridding kernel's run order: run q = (y & 7) + 8 kg + 8 nkg (y >> 3)
        // holds cells 4 kg .. 4 kg + 3 of row y
        const int nkg = g.kb1 * 8;
        dense_elem.assign(ncellp, -1);
        dense_w.assign(ncellp, make_float2(0.f, 0.f));
        for (int q = 0; q < 128 * nkg; q++) {
            const int y = (q & 7) + 8 * (q / (8 * nkg)), kg = (q >> 3) % nkg;
            for (int i = 0; i < 4; i++) {
                const int x = 4 * kg + i;
                if (y >= g.by || x >= g.bx) continue;
                const int c = y * g.bx + x;
                if (cstart[c + 1] > cstart[c]) {
                    dense_elem[4 * q + i] = celem[cstart[c]];
                    dense_w[4 * q + i] = cw[cstart[c]];
                }
            }
        }
    }
    const size_t dense_bytes = dense ? (size_t)ncellp * (sizeof(int32_t) + sizeof(float2)) : 0;
    const size_t per_ct = (size_t)g.P * g.kb1 * kTile16 + (size_t)g.lb2 * kKb2 * kTile16;
    // 512 MB of scratch; 64 MB at N = 128 (a batch of ~170 split (channel,
    // sample) pairs, and the many small stations of an uneven array each hold one)
    const size_t budget = (size_t)(split_only ? 64 : 512) << 20;
    L->big_batch = (long long)std::max<size_t>(2, budget / per_ct) & ~1ll;    // even: halves hold hi and lo
    const size_t a1 = (size_t)L->big_batch * g.P * g.kb1 * kTile16;
    const size_t a2 = (size_t)L->big_batch * g.lb2 * kKb2 * kTile16;
    const size_t slots =
        (size_t)L->ctx->num_sms * (split_only ? Var<true>::SlotFloats : Var<false>::SlotFloats) * sizeof(float);
    cudaError_t e = cudaMalloc(&L->d_big, op_bytes + a1 + a2 + slots + dense_bytes);
    if (e != cudaSuccess) return hai_cuda_fail(e, "epic tensor cores (large grid): scratch");
    L->dev_bytes += op_bytes + a1 + a2 + slots + dense_bytes;
    uint8_t *base = static_cast<uint8_t *>(L->d_big);
    size_t off = 0;
    int idx = 0;
    for (int vi = 0; vi < 4; vi++)
        for (int stage = 0; stage < 2; stage++)
            for (int part = 0; part < 2; part++, idx++) {
                void *&dst = stage == 0 ? L->big_b1[vi][part] : L->big_b2[vi][part];
                dst = nullptr;
                if (ops[idx].empty()) continue;
                dst = base + off;
                e = cudaMemcpy(dst, ops[idx].data(), ops[idx].size() * 2, cudaMemcpyHostToDevice);
                if (e != cudaSuccess) return hai_cuda_fail(e, "epic tensor cores (large grid): DFT operands");
                off += (ops[idx].size() * 2 + 1023) & ~(size_t)1023;
            }
    L->big_a1 = base + off;
    L->big_a2 = base + off + a1;
    L->big_slots = base + off + a1 + a2;
    L->big_cell = nullptr;
    if (dense) {
        // [run][4] int32 elements, then [run][4] float2 weights (runs of 4 cells)
        uint8_t *d = base + off + a1 + a2 + slots;
        L->big_cell = d;
        L->big_cell_w_off = sizeof(int32_t) * (size_t)ncellp;
        e = cudaMemcpy(d, dense_elem.data(), sizeof(int32_t) * ncellp, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(d + L->big_cell_w_off, dense_w.data(), sizeof(float2) * ncellp, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return hai_cuda_fail(e, "epic tensor cores (large grid): cell table");
    }
    e = cudaStreamCreateWithFlags(&L->big_stream, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; i++) e = cudaEventCreateWithFlags(&L->big_ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return hai_cuda_fail(e, "epic tensor cores (large grid): fixup stream");
    return HAI_OK;
}

hai_status epic_big_launch(const hai_layout *L, const int8_t *volt, int C, int T, float *img, int accumulate,
                           hai_precision prec, cudaStream_t st) {
    if (!epic_big_used(L, prec))
        return hai_fail(HAI_ERR_UNSUPPORTED, "epic tensor cores: large-grid path needs N = 256 or 512 (or 128 with "
                                             "split operands), 2 pols, a box <= N/2 wide and <= 128 cells high");
    switch (variant(prec)) {
        case 0: return launch_variant<false, false>(L, volt, C, T, img, accumulate, st);
        case 1: return launch_variant<true, false>(L, volt, C, T, img, accumulate, st);
        case 2: return launch_variant<false, true>(L, volt, C, T, img, accumulate, st);
        case 3: return launch_variant<true, true>(L, volt, C, T, img, accumulate, st);
        default: return hai_fail(HAI_ERR_INVALID_ARG, "epic tensor cores (large grid): precision");
    }
}
