// EPIC direct imager on tcgen05 tensor cores for grid sides N = 32 and 64
// (Eq. intra-station EPIC, then the squaring and temporal sum of Eq.
// intra-station squaring), FP16 operands with FP32 accumulation in tensor
// memory.
//
// The 2D DFT of each gridded field is two dense complex products with a
// constant DFT matrix, written as real GEMMs (complex -> (re, im) pairs):
//   stage 1 (along x):  H[y][l_x] = sum_x G[y][x] W'[x][l_x]
//   stage 2 (along y):  F[l_y][l_x] = sum_y W'[y][l_y] H[y][l_x]
// with W'[j][l] = (-1)^j exp(+2 pi i l j / N).  Only the kernel's bounding
// box (<= N/2 x N/2 cells) is transformed, from the box origin: the shift by
// the box corner multiplies F by a phase common to both polarisations, which
// cancels in every F_a conj(F_b); the (-1)^j factor puts the phase centre at
// pixel (N/2, N/2).
//
// A step takes 128 / (N/2) fields (samples x 2 pols) so that stage 1 is one
// M = 128 product: rows (field, y), columns (re/im, l_x), contraction (x,
// re/im).  Stage 2 runs per "tile" of 128 rows (sample, l_x, pol) with the
// transposed stage-1 result as the MN-major operand A and the same DFT matrix
// as B; a tile holds one sample for N = 64 and two for N = 32.
//
// CTA = 16 warps, one CTA per SM, persistent over a contiguous range of the
// flattened (station, channel, sample) index:
//   warps 0-6  "front": re-pack the step's voltages (landed by TMA bulk
//              copies) as fp16 per element, gather-grid the step's fields
//              over tiles of the station's non-empty cells into A1 (fp16,
//              K-major) with FP32 sums; warps 0-3 then move stage-1 results
//              from TMEM into the stage-2 operand A2 (fp16, MN-major),
//              transposing on the way;
//   warp 7     one thread streams the voltages (TMA) and issues every MMA;
//   warps 8-15 epilogue: read stage-2 results from TMEM, add |F_X|^2,
//              |F_Y|^2 and F_X conj(F_Y) into register accumulators, and
//              write them out when a (station, channel) block ends.
// Every hand-off between the roles is an mbarrier phase.  TMEM: stage-1
// results double-buffered, stage-2 results in two tile slots, so the MMAs of
// one tile overlap the epilogue of the previous one.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "epic_tc.cuh"
#include "hai_internal.h"
#include "tc.cuh"

namespace {

constexpr int kThreads = 512;
constexpr int kFront = 224;             // warps 0-6
constexpr int kMmaWarp = 7;
constexpr int kEpi = 256;               // warps 8-15
constexpr int kStages = 4;              // voltage steps in flight
constexpr uint32_t kKs = 128;           // K-major operands: K-group stride
constexpr uint32_t kA2Ks = 2064;        // MN-major A2: K-group stride (16 groups + 16 B pad)
constexpr uint32_t kA2MNs = 128;        // MN-major A2: MN-group stride

template <int N, bool SP>
struct Geo {
    static constexpr int kSet = SP ? 2 : 1;            // operand copies: hi (and lo)
    static constexpr int kA2Steps = SP ? 1 : 2;        // stage-2 operand buffering (steps)
    static constexpr int kBox = N / 2;                 // box side
    static constexpr int kFields = 128 / kBox;         // fields per step: 4 or 8
    static constexpr int kSps = kFields / 2;           // samples per step: 2 or 4
    static constexpr int kTileSamples = 128 / (2 * N); // samples per stage-2 tile: 1 or 2
    static constexpr int kTiles = kSps / kTileSamples; // tiles per step
    static constexpr int kK = 2 * kBox;                // contraction of both stages: 64 or 32
    static constexpr int kNcol = 2 * N;                // MMA N of both stages: 128 or 64
    static constexpr int kU = kFields / 4;             // uint4 of fp16 voltages per element
    static constexpr int kLy = N / 2;                  // output rows per epilogue thread
    static constexpr uint32_t kMNs = (kK / 8) * kKs;   // K-major MN-group stride
    static constexpr uint32_t kBBytes = (kNcol / 8) * kMNs;
    static constexpr uint32_t kA1Bytes = 16 * kMNs;    // 128 rows
    static constexpr uint32_t kImgBytes = (kBox / 8) * kMNs;   // one field's rows
    static constexpr uint32_t kA2Bytes = (kK / 8) * kA2Ks;
    static constexpr uint32_t kOffA1 = kSet * kBBytes;                  // B hi [, B lo]
    static constexpr uint32_t kOffA2 = kOffA1 + 2 * kSet * kA1Bytes;    // A1 [2 buffers][hi, lo]
    static constexpr uint32_t kOffE = kOffA2 + kA2Steps * kTiles * kSet * kA2Bytes;
    static constexpr uint32_t kTmemCols = (4 * kNcol <= 256) ? 256 : 512;
    static_assert(kTiles == 2, "two stage-2 tiles per step");
};

struct Params {
    const int8_t *volt;
    float *img;
    const TcStation *stations;
    const uint8_t *dft;          // DFT operand B (K-major)
    const long long *cta_begin;
    long long len, total;
    int C, T;
    int ne_max;
    uint32_t vstage;
    int direct, accumulate, use_tma, guard;
    float *partials;
    unsigned *status;
};

__device__ __forceinline__ void bar_front() { asm volatile("bar.sync 1, 224;" ::: "memory"); }
__device__ __forceinline__ void bar_epi() { asm volatile("bar.sync 2, 256;" ::: "memory"); }

template <int N, bool SP, bool BF>
__global__ void __launch_bounds__(kThreads, 1) epic_tc_kernel(const Params p) {
    using G = Geo<N, SP>;
    // operand type of both MMA operands: FP16, or BF16 when BF
    constexpr uint32_t kIdesc1 = tc::idesc_f16_as(BF, 128, G::kNcol, 0, 0);
    constexpr uint32_t kIdesc2 = tc::idesc_f16_as(BF, 128, G::kNcol, 1, 0);
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mb_v[kStages];
    __shared__ __align__(8) uint64_t mb_a1[2], mb_d1[2], mb_a2[2], mb_full[2], mb_empty[2], mb_a2free;
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t *sB = smem;
    uint8_t *sA1 = smem + G::kOffA1;
    uint8_t *sA2 = smem + G::kOffA2;
    uint4 *sE = reinterpret_cast<uint4 *>(smem + G::kOffE);   // [2][ne_max][kU]
    const uint32_t off_v = G::kOffE + 2u * 16u * G::kU * p.ne_max;
    int8_t *sV = reinterpret_cast<int8_t *>(smem + off_v);
    uint8_t *sT = smem + off_v + kStages * p.vstage;         // the current station's gather table

    // ---- set-up: DFT operand, barriers, TMEM
    for (int i = tid; i < (int)(G::kSet * G::kBBytes / 16); i += kThreads)
        reinterpret_cast<int4 *>(sB)[i] = __ldg(reinterpret_cast<const int4 *>(p.dft) + i);
    if (tid == 0) {
        for (int s = 0; s < kStages; s++) tc::mbar_init(&mb_v[s], 1);
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&mb_a1[b], kFront);
            tc::mbar_init(&mb_d1[b], 1);
            tc::mbar_init(&mb_a2[b], 128);
            tc::mbar_init(&mb_full[b], 1);
            tc::mbar_init(&mb_empty[b], kEpi);
        }
        tc::mbar_init(&mb_a2free, 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot, G::kTmemCols);
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_slot;

    const long long s0 = p.cta_begin ? p.cta_begin[blockIdx.x] : (long long)blockIdx.x * p.len;
    const long long s1 = p.cta_begin ? p.cta_begin[blockIdx.x + 1] : min(s0 + p.len, p.total);
    const int nsteps = tc_count_steps(s0, s1, p.T, G::kSps);

    if (warp < kMmaWarp) {
        // ================================================================ front
        int cur_station = -1, ne = 0;
        int a1_st0 = -1, a1_st1 = -1;          // station whose cells buffer 0 / 1 holds
        int ntile = 0;
        const uint32_t *s_cell = nullptr;
        const int32_t *s_base = nullptr, *s_warp = nullptr;
        const float2 *s_w = nullptr;
        const uint16_t *s_e = nullptr;

        // new station: its gather table into shared memory; A1 buffer b zeroed
        // when it last held another station's cells
        auto prepare = [&](const TcStep &s, int i) {
            const int stn = s.stn;
            const int b = i & 1;
            if (stn == cur_station && (b ? a1_st1 : a1_st0) == stn) return;
            bar_front();                           // every front warp is done with step i-1
            if (stn != cur_station) {
                const TcStation st = p.stations[stn];
                for (int k = tid; k < (int)(st.table_bytes / 16); k += kFront)
                    reinterpret_cast<int4 *>(sT)[k] = __ldg(reinterpret_cast<const int4 *>(st.table) + k);
                const GatherLayout gl = gather_layout(st.ntile, st.nent);
                s_cell = reinterpret_cast<const uint32_t *>(sT + gl.off_cell);
                s_base = reinterpret_cast<const int32_t *>(sT + gl.off_base);
                s_warp = reinterpret_cast<const int32_t *>(sT + gl.off_warp);
                s_w = reinterpret_cast<const float2 *>(sT + gl.off_w);
                s_e = reinterpret_cast<const uint16_t *>(sT + gl.off_e);
                ntile = st.ntile;
                ne = st.ne;
                cur_station = stn;
            }
            if ((b ? a1_st1 : a1_st0) != stn) {
                for (int k = tid; k < (int)(G::kSet * G::kA1Bytes / 16); k += kFront)
                    reinterpret_cast<int4 *>(sA1 + b * G::kSet * G::kA1Bytes)[k] = make_int4(0, 0, 0, 0);
                (b ? a1_st1 : a1_st0) = stn;
            }
            bar_front();
        };
        // voltages of step i -> sE[i & 1]: per element the step's fields as
        // half2 (int8 values are exact in fp16); ends with a front barrier
        auto stage_volt = [&](const TcStep &s, int i) {
            const int8_t *V;
            uint32_t delta;
            const int8_t *src = tc_aligned_src(s.src, p.guard, delta);
            if (p.use_tma) {
                tc::mbar_wait(&mb_v[i % kStages], (uint32_t)((i / kStages) & 1), p.status);
                V = sV + (i % kStages) * p.vstage + delta;
            } else {
                const int bytes = s.nv * 4 * ne;
                int8_t *dst = sV + (i % kStages) * p.vstage;
                for (int b = tid; b < bytes; b += kFront) dst[b] = src[b];
                bar_front();
                V = dst;
            }
            uint4 *E = sE + (size_t)(i & 1) * p.ne_max * G::kU;
            const char2 *v2 = reinterpret_cast<const char2 *>(V);
            for (int a = tid; a < ne; a += kFront) {
                uint32_t h[G::kFields];
#pragma unroll
                for (int f = 0; f < G::kFields; f++) {
                    char2 x = make_char2(0, 0);    // missing sample: 0
                    if (f < 2 * s.nv) x = v2[f * ne + a];
                    h[f] = tc::pack_half2((float)x.x, (float)x.y);
                }
#pragma unroll
                for (int u = 0; u < G::kU; u++)
                    E[a * G::kU + u] = make_uint4(h[4 * u], h[4 * u + 1], h[4 * u + 2], h[4 * u + 3]);
            }
            bar_front();
        };
        // gridded values of the step's fields: G_f[cell] = sum conj(W~) E_f,
        // one cell per lane, one tile of 32 cells per warp at a time
        auto grid_step = [&](int i) {
            uint8_t *A = sA1 + (i & 1) * G::kSet * G::kA1Bytes;
            const uint4 *E = sE + (size_t)(i & 1) * p.ne_max * G::kU;
            for (int t = s_warp[warp]; t < s_warp[warp + 1]; t++) {
                float2 g[G::kFields];
#pragma unroll
                for (int f = 0; f < G::kFields; f++) g[f] = make_float2(0.f, 0.f);
                const int qe = s_base[t + 1];
                // add one slot's conj(W~) E into the fields' sums
                auto mac = [&](const float2 w, const uint4 *e) {
#pragma unroll
                    for (int u = 0; u < G::kU; u++) {
                        const uint32_t ev[4] = {e[u].x, e[u].y, e[u].z, e[u].w};
#pragma unroll
                        for (int k = 0; k < 4; k++) {
                            const float2 x = __half22float2(*reinterpret_cast<const __half2 *>(&ev[k]));
                            float2 &acc = g[4 * u + k];
                            acc.x = fmaf(w.x, x.x, fmaf(-w.y, x.y, acc.x));
                            acc.y = fmaf(w.x, x.y, fmaf(w.y, x.x, acc.y));
                        }
                    }
                };
                // the lane's slots are q, q + 32, ...: four at a time with all
                // their shared-memory loads issued before the first use (the
                // loop is bound by load latency, not by issue)
                int q = s_base[t] + lane;
                for (; q + 96 < qe; q += 128) {
                    float2 w[4];
                    int en[4];
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        w[j] = s_w[q + 32 * j];
                        en[j] = s_e[q + 32 * j];
                    }
                    uint4 e[4][G::kU];
#pragma unroll
                    for (int j = 0; j < 4; j++)
#pragma unroll
                        for (int u = 0; u < G::kU; u++) e[j][u] = E[en[j] * G::kU + u];
#pragma unroll
                    for (int j = 0; j < 4; j++) mac(w[j], e[j]);
                }
                for (; q < qe; q += 32) {
                    const float2 w = s_w[q];
                    uint4 e[G::kU];
                    const int en = s_e[q];
#pragma unroll
                    for (int u = 0; u < G::kU; u++) e[u] = E[en * G::kU + u];
                    mac(w, e);
                }
                const uint32_t off = s_cell[t * 32 + lane];
                if (off != 0xffffffffu) {
                    uint8_t *c = A + off;
#pragma unroll
                    for (int f = 0; f < G::kFields; f++) {
                        if (SP) {              // the rounding remainder as the lo copy
                            uint32_t hi, lo;
                            tc::pack2_split<BF>(g[f].x, g[f].y, hi, lo);
                            *reinterpret_cast<uint32_t *>(c + f * G::kImgBytes) = hi;
                            *reinterpret_cast<uint32_t *>(c + G::kA1Bytes + f * G::kImgBytes) = lo;
                        } else {
                            *reinterpret_cast<uint32_t *>(c + f * G::kImgBytes) = tc::pack2<BF>(g[f].x, g[f].y);
                        }
                    }
                }
            }
        };
        // warps 0-3: D1 row m = (field, y) -> A2 tile of its sample, column
        // (y, re/im), rows (sample in tile, l_x, pol)
        auto convert = [&](const TcStep &s, int i) {
            const int m = warp * 32 + lane;
            const int f = m / G::kBox, y = m % G::kBox;
            const int smp = f >> 1, pol = f & 1;
            const int tile = smp / G::kTileSamples, s2 = smp % G::kTileSamples;
            if (tile * G::kTileSamples >= s.nv) return;   // tile not issued
            uint8_t *A2 = sA2 + (((i % G::kA2Steps) * G::kTiles + tile) * G::kSet) * G::kA2Bytes;
            const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(i & 1) * G::kNcol;
#pragma unroll
            for (int ch = 0; ch < G::kNcol / 32; ch++) {   // 32 columns: component c, l_x = kx0 .. kx0+31
                uint32_t r[32];
                tc::tmem_ld32(base + ch * 32, r);
                tc::tmem_wait_ld();
                const int c = (ch * 32) / N, kx0 = (ch * 32) % N;
                const int kappa = 2 * y + c;
#pragma unroll
                for (int h = 0; h < 4; h++) {      // 8 frequencies -> one 16-byte row of A2
                    const int kx = kx0 + 8 * h;
                    const int m2 = s2 * 2 * N + (kx >> 4) * 32 + pol * 16 + (kx & 15);
                    uint32_t hv[4], lv[4];
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const float x0 = __uint_as_float(r[8 * h + 2 * e]), x1 = __uint_as_float(r[8 * h + 2 * e + 1]);
                        if (SP) tc::pack2_split<BF>(x0, x1, hv[e], lv[e]);
                        else hv[e] = tc::pack2<BF>(x0, x1);
                    }
                    const uint32_t off = tc::off_mnmajor(m2, kappa, kA2Ks, kA2MNs);
                    *reinterpret_cast<uint4 *>(A2 + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                    if (SP) *reinterpret_cast<uint4 *>(A2 + G::kA2Bytes + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
                }
            }
        };
        // A1 buffer (i+1)&1 was last read by MMA1(i-1), whose completion the
        // converters saw before the next front barrier; A2 buffer i&1 was last
        // read by MMA2(i-2), issued before MMA1(i), whose completion convert waits.
        TcWalker wk;
        wk.init(p.volt, p.stations, p.C, p.T, s0, s1);
        TcStep prev{}, nxt{};
        for (int i = -1; i < nsteps; i++) {
            if (i + 1 < nsteps) {
                nxt = wk.next(G::kSps);
                prepare(nxt, i + 1);
                stage_volt(nxt, i + 1);
                grid_step(i + 1);
                tc::fence_proxy_async();
                tc::mbar_arrive(&mb_a1[(i + 1) & 1]);
            }
            if (i >= 0 && warp < 4) {
                tc::mbar_wait(&mb_d1[i & 1], (uint32_t)((i >> 1) & 1), p.status);
                // one stage-2 operand buffer (split): the MMAs of step i-1 read it
                if (SP && i >= 1) tc::mbar_wait(&mb_a2free, (uint32_t)((i - 1) & 1), p.status);
                tc::fence_after();
                convert(prev, i);
                tc::fence_proxy_async();
                tc::fence_before();
                tc::mbar_arrive(&mb_a2[i & 1]);
            }
            prev = nxt;
        }
    } else if (warp == kMmaWarp) {
        // ================================================================ MMA + TMA
        if (lane == 0) {
            const uint32_t b = tc::smem_u32(sB);
            TcWalker ld;
            ld.init(p.volt, p.stations, p.C, p.T, s0, s1);
            int n_loaded = 0;
            auto issue_load = [&]() {
                if (n_loaded >= nsteps || !p.use_tma) return;
                const TcStep s = ld.next(G::kSps);
                uint32_t delta;
                const int8_t *src = tc_aligned_src(s.src, p.guard, delta);
                const uint32_t bytes = (delta + (uint32_t)s.nv * 4u * s.ne + 15u) & ~15u;
                const int sg = n_loaded % kStages;
                tc::mbar_arrive_expect_tx(&mb_v[sg], bytes);
                tc::bulk_g2s(sV + sg * p.vstage, src, bytes, &mb_v[sg]);
                n_loaded++;
            };
            for (int q = 0; q < kStages; q++) issue_load();
            TcWalker wk;
            wk.init(p.volt, p.stations, p.C, p.T, s0, s1);
            TcStep prev{}, nxt{};
            int jt = 0;                            // stage-2 tiles issued
            for (int k = -1; k < nsteps; k++) {
                if (k + 1 < nsteps) {              // stage 1 of step k+1
                    const int i = k + 1;
                    nxt = wk.next(G::kSps);
                    tc::mbar_wait(&mb_a1[i & 1], (uint32_t)((i >> 1) & 1), p.status);
                    issue_load();                  // its voltage stage has been widened
                    tc::fence_after();
                    const uint32_t a = tc::smem_u32(sA1 + (i & 1) * G::kSet * G::kA1Bytes);
                    const uint32_t d = tmem + (uint32_t)(i & 1) * G::kNcol;
                    // products hi*hi [+ hi*lo + lo*hi]: (A offset, B offset) per product
#pragma unroll
                    for (int pr = 0; pr < (SP ? 3 : 1); pr++) {
                        const uint32_t ao = pr == 2 ? G::kA1Bytes : 0u, bo = pr == 1 ? G::kBBytes : 0u;
#pragma unroll
                        for (int s = 0; s < G::kK / 16; s++)
                            tc::mma_f16(d, tc::desc(a + ao + s * 2 * kKs, kKs, G::kMNs),
                                        tc::desc(b + bo + s * 2 * kKs, kKs, G::kMNs), kIdesc1, (pr > 0 || s > 0));
                    }
                    tc::mma_commit(&mb_d1[i & 1]);
                }
                if (k >= 0) {                      // stage 2 of step k, one slot per tile
                    tc::mbar_wait(&mb_a2[k & 1], (uint32_t)((k >> 1) & 1), p.status);
                    const int ntl = (prev.nv + G::kTileSamples - 1) / G::kTileSamples;
                    for (int g = 0; g < ntl; g++, jt++) {
                        const int slot = jt & 1;
                        if (jt >= 2) tc::mbar_wait(&mb_empty[slot], (uint32_t)(((jt >> 1) - 1) & 1), p.status);
                        tc::fence_after();
                        const uint32_t a =
                            tc::smem_u32(sA2 + (((k % G::kA2Steps) * G::kTiles + g) * G::kSet) * G::kA2Bytes);
                        const uint32_t d = tmem + 2u * G::kNcol + (uint32_t)slot * G::kNcol;
#pragma unroll
                        for (int pr = 0; pr < (SP ? 3 : 1); pr++) {
                            const uint32_t ao = pr == 2 ? G::kA2Bytes : 0u, bo = pr == 1 ? G::kBBytes : 0u;
#pragma unroll
                            for (int s = 0; s < G::kK / 16; s++)
                                tc::mma_f16(d, tc::desc(a + ao + s * 2 * kA2Ks, kA2Ks, kA2MNs),
                                            tc::desc(b + bo + s * 2 * kKs, kKs, G::kMNs), kIdesc2, (pr > 0 || s > 0));
                        }
                        tc::mma_commit(&mb_full[slot]);
                    }
                    if (SP) tc::mma_commit(&mb_a2free);   // the single stage-2 operand may be rewritten
                }
                prev = nxt;
            }
        }
    } else {
        // ============================================================= epilogue
        const int q = warp & 3, h = (warp - 8) >> 2;
        const int m = 32 * q + lane;
        const int s2 = m / (2 * N), mm = m % (2 * N);
        const int pol = (mm >> 4) & 1, kx = (mm >> 5) * 16 + (mm & 15);
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        constexpr int kLy = G::kLy;
        constexpr int kNN = N * N;
        // packed pairs: acc_a[t / 2] holds rows t, t + 1 of the own polarisation's
        // power; acc_x[t] the (re, im) cross product of one row
        float2 acc_a[kLy / 2], acc_x[kLy / 2];
#pragma unroll
        for (int t = 0; t < kLy / 2; t++) acc_a[t] = acc_x[t] = make_float2(0.f, 0.f);
        int seg = 0;
        long long cur_blk = -1;
        // the two sample slots of an N = 32 tile hold partial sums of the same
        // pixels: slot 0 writes, slot 1 adds after an epilogue barrier
        auto flush = [&](int stn, int c, int sgm) {
            float *dst = p.direct ? p.img + p.stations[stn].img_off + (size_t)c * 4 * kNN
                                  : p.partials + ((size_t)blockIdx.x * 2 + sgm) * 4 * kNN;
#pragma unroll
            for (int phase = 0; phase < G::kTileSamples; phase++) {
                if (phase > 0) bar_epi();
                if (s2 != phase) continue;
                const bool add = phase > 0 || (p.direct && p.accumulate);
#pragma unroll
                for (int t = 0; t < kLy; t++) {
                    const int idx = pol * kNN + (kLy * h + t) * N + kx;
                    float v = (t & 1) ? acc_a[t >> 1].y : acc_a[t >> 1].x;
                    if (add) v += dst[idx];
                    dst[idx] = v;
                }
#pragma unroll
                for (int t = 0; t < kLy / 2; t++) acc_a[t] = make_float2(0.f, 0.f);
                // cross products: the X thread holds X conj(Y) at even rows, the Y
                // thread Y conj(X) = conj(X conj(Y)) at odd rows
                const float sgn = pol ? -1.f : 1.f;
#pragma unroll
                for (int t = 0; t < kLy / 2; t++) {
                    const int ly = kLy * h + 16 * (t >> 3) + 2 * (t & 7) + pol;
                    const int idx = 2 * kNN + ly * N + kx;
                    float vr = acc_x[t].x, vi = sgn * acc_x[t].y;
                    if (add) {
                        vr += dst[idx];
                        vi += dst[idx + kNN];
                    }
                    dst[idx] = vr;
                    dst[idx + kNN] = vi;
                    acc_x[t] = make_float2(0.f, 0.f);
                }
            }
        };
        TcWalker wk;
        wk.init(p.volt, p.stations, p.C, p.T, s0, s1);
        int jt = 0, cur_stn = 0, cur_chan = 0;
        for (int i = 0; i < nsteps; i++) {
            const TcStep s = wk.next(G::kSps);
            const long long blk = s.blk(p.C);
            if (blk != cur_blk) {
                if (cur_blk >= 0) {
                    flush(cur_stn, cur_chan, seg);
                    seg++;
                }
                cur_blk = blk;
                cur_stn = s.stn;
                cur_chan = s.chan;
            }
            const int ntl = (s.nv + G::kTileSamples - 1) / G::kTileSamples;
            for (int g = 0; g < ntl; g++, jt++) {
                const int slot = jt & 1;
                tc::mbar_wait(&mb_full[slot], (uint32_t)((jt >> 1) & 1), p.status);
                tc::fence_after();
#pragma unroll
                for (int cc = 0; cc < kLy / 16; cc++) {
                    const uint32_t col = 2u * G::kNcol + (uint32_t)slot * G::kNcol + (uint32_t)(kLy * h + 16 * cc);
                    uint32_t rr[16], ri[16];
                    tc::tmem_ld16(tmem + lane_base + col, rr);
                    tc::tmem_ld16(tmem + lane_base + col + N, ri);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int t = 0; t < 16; t += 2) {
                        const float2 fr = make_float2(__uint_as_float(rr[t]), __uint_as_float(rr[t + 1]));
                        const float2 fi = make_float2(__uint_as_float(ri[t]), __uint_as_float(ri[t + 1]));
                        float2 &a = acc_a[(16 * cc + t) >> 1];
                        a = __ffma2_rn(fr, fr, __ffma2_rn(fi, fi, a));     // fmaf(fr, fr, fmaf(fi, fi, a))
                    }
#pragma unroll
                    for (int k = 0; k < 8; k++) {
                        // own value at row 2k + pol, partner's value at the same row
                        const float e_r = __uint_as_float(rr[2 * k]), e_i = __uint_as_float(ri[2 * k]);
                        const float o_r = __uint_as_float(rr[2 * k + 1]), o_i = __uint_as_float(ri[2 * k + 1]);
                        const float mr = pol ? o_r : e_r, mi = pol ? o_i : e_i;
                        const float sr = __shfl_xor_sync(0xffffffffu, pol ? e_r : o_r, 16);
                        const float si = __shfl_xor_sync(0xffffffffu, pol ? e_i : o_i, 16);
                        // (Re, Im) own conj(other): fmaf(mr, sr, fmaf(mi, si, re)),
                        // fmaf(mi, sr, fmaf(-mr, si, im)) as packed pairs
                        float2 &a = acc_x[8 * cc + k];
                        a = __ffma2_rn(make_float2(mr, mi), make_float2(sr, sr),
                                       __ffma2_rn(make_float2(mi, -mr), make_float2(si, si), a));
                    }
                }
                tc::fence_before();
                tc::mbar_arrive(&mb_empty[slot]);
            }
        }
        if (cur_blk >= 0) flush(cur_stn, cur_chan, seg);
    }

    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, G::kTmemCols);
}

template <int N, bool SP>
size_t smem_bytes(int ne_max, uint32_t table_max) {
    using G = Geo<N, SP>;
    const uint32_t vstage = ((uint32_t)G::kSps * 4u * ne_max + 16u + 15u) & ~15u;
    return G::kOffE + 32ull * G::kU * ne_max + (size_t)kStages * vstage + table_max;
}

// Dynamic shared memory a kernel may use: the device's opt-in limit less the
// kernel's static shared memory.
template <typename K>
hai_status raise_limit(hai_ctx *ctx, K kern) {
    cudaFuncAttributes a;
    HAI_CUDA_TRY(cudaFuncGetAttributes(&a, kern));
    HAI_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      ctx->smem_optin - (int)a.sharedSizeBytes));
    return HAI_OK;
}

template <int N, bool SP, bool BF>
hai_status run_n(hai_ctx *ctx, const TcLaunch &l, cudaStream_t st) {
    using G = Geo<N, SP>;
    const size_t smem = smem_bytes<N, SP>(l.ne_max, l.table_max);
    if (smem + kStaticSmem > (size_t)ctx->smem_optin)
        return hai_fail(HAI_ERR_UNSUPPORTED, "epic fp16: shared memory need exceeds the device limit");
    const void *dft = epic_tc_dft(ctx, N, BF);
    if (!dft) return hai_fail(HAI_ERR_INVALID_ARG, "epic tensor cores: DFT operand not prepared");
    // the limit is the device's, so launches of any size (and captured graphs) stay valid
    if (!l.no_attr) {
        const hai_status s = epic_tc_set_attr(ctx, N);
        if (s != HAI_OK) return s;
    }
    if (SP || BF) {
        const hai_status s = raise_limit(ctx, epic_tc_kernel<N, SP, BF>);
        if (s != HAI_OK) return s;
    }
    Params p;
    p.volt = l.volt;
    p.img = l.img;
    p.stations = l.stations;
    p.dft = static_cast<const uint8_t *>(dft);
    p.cta_begin = l.cta_begin;
    p.len = l.len;
    p.total = (long long)l.n_station * l.C * l.T;
    p.C = l.C;
    p.T = l.T;
    p.ne_max = l.ne_max;
    p.vstage = ((uint32_t)G::kSps * 4u * l.ne_max + 16u + 15u) & ~15u;
    p.direct = l.direct;
    p.accumulate = l.accumulate;
    p.guard = l.guard;
    // without guard bytes every step must start on 16 bytes: 4 ne % 16 == 0
    // for every station and an aligned base
    p.use_tma = l.guard || (((uintptr_t)l.volt & 15) == 0 && (4 * l.ne_max) % 16 == 0 && l.n_station == 1);
    p.partials = l.partials;
    p.status = ctx->d_status;
    const int pidx = prof_begin(ctx, st);
    epic_tc_kernel<N, SP, BF><<<l.n_cta, kThreads, smem, st>>>(p);
    prof_end(ctx, pidx, st);
    prof_count(ctx, 1);
    HAI_CUDA_TRY(cudaGetLastError());
    return HAI_OK;
}

}  // namespace

void epic_tc_a1_strides(int N, uint32_t &k_stride, uint32_t &mn_stride) {
    k_stride = kKs;
    mn_stride = (N == 32) ? Geo<32, false>::kMNs : (N == 64) ? Geo<64, false>::kMNs : 16 * kKs;   // N = 128: K = 128
}

int epic_tc_group(int N) { return N == 128 ? 4 : 1; }

size_t epic_tc_smem(hai_ctx *, int N, int ne_max, uint32_t table_max) {
    if (N == 32) return smem_bytes<32, false>(ne_max, table_max);
    if (N == 64) return smem_bytes<64, false>(ne_max, table_max);
    if (N == 128) return epic_tc128_smem(ne_max, table_max);
    return (size_t)-1;
}

hai_status epic_tc_set_attr(hai_ctx *ctx, int N) {
    if (N == 32) return raise_limit(ctx, epic_tc_kernel<32, false, false>);
    if (N == 64) return raise_limit(ctx, epic_tc_kernel<64, false, false>);
    if (N == 128) return epic_tc128_set_attr(ctx);
    return HAI_OK;
}

hai_status epic_tc_run(hai_ctx *ctx, int N, const TcLaunch &l, cudaStream_t st) {
    if (l.n_cta <= 0) return HAI_OK;
    if (l.split || l.bf16) {
        if (N == 32 && l.split) return l.bf16 ? run_n<32, true, true>(ctx, l, st) : run_n<32, true, false>(ctx, l, st);
        if (N == 64 && l.split) return l.bf16 ? run_n<64, true, true>(ctx, l, st) : run_n<64, true, false>(ctx, l, st);
        if (N == 32) return run_n<32, false, true>(ctx, l, st);
        if (N == 64) return run_n<64, false, true>(ctx, l, st);
        if (N == 128 && !l.split) return epic_tc128_run(ctx, l, st);
        return hai_fail(HAI_ERR_UNSUPPORTED, "epic tensor cores: the hi/lo split needs N = 32, 64, 256 or 512");
    }
    if (N == 32) return run_n<32, false, false>(ctx, l, st);
    if (N == 64) return run_n<64, false, false>(ctx, l, st);
    if (N == 128) return epic_tc128_run(ctx, l, st);
    return hai_fail(HAI_ERR_UNSUPPORTED, "epic fp16: grid size");
}

double epic_tc_dft_entry(int N, int c_out, int l, int j, int c_in) {
    const double ang = 2.0 * 3.14159265358979323846 * (double)(((long long)l * j) % N) / N;
    const double sgn = (j & 1) ? -1.0 : 1.0;
    const double wr = sgn * cos(ang), wi = sgn * sin(ang);
    // y_re = sum x_re wr - x_im wi ; y_im = sum x_re wi + x_im wr
    if (c_out == 0) return c_in == 0 ? wr : -wi;
    return c_in == 0 ? wi : wr;
}

// DFT operands, one blob per grid side, owned by the context.  N = 32, 64:
// B[n = (c_out, l)][kappa = (j, c_in)], K-major, j < N/2.  N = 128: the four
// column-quarter operands B1[r][n = (c_out, l mod 32)][kappa = (x, c_in)]
// (l = 32 r + l mod 32), then the stage-2 operand A2[l_y][kappa = (y, c_in)]
// (see epic_tc128.cu), all K-major with K = 128.
hai_status epic_tc_dft_prepare(hai_ctx *ctx, int N) {
    const int slot = (N == 32) ? 0 : (N == 64) ? 1 : (N == 128) ? 2 : -1;
    if (slot < 0) return hai_fail(HAI_ERR_UNSUPPORTED, "epic fp16: grid size");
    if (ctx->d_dft[slot]) return HAI_OK;
    std::vector<uint8_t> out, outb;
    auto put = [&](size_t base, uint32_t off, double v) {
        const __half hv = __double2half(v);
        memcpy(&out[base + off], &hv, 2);
        if (!outb.empty() && N == 128) {          // the BF16 copy of the N = 128 operands
            const __nv_bfloat16 bv = __double2bfloat16(v);
            memcpy(&outb[base + off], &bv, 2);
        }
    };
    if (N <= 64) {
        // hi = fp16(W'), then lo = fp16(W' - hi) for the split variant; the
        // same in BF16 in a second blob
        const int box = N / 2, K = 2 * box;
        const uint32_t mns = (uint32_t)(K / 8) * kKs;
        const size_t half_bytes = (size_t)(2 * N / 8) * mns;
        out.assign(2 * half_bytes, 0);
        outb.assign(2 * half_bytes, 0);
        for (int n = 0; n < 2 * N; n++)
            for (int kappa = 0; kappa < K; kappa++) {
                const double v = epic_tc_dft_entry(N, n / N, n % N, kappa >> 1, kappa & 1);
                const double hi = (double)__half2float(__double2half(v));
                put(0, tc::off_kmajor(n, kappa, kKs, mns), v);
                put(half_bytes, tc::off_kmajor(n, kappa, kKs, mns), v - hi);
                const __nv_bfloat16 bh = __double2bfloat16(v);
                const __nv_bfloat16 bl = __double2bfloat16(v - (double)__bfloat162float(bh));
                memcpy(&outb[tc::off_kmajor(n, kappa, kKs, mns)], &bh, 2);
                memcpy(&outb[half_bytes + tc::off_kmajor(n, kappa, kKs, mns)], &bl, 2);
            }
    } else {
        const uint32_t mns = 16 * kKs;              // K = 128
        const size_t qbytes = 8 * (size_t)mns;     // 64 rows
        out.assign(4 * qbytes + 16 * (size_t)mns, 0);
        outb.assign(out.size(), 0);
        for (int r = 0; r < 4; r++)
            for (int n = 0; n < 64; n++)
                for (int kappa = 0; kappa < 128; kappa++)
                    put(r * qbytes, tc::off_kmajor(n, kappa, kKs, mns),
                        epic_tc_dft_entry(N, n >> 5, 32 * r + (n & 31), kappa >> 1, kappa & 1));
        // A2[l_y][(y, c_in)]: row l_y of W'^T as the left factor of stage 2;
        // (y, 0) -> Re W'[y][l_y], (y, 1) -> Im W'[y][l_y]
        for (int ly = 0; ly < 128; ly++)
            for (int kappa = 0; kappa < 128; kappa++) {
                const double re = epic_tc_dft_entry(N, 0, ly, kappa >> 1, 0);   // wr
                const double im = epic_tc_dft_entry(N, 1, ly, kappa >> 1, 0);   // wi
                put(4 * qbytes, tc::off_kmajor(ly, kappa, kKs, mns), (kappa & 1) ? im : re);
            }
    }
    void *d = nullptr;
    HAI_CUDA_TRY(cudaSetDevice(ctx->device));
    HAI_CUDA_TRY(cudaMalloc(&d, out.size()));
    HAI_CUDA_TRY(cudaMemcpy(d, out.data(), out.size(), cudaMemcpyHostToDevice));
    ctx->d_dft[slot] = d;
    ctx->dev_bytes += out.size();
    if (!outb.empty()) {
        void *db = nullptr;
        HAI_CUDA_TRY(cudaMalloc(&db, outb.size()));
        HAI_CUDA_TRY(cudaMemcpy(db, outb.data(), outb.size(), cudaMemcpyHostToDevice));
        ctx->d_dft[3 + slot] = db;
        ctx->dev_bytes += outb.size();
    }
    return HAI_OK;
}

const void *epic_tc_dft(hai_ctx *ctx, int N, bool bf16) {
    const int slot = (N == 32) ? 0 : (N == 64) ? 1 : (N == 128) ? 2 : -1;
    if (slot < 0) return nullptr;
    return ctx->d_dft[slot + (bf16 ? 3 : 0)];
}

void epic_tc_build_gather(int box_w, int box_h, const std::vector<int32_t> &cstart,
                          const std::vector<int32_t> &elem, const std::vector<float2> &w, uint32_t k_stride,
                          uint32_t mn_stride, std::vector<uint8_t> &out, int &ntile, int &nent, int n_warps) {
    std::vector<int> cells;
    for (int y = 0; y < box_h; y++)
        for (int x = 0; x < box_w; x++)
            if (cstart[y * box_w + x + 1] > cstart[y * box_w + x]) cells.push_back(y * box_w + x);
    auto count = [&](int c) { return cstart[c + 1] - cstart[c]; };
    auto a1off = [&](int cell) { return tc::off_kmajor(cell / box_w, 2 * (cell % box_w), k_stride, mn_stride); };
    std::stable_sort(cells.begin(), cells.end(), [&](int a, int b) {
        if (count(a) != count(b)) return count(a) > count(b);
        return a1off(a) < a1off(b);
    });
    ntile = ((int)cells.size() + 31) / 32;
    // tiles in cell order, then dealt to the gridding warps longest-first
    std::vector<int> slots(ntile, 0);
    for (int t = 0; t < ntile; t++)
        for (int l = 0; l < 32 && t * 32 + l < (int)cells.size(); l++) slots[t] = std::max(slots[t], count(cells[t * 32 + l]));
    std::vector<int> by_cost(ntile);
    for (int t = 0; t < ntile; t++) by_cost[t] = t;
    std::stable_sort(by_cost.begin(), by_cost.end(), [&](int a, int b) { return slots[a] > slots[b]; });
    std::vector<std::vector<int>> mine(kGatherWarps);
    std::vector<int> load(n_warps, 0);
    for (int t : by_cost) {
        const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        mine[w].push_back(t);
        load[w] += slots[t] + 1;
    }
    std::vector<int> order;                  // new position -> original tile
    std::vector<int> wrange(kGatherWarps + 1, 0);
    for (int w = 0; w < kGatherWarps; w++) {
        order.insert(order.end(), mine[w].begin(), mine[w].end());
        wrange[w + 1] = (int)order.size();
    }
    std::vector<int> base(ntile + 1, 0);
    for (int t = 0; t < ntile; t++) base[t + 1] = base[t] + 32 * slots[order[t]];
    nent = base[ntile];
    const GatherLayout gl = gather_layout(ntile, nent);
    out.assign(gl.bytes, 0);
    uint32_t *o_cell = reinterpret_cast<uint32_t *>(&out[gl.off_cell]);
    int32_t *o_base = reinterpret_cast<int32_t *>(&out[gl.off_base]);
    int32_t *o_warp = reinterpret_cast<int32_t *>(&out[gl.off_warp]);
    float2 *o_w = reinterpret_cast<float2 *>(&out[gl.off_w]);
    uint16_t *o_e = reinterpret_cast<uint16_t *>(&out[gl.off_e]);
    for (int t = 0; t <= ntile; t++) o_base[t] = base[t];
    for (int w = 0; w <= kGatherWarps; w++) o_warp[w] = wrange[w];
    for (int t = 0; t < ntile; t++)
        for (int l = 0; l < 32; l++) {
            const int ci = order[t] * 32 + l;      // cell of lane l of the tile now at position t
            if (ci >= (int)cells.size()) {
                o_cell[t * 32 + l] = 0xffffffffu;
                continue;
            }
            const int cell = cells[ci];
            o_cell[t * 32 + l] = a1off(cell);
            for (int k = 0; k < count(cell); k++) {
                const int q = base[t] + 32 * k + l;
                o_w[q] = w[cstart[cell] + k];                 // conj(W~) = a + ib
                o_e[q] = (uint16_t)elem[cstart[cell] + k];
            }
        }
}

void epic_tc_station_table(int grid_n, int box_w, int box_h, const std::vector<int32_t> &cstart,
                           const std::vector<int32_t> &elem, const std::vector<float2> &w,
                           std::vector<uint8_t> &out, int &ntile, int &nent, uint32_t &shared_bytes,
                           long long &entries) {
    if (grid_n == 128) {
        epic_tc128_build_blob(box_w, box_h, cstart, elem, w, out, shared_bytes, entries);
        ntile = nent = 0;
        return;
    }
    uint32_t ks, mns;
    epic_tc_a1_strides(grid_n, ks, mns);
    epic_tc_build_gather(box_w, box_h, cstart, elem, w, ks, mns, out, ntile, nent);
    shared_bytes = (uint32_t)out.size();
    entries = nent;
}

// ---------------------------------------------------------------- one layout
bool epic_tc_supported(const hai_layout *L) {
    const int n = L->grid_n;
    return (n == 32 || n == 64 || n == 128) && L->n_pol == 2 && L->box_w <= n / 2 && L->box_h <= n / 2 &&
           L->n_elem <= 65535;
}

hai_status epic_tc_launch(const hai_layout *L, const int8_t *volt, int C, int T, float *img, int accumulate,
                          cudaStream_t st, int split, int bf16) {
    if (!epic_tc_supported(L) || !L->d_tc_station)
        return hai_fail(HAI_ERR_UNSUPPORTED,
                        "epic fp16: the tensor-core path needs N = 32, 64 or 128, 2 pols and a kernel box "
                        "<= N/2 x N/2");
    hai_ctx *ctx = L->ctx;
    const int N = L->grid_n, grp = epic_tc_group(N);
    const EpicSplit sp = epic_make_split(C, T, N == 128 ? L->tc_groups : ctx->num_sms / grp);
    if (!sp.direct && (size_t)sp.n_cta * 2 > L->partial_slots)
        return hai_fail(HAI_ERR_INVALID_ARG, "epic fp16: partial buffer too small");
    TcLaunch l;
    l.volt = volt;
    l.img = img;
    l.stations = static_cast<const TcStation *>(L->d_tc_station);
    l.n_station = 1;
    l.ne_max = L->n_elem;
    l.table_max = (uint32_t)L->tc_tables_bytes;
    l.cta_begin = nullptr;
    l.len = sp.len;
    l.n_cta = sp.n_cta;
    l.C = C;
    l.T = T;
    l.direct = sp.direct;
    l.accumulate = accumulate;
    l.guard = 0;
    l.partials = L->d_partials;
    l.no_attr = 0;
    l.split = split;
    l.bf16 = bf16;
    const hai_status s = epic_tc_run(ctx, N, l, st);
    if (s != HAI_OK) return s;
    if (!sp.direct) return epic_reduce_launch(L, sp, C, T, img, accumulate, st);
    return HAI_OK;
}
