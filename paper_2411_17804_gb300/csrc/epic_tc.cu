// EPIC direct imager on tcgen05 tensor cores (Eq. intra-station EPIC, then the
// squaring and temporal sum of Eq. intra-station squaring), FP16 operands with
// FP32 accumulation in tensor memory.
//
// The 2D DFT of each gridded field is two dense complex products with a
// constant DFT matrix, written as real GEMMs (complex -> (re, im) pairs):
//   stage 1 (along x):  H[y][l_x] = sum_x G[y][x] W'[x][l_x]
//   stage 2 (along y):  F[l_y][l_x] = sum_y W'[y][l_y] H[y][l_x]
// with W'[j][l] = (-1)^j exp(+2 pi i l j / N).  Only the kernel's bounding
// box (<= 32 x 32 cells) is transformed, from the box origin: the shift by the
// box corner multiplies F by a phase common to both polarisations, which
// cancels in every F_a conj(F_b); the (-1)^j factor puts the phase centre at
// pixel (N/2, N/2).
//
// CTA = 16 warps, one CTA per SM, persistent over a contiguous range of the
// flattened (channel, sample) index, two samples (four fields: 2 samples x
// 2 pols) per step:
//   warps 0-6  "front": re-pack the step's voltages (landed by TMA bulk
//              copies) as fp16 per element, gather-grid the four fields over
//              tiles of the layout's non-empty cells into A1 (fp16, K-major)
//              with FP32 sums; warps 0-3 then move
//              stage-1 results from TMEM into the stage-2 operand A2 (fp16,
//              MN-major), transposing on the way;
//   warp 7     one thread streams the voltages (TMA) and issues every MMA;
//   warps 8-15 epilogue: read stage-2 results from TMEM, add |F_X|^2,
//              |F_Y|^2 and F_X conj(F_Y) into register accumulators.
// Every hand-off between the roles is an mbarrier phase, so no role blocks
// on another's barrier.  TMEM (512 columns): stage-1 results double-buffered
// (2 x 128 columns) and stage-2 results in two per-sample slots (2 x 128), so
// the MMAs of one sample overlap the epilogue of the previous one.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "hai_internal.h"
#include "tc.cuh"

namespace {

constexpr int kN = 64;                  // grid side
constexpr int kBox = 32;                // padded box side
constexpr int kThreads = 512;
constexpr int kFront = 224;             // warps 0-6
constexpr int kMmaWarp = 7;
constexpr int kEpi = 256;               // warps 8-15
constexpr int kStages = 4;              // voltage steps in flight
constexpr uint32_t kKs = 128;           // K-major operands: K-group stride
constexpr uint32_t kMNs = 1024;         // K-major operands: MN-group stride (8 K groups)
constexpr uint32_t kOpBytes = 16384;    // 128 rows x 64 K x 2 bytes
constexpr uint32_t kImgBytes = 4096;    // one field's 32 rows inside A1
constexpr uint32_t kA2Ks = 2064;        // MN-major A2: K-group stride (16 groups + 16 B pad)
constexpr uint32_t kA2MNs = 128;        // MN-major A2: MN-group stride
constexpr uint32_t kA2Bytes = 8 * kA2Ks;
constexpr uint32_t kOffA1 = kOpBytes;   // after B
constexpr uint32_t kOffA2 = kOffA1 + 2 * kOpBytes;
constexpr uint32_t kOffE = kOffA2 + 4 * kA2Bytes;
constexpr uint32_t kIdesc1 = tc::idesc_f16(128, 128, 0, 0);
constexpr uint32_t kIdesc2 = tc::idesc_f16(128, 128, 1, 0);

// Device table written by epic_tc_build_table (byte layout).  The non-empty
// cells of the kernel's box are dealt into tiles of 32 (one per warp lane),
// sorted by entry count so a tile's lanes run the same number of slots; a
// tile's entries are stored slot-major, entry (slot k, lane l) at
// tile_base + 32 k + l, with zero-weight padding.
//   [0, 16384)         DFT operand B (K-major)
//   cell offsets       uint32 [ntile * 32]  A1 byte offset of the lane's cell (field 0),
//                                           0xffffffff for an unused lane
//   tile bases         int32 [ntile + 1]    first entry of each tile (slots = diff / 32)
//   (pad to 16)
//   entry weights      float2 [nent]        a + ib = conj(W~)
//   entry elements     uint16 [nent]
struct TableLayout {
    uint32_t off_cell, off_base, off_w, off_e, bytes;
};
__host__ __device__ inline TableLayout table_layout(int ntile, int nent) {
    TableLayout t;
    t.off_cell = kOpBytes;
    t.off_base = t.off_cell + 4u * 32u * ntile;
    t.off_w = (t.off_base + 4u * (ntile + 1) + 15u) & ~15u;
    t.off_e = t.off_w + 8u * nent;
    t.bytes = (t.off_e + 2u * nent + 15u) & ~15u;
    return t;
}

struct EpicTcParams {
    const int8_t *volt;
    int C, T, ne;
    long long len;
    int ntile, nent;
    const uint8_t *table;
    float *out;
    int direct, accumulate, use_tma;
    unsigned *status;
};

__device__ __forceinline__ void bar_front() { asm volatile("bar.sync 1, 224;" ::: "memory"); }

__global__ void __launch_bounds__(kThreads, 1) epic_tc_kernel(const EpicTcParams p) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mb_v[kStages];
    __shared__ __align__(8) uint64_t mb_a1[2], mb_d1[2], mb_a2[2], mb_full[2], mb_empty[2];
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ne = p.ne;
    const int sample_bytes = 4 * ne;                       // 2 pols x ne x (re, im)
    const uint32_t vstage = (2u * sample_bytes + 15u) & ~15u;
    const TableLayout tl = table_layout(p.ntile, p.nent);
    uint8_t *sB = smem;
    uint8_t *sA1 = smem + kOffA1;
    uint8_t *sA2 = smem + kOffA2;
    uint4 *sE = reinterpret_cast<uint4 *>(smem + kOffE);    // [2 buffers][ne] 4 fields as half2
    const uint32_t off_v = kOffE + 2u * 16u * ne;
    int8_t *sV = reinterpret_cast<int8_t *>(smem + off_v);
    uint8_t *sT = smem + off_v + kStages * vstage;          // copy of the table after B
    const uint32_t *s_cell = reinterpret_cast<const uint32_t *>(sT + tl.off_cell - kOpBytes);
    const int32_t *s_base = reinterpret_cast<const int32_t *>(sT + tl.off_base - kOpBytes);
    const float2 *s_w = reinterpret_cast<const float2 *>(sT + tl.off_w - kOpBytes);
    const uint16_t *s_e = reinterpret_cast<const uint16_t *>(sT + tl.off_e - kOpBytes);

    // ---- set-up: constant tables, zeroed A1, barriers, TMEM
    for (int i = tid; i < (int)(kOpBytes / 16); i += kThreads)
        reinterpret_cast<int4 *>(sB)[i] = __ldg(reinterpret_cast<const int4 *>(p.table) + i);
    for (int i = tid; i < (int)((tl.bytes - kOpBytes) / 16); i += kThreads)
        reinterpret_cast<int4 *>(sT)[i] = __ldg(reinterpret_cast<const int4 *>(p.table + kOpBytes) + i);
    for (int i = tid; i < (int)(2 * kOpBytes / 16); i += kThreads)
        reinterpret_cast<int4 *>(sA1)[i] = make_int4(0, 0, 0, 0);
    if (tid == 0) {
        for (int s = 0; s < kStages; s++) tc::mbar_init(&mb_v[s], 1);
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&mb_a1[b], kFront);
            tc::mbar_init(&mb_d1[b], 1);
            tc::mbar_init(&mb_a2[b], 128);
            tc::mbar_init(&mb_full[b], 1);
            tc::mbar_init(&mb_empty[b], kEpi);
        }
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot, 512);
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_slot;

    const long long total = (long long)p.C * p.T;
    const long long s0 = (long long)blockIdx.x * p.len;
    const long long s1 = min(total, s0 + p.len);
    const int nsamp = (int)max(0ll, s1 - s0);
    const int npairs = (nsamp + 1) / 2;
    auto pair_valid = [&](int i) { return min(2, nsamp - 2 * i); };

    if (warp < kMmaWarp) {
        // ================================================================ front
        // voltages of step i -> sE[i & 1]: per element the four fields as
        // half2 (int8 values are exact in fp16); ends with a front barrier
        auto stage_volt = [&](int i) {
            const int8_t *V = sV + (i % kStages) * vstage;
            const int nv = pair_valid(i);
            if (p.use_tma) {
                tc::mbar_wait(&mb_v[i % kStages], (uint32_t)((i / kStages) & 1), p.status);
            } else {
                const int bytes = nv * sample_bytes;
                const int8_t *src = p.volt + (size_t)(s0 + 2 * i) * sample_bytes;
                int8_t *dst = sV + (i % kStages) * vstage;
                for (int b = tid; b < bytes; b += kFront) dst[b] = src[b];
                bar_front();
            }
            // two consecutive elements x four fields per thread
            uint4 *E = sE + (i & 1) * ne;
            const char2 *v2 = reinterpret_cast<const char2 *>(V);
            for (int a0 = 2 * tid; a0 < ne; a0 += 2 * kFront) {
                uint32_t h0[4], h1[4];
#pragma unroll
                for (int f = 0; f < 4; f++) {
                    char2 x = make_char2(0, 0), y = make_char2(0, 0);   // missing sample: 0
                    if (f < 2 * nv) {
                        x = v2[f * ne + a0];
                        if (a0 + 1 < ne) y = v2[f * ne + a0 + 1];
                    }
                    h0[f] = tc::pack_half2((float)x.x, (float)x.y);
                    h1[f] = tc::pack_half2((float)y.x, (float)y.y);
                }
                E[a0] = make_uint4(h0[0], h0[1], h0[2], h0[3]);
                if (a0 + 1 < ne) E[a0 + 1] = make_uint4(h1[0], h1[1], h1[2], h1[3]);
            }
            bar_front();
        };
        // gridded values of the four fields: G_f[cell] = sum conj(W~) E_f,
        // one cell per lane, one tile of 32 cells per warp at a time
        auto grid_pair = [&](int i) {
            uint8_t *A = sA1 + (i & 1) * kOpBytes;
            const uint4 *E = sE + (i & 1) * ne;
            for (int t = warp; t < p.ntile; t += kMmaWarp) {
                float2 g0 = make_float2(0.f, 0.f), g1 = g0, g2 = g0, g3 = g0;
                const int qe = s_base[t + 1];
                int q = s_base[t] + lane;
                // software pipeline: slot k+1's weight and voltages load while slot k computes
                float2 w_n = s_w[q];
                uint4 e_n = E[s_e[q]];
                for (; q < qe; q += 32) {
                    const float2 w = w_n;
                    const uint4 e = e_n;
                    if (q + 32 < qe) {
                        w_n = s_w[q + 32];
                        e_n = E[s_e[q + 32]];
                    }
                    const float2 e0 = __half22float2(*reinterpret_cast<const __half2 *>(&e.x));
                    const float2 e1 = __half22float2(*reinterpret_cast<const __half2 *>(&e.y));
                    const float2 e2 = __half22float2(*reinterpret_cast<const __half2 *>(&e.z));
                    const float2 e3 = __half22float2(*reinterpret_cast<const __half2 *>(&e.w));
                    g0.x = fmaf(w.x, e0.x, fmaf(-w.y, e0.y, g0.x));
                    g0.y = fmaf(w.x, e0.y, fmaf(w.y, e0.x, g0.y));
                    g1.x = fmaf(w.x, e1.x, fmaf(-w.y, e1.y, g1.x));
                    g1.y = fmaf(w.x, e1.y, fmaf(w.y, e1.x, g1.y));
                    g2.x = fmaf(w.x, e2.x, fmaf(-w.y, e2.y, g2.x));
                    g2.y = fmaf(w.x, e2.y, fmaf(w.y, e2.x, g2.y));
                    g3.x = fmaf(w.x, e3.x, fmaf(-w.y, e3.y, g3.x));
                    g3.y = fmaf(w.x, e3.y, fmaf(w.y, e3.x, g3.y));
                }
                const uint32_t off = s_cell[t * 32 + lane];
                if (off != 0xffffffffu) {
                    uint8_t *c = A + off;
                    *reinterpret_cast<uint32_t *>(c) = tc::pack_half2(g0.x, g0.y);
                    *reinterpret_cast<uint32_t *>(c + kImgBytes) = tc::pack_half2(g1.x, g1.y);
                    *reinterpret_cast<uint32_t *>(c + 2 * kImgBytes) = tc::pack_half2(g2.x, g2.y);
                    *reinterpret_cast<uint32_t *>(c + 3 * kImgBytes) = tc::pack_half2(g3.x, g3.y);
                }
            }
        };
        auto convert = [&](int i) {               // warps 0-3: field f = warp, row y = lane
            const int f = warp, g = f >> 1, pol = f & 1, y = lane;
            if (g >= pair_valid(i)) return;
            uint8_t *A2 = sA2 + ((i & 1) * 2 + g) * kA2Bytes;
            const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(i & 1) * 128u;
#pragma unroll
            for (int ch = 0; ch < 4; ch++) {       // 32 columns: component c, frequencies kx0..kx0+31
                uint32_t r[32];
                tc::tmem_ld32(base + ch * 32, r);
                tc::tmem_wait_ld();
                const int c = ch >> 1, kx0 = (ch & 1) * 32;
                const int kappa = 2 * y + c;
#pragma unroll
                for (int h = 0; h < 4; h++) {      // 8 frequencies -> one 16-byte row of A2
                    const int kx = kx0 + 8 * h;
                    const int m = (kx >> 4) * 32 + pol * 16 + (kx & 15);
                    uint4 v;
                    v.x = tc::pack_half2(__uint_as_float(r[8 * h + 0]), __uint_as_float(r[8 * h + 1]));
                    v.y = tc::pack_half2(__uint_as_float(r[8 * h + 2]), __uint_as_float(r[8 * h + 3]));
                    v.z = tc::pack_half2(__uint_as_float(r[8 * h + 4]), __uint_as_float(r[8 * h + 5]));
                    v.w = tc::pack_half2(__uint_as_float(r[8 * h + 6]), __uint_as_float(r[8 * h + 7]));
                    *reinterpret_cast<uint4 *>(A2 + tc::off_mnmajor(m, kappa, kA2Ks, kA2MNs)) = v;
                }
            }
        };
        // A1 buffer (i+1)&1 was last read by MMA1(i-1), whose completion the
        // converters saw before the stage barrier; A2 buffer i&1 was last read
        // by MMA2(i-2), issued before MMA1(i), whose completion convert waits.
        for (int i = -1; i < npairs; i++) {
            if (i + 1 < npairs) {
                stage_volt(i + 1);
                grid_pair(i + 1);
                tc::fence_proxy_async();
                tc::mbar_arrive(&mb_a1[(i + 1) & 1]);
            }
            if (i >= 0 && warp < 4) {
                tc::mbar_wait(&mb_d1[i & 1], (uint32_t)((i >> 1) & 1), p.status);
                tc::fence_after();
                convert(i);
                tc::fence_proxy_async();
                tc::fence_before();
                tc::mbar_arrive(&mb_a2[i & 1]);
            }
        }
    } else if (warp == kMmaWarp) {
        // ================================================================ MMA + TMA
        if (lane == 0) {
            const uint32_t b = tc::smem_u32(sB);
            auto issue_load = [&](int i) {
                if (i >= npairs || !p.use_tma) return;
                const uint32_t bytes = (uint32_t)pair_valid(i) * sample_bytes;
                const int st = i % kStages;
                tc::mbar_arrive_expect_tx(&mb_v[st], bytes);
                tc::bulk_g2s(sV + st * vstage, p.volt + (size_t)(s0 + 2 * i) * sample_bytes, bytes, &mb_v[st]);
            };
            for (int q = 0; q < kStages; q++) issue_load(q);
            for (int k = -1; k < npairs; k++) {
                if (k + 1 < npairs) {              // stage 1 of step k+1
                    const int i = k + 1;
                    tc::mbar_wait(&mb_a1[i & 1], (uint32_t)((i >> 1) & 1), p.status);
                    issue_load(i + kStages);       // its voltage stage has been widened
                    tc::fence_after();
                    const uint32_t a = tc::smem_u32(sA1 + (i & 1) * kOpBytes);
                    const uint32_t d = tmem + (uint32_t)(i & 1) * 128u;
#pragma unroll
                    for (int s = 0; s < 4; s++)
                        tc::mma_f16(d, tc::desc(a + s * 2 * kKs, kKs, kMNs), tc::desc(b + s * 2 * kKs, kKs, kMNs),
                                    kIdesc1, s > 0);
                    tc::mma_commit(&mb_d1[i & 1]);
                }
                if (k >= 0) {                      // stage 2 of step k, one slot per sample
                    tc::mbar_wait(&mb_a2[k & 1], (uint32_t)((k >> 1) & 1), p.status);
                    const int nv = pair_valid(k);
                    for (int g = 0; g < nv; g++) {
                        const int j = 2 * k + g;
                        if (j >= 2) tc::mbar_wait(&mb_empty[g], (uint32_t)(((j >> 1) - 1) & 1), p.status);
                        tc::fence_after();
                        const uint32_t a = tc::smem_u32(sA2 + ((k & 1) * 2 + g) * kA2Bytes);
                        const uint32_t d = tmem + 256u + (uint32_t)g * 128u;
#pragma unroll
                        for (int s = 0; s < 4; s++)
                            tc::mma_f16(d, tc::desc(a + s * 2 * kA2Ks, kA2Ks, kA2MNs),
                                        tc::desc(b + s * 2 * kKs, kKs, kMNs), kIdesc2, s > 0);
                        tc::mma_commit(&mb_full[g]);
                    }
                }
            }
        }
    } else {
        // ============================================================= epilogue
        const int q = warp & 3, h = (warp - 8) >> 2;
        const int pol = lane >> 4, kx = 16 * q + (lane & 15);
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        float acc_a[32], acc_x[32];
#pragma unroll
        for (int t = 0; t < 32; t++) acc_a[t] = acc_x[t] = 0.f;
        int seg = 0;
        int cur_c = nsamp > 0 ? (int)(s0 / p.T) : 0;
        auto flush = [&](int c, int sgm) {
            float *dst = p.direct ? p.out + (size_t)c * 4 * kN * kN
                                  : p.out + ((size_t)blockIdx.x * 2 + sgm) * 4 * kN * kN;
#pragma unroll
            for (int t = 0; t < 32; t++) {
                const int idx = pol * kN * kN + (32 * h + t) * kN + kx;
                float v = acc_a[t];
                if (p.direct && p.accumulate) v += dst[idx];
                dst[idx] = v;
                acc_a[t] = 0.f;
            }
            // cross products: the X thread holds X conj(Y) at even rows, the Y
            // thread Y conj(X) = conj(X conj(Y)) at odd rows
            const float sgn = pol ? -1.f : 1.f;
#pragma unroll
            for (int t = 0; t < 16; t++) {
                const int ly = 32 * h + 16 * (t >> 3) + 2 * (t & 7) + pol;
                const int idx = 2 * kN * kN + ly * kN + kx;
                float vr = acc_x[2 * t], vi = sgn * acc_x[2 * t + 1];
                if (p.direct && p.accumulate) {
                    vr += dst[idx];
                    vi += dst[idx + kN * kN];
                }
                dst[idx] = vr;
                dst[idx + kN * kN] = vi;
                acc_x[2 * t] = acc_x[2 * t + 1] = 0.f;
            }
        };
        for (int j = 0; j < nsamp; j++) {
            const int g = j & 1;
            tc::mbar_wait(&mb_full[g], (uint32_t)((j >> 1) & 1), p.status);
            tc::fence_after();
            const int c = (int)((s0 + j) / p.T);
            if (c != cur_c) {
                flush(cur_c, seg);
                seg++;
                cur_c = c;
            }
#pragma unroll
            for (int cc = 0; cc < 2; cc++) {
                const uint32_t col = 256u + (uint32_t)g * 128u + (uint32_t)(32 * h + 16 * cc);
                uint32_t rr[16], ri[16];
                tc::tmem_ld16(tmem + lane_base + col, rr);
                tc::tmem_ld16(tmem + lane_base + col + 64, ri);
                tc::tmem_wait_ld();
#pragma unroll
                for (int t = 0; t < 16; t++) {
                    const float fr = __uint_as_float(rr[t]), fi = __uint_as_float(ri[t]);
                    acc_a[16 * cc + t] = fmaf(fr, fr, fmaf(fi, fi, acc_a[16 * cc + t]));
                }
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    // own value at row 2k + pol, partner's value at the same row
                    const float e_r = __uint_as_float(rr[2 * k]), e_i = __uint_as_float(ri[2 * k]);
                    const float o_r = __uint_as_float(rr[2 * k + 1]), o_i = __uint_as_float(ri[2 * k + 1]);
                    const float mr = pol ? o_r : e_r, mi = pol ? o_i : e_i;
                    const float sr = __shfl_xor_sync(0xffffffffu, pol ? e_r : o_r, 16);
                    const float si = __shfl_xor_sync(0xffffffffu, pol ? e_i : o_i, 16);
                    const int a = 2 * (8 * cc + k);
                    acc_x[a] = fmaf(mr, sr, fmaf(mi, si, acc_x[a]));            // Re own conj(other)
                    acc_x[a + 1] = fmaf(mi, sr, fmaf(-mr, si, acc_x[a + 1]));   // Im own conj(other)
                }
            }
            tc::fence_before();
            tc::mbar_arrive(&mb_empty[g]);
        }
        if (nsamp > 0) flush(cur_c, seg);
    }

    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

size_t smem_bytes(int ne, int ntile, int nent) {
    const uint32_t vstage = (8u * ne + 15u) & ~15u;
    return kOffE + 32ull * ne + (size_t)kStages * vstage + (table_layout(ntile, nent).bytes - kOpBytes);
}

}  // namespace

bool epic_tc_supported(const hai_layout *L) {
    return L->grid_n == kN && L->n_pol == 2 && L->box_w <= kBox && L->box_h <= kBox && L->n_elem <= 65535;
}

// Tables of the tensor-core path: the DFT operand of both stages,
// B[n][kappa] with n = (out re/im, l) and kappa = (j, in re/im), in the
// K-major layout (W'[j][l] = (-1)^j exp(+2 pi i l j / 64)); and the gather
// tiles of the non-empty cells (see TableLayout).
void epic_tc_build_table(const hai_layout *L, const std::vector<int32_t> &cstart,
                         const std::vector<int32_t> &elem, const std::vector<float2> &w,
                         std::vector<uint8_t> &out, int &ntile, int &nent) {
    std::vector<int> cells;
    for (int y = 0; y < L->box_h; y++)
        for (int x = 0; x < L->box_w; x++)
            if (cstart[y * L->box_w + x + 1] > cstart[y * L->box_w + x]) cells.push_back(y * L->box_w + x);
    auto count = [&](int c) { return cstart[c + 1] - cstart[c]; };
    auto a1off = [&](int cell) {
        const int y = cell / L->box_w, x = cell % L->box_w;
        return tc::off_kmajor(y, 2 * x, kKs, kMNs);
    };
    std::stable_sort(cells.begin(), cells.end(), [&](int a, int b) {
        if (count(a) != count(b)) return count(a) > count(b);
        return a1off(a) < a1off(b);
    });
    ntile = ((int)cells.size() + 31) / 32;
    std::vector<int> base(ntile + 1, 0);
    for (int t = 0; t < ntile; t++) {
        int slots = 0;
        for (int l = 0; l < 32 && t * 32 + l < (int)cells.size(); l++) slots = std::max(slots, count(cells[t * 32 + l]));
        base[t + 1] = base[t] + 32 * slots;
    }
    nent = base[ntile];
    const TableLayout tl = table_layout(ntile, nent);
    out.assign(tl.bytes, 0);
    for (int n = 0; n < 128; n++)
        for (int kappa = 0; kappa < 2 * kBox; kappa++) {
            const int j = kappa >> 1, c = kappa & 1, l = n & 63, im_out = n >> 6;
            const double ang = 2.0 * 3.14159265358979323846 * (double)((l * j) % kN) / kN;
            const double sgn = (j & 1) ? -1.0 : 1.0;
            const double wr = sgn * cos(ang), wi = sgn * sin(ang);
            const double v = im_out ? (c == 0 ? wi : wr) : (c == 0 ? wr : -wi);
            const __half hv = __double2half(v);
            memcpy(&out[tc::off_kmajor(n, kappa, kKs, kMNs)], &hv, 2);
        }
    uint32_t *o_cell = reinterpret_cast<uint32_t *>(&out[tl.off_cell]);
    int32_t *o_base = reinterpret_cast<int32_t *>(&out[tl.off_base]);
    float2 *o_w = reinterpret_cast<float2 *>(&out[tl.off_w]);
    uint16_t *o_e = reinterpret_cast<uint16_t *>(&out[tl.off_e]);
    for (int t = 0; t <= ntile; t++) o_base[t] = base[t];
    for (int t = 0; t < ntile; t++)
        for (int l = 0; l < 32; l++) {
            const int ci = t * 32 + l;
            if (ci >= (int)cells.size()) {
                o_cell[ci] = 0xffffffffu;
                continue;
            }
            const int cell = cells[ci];
            o_cell[ci] = a1off(cell);
            for (int k = 0; k < count(cell); k++) {
                const int q = base[t] + 32 * k + l;
                o_w[q] = w[cstart[cell] + k];                 // conj(W~) = a + ib
                o_e[q] = (uint16_t)elem[cstart[cell] + k];
            }
        }
}

hai_status epic_tc_launch(const hai_layout *L, const int8_t *volt, int C, int T, float *img, int accumulate,
                          cudaStream_t st) {
    if (!epic_tc_supported(L) || !L->d_tc_tables)
        return hai_fail(HAI_ERR_UNSUPPORTED,
                        "epic fp16: this build's tensor-core path needs N = 64, 2 pols and a kernel box <= 32 x 32");
    const size_t smem = smem_bytes(L->n_elem, L->tc_ntile, L->tc_nent);
    if (smem > (size_t)L->ctx->smem_optin)
        return hai_fail(HAI_ERR_UNSUPPORTED, "epic fp16: shared memory need exceeds the device limit");
    HAI_CUDA_TRY(cudaFuncSetAttribute(epic_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const EpicSplit sp = epic_make_split(C, T, L->ctx->num_sms);
    if (!sp.direct && (size_t)sp.n_cta * 2 > L->partial_slots)
        return hai_fail(HAI_ERR_INVALID_ARG, "epic fp16: partial buffer too small");
    EpicTcParams p;
    p.volt = volt;
    p.C = C;
    p.T = T;
    p.ne = L->n_elem;
    p.len = sp.len;
    p.ntile = L->tc_ntile;
    p.nent = L->tc_nent;
    p.table = static_cast<const uint8_t *>(L->d_tc_tables);
    p.out = sp.direct ? img : L->d_partials;
    p.direct = sp.direct;
    p.accumulate = accumulate;
    p.use_tma = ((4 * L->n_elem) % 16 == 0) && ((((uintptr_t)volt) & 15) == 0);
    p.status = L->ctx->d_status;
    const int pidx = prof_begin(L->ctx, st);
    epic_tc_kernel<<<sp.n_cta, kThreads, smem, st>>>(p);
    prof_end(L->ctx, pidx, st);
    prof_count(L->ctx, 1);
    HAI_CUDA_TRY(cudaGetLastError());
    if (!sp.direct) return epic_reduce_launch(L, sp, C, T, img, accumulate, st);
    return HAI_OK;
}
