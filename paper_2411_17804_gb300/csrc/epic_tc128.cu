// EPIC direct imager on tcgen05 tensor cores for grid side N = 128 (Eq.
// intra-station EPIC, squaring and temporal sum of Eq. intra-station
// squaring), FP16 operands, FP32 accumulation.
//
// At N = 128 the accumulated image of one channel (XX, YY, XY: 4 x 128^2
// FP32 = 256 KB) no longer fits one SM, so a cluster of four CTAs images
// each channel, CTA r owning the output columns l_x in [32 r, 32 r + 32):
//   stage 1 (per CTA):  H[y][l_x] = sum_x G[y][x] W'[x][l_x] for its l_x only
//                       (M = 128 rows (pol, y), N = 64 columns (re/im, l_x),
//                       K = 128 (x, re/im));
//   stage 2 (per CTA):  F[l_y][l_x] = sum_y W'[y][l_y] H[y][l_x] with the
//                       constant DFT matrix as operand A (M = 128 rows l_y)
//                       and the stage-1 result as operand B (N = 128 columns
//                       (pol, re/im, l_x), MN-major), so each epilogue thread
//                       holds X and Y of the same pixels.
// Nothing is computed twice except the stage-1 input: every CTA needs the
// whole gridded field G.  The box (<= 64 rows) is cut into eight 8-row
// groups, dealt to the four CTAs to balance their gather entries; each CTA
// grids its groups into its own copy of G, then the lanes of one warp send
// them to the three other CTAs at once with shared-to-shared bulk copies
// that complete on the receiver's mbarrier.  Each CTA's MMA warp reports the
// end of its stage-1 MMAs to every CTA of the cluster (multicast commit),
// which frees that G buffer for the next-but-one step.  Only a group's owner
// ever writes its rows, in any copy.
//
// Roles as in the N = 32/64 kernel: warps 0-6 front (voltages, gridding,
// warps 0-3 also move stage-1 results from TMEM into operand B2), warp 7 TMA
// and MMA issue, warps 8-15 epilogue (register accumulators, 64 per thread).
// One sample per step.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "epic_tc.cuh"
#include "hai_internal.h"
#include "tc.cuh"

namespace {

constexpr int kN = 128;
constexpr int kNN = kN * kN;
constexpr int kThreads = 512;
constexpr int kFront = 224;
constexpr int kMmaWarp = 7;
constexpr int kEpi = 256;
constexpr int kStages = 4;
constexpr int kRanks = 4;
constexpr int kSendWarp = 6;                 // front warp that ships G rows to the peers
constexpr uint32_t kKs = 128;                // K-major: K-group stride
constexpr uint32_t kMNs = 16 * kKs;          // K-major, K = 128: MN-group stride (2048)
constexpr uint32_t kGroupBytes = kMNs;       // 8 rows of a K-major operand
constexpr uint32_t kB1Bytes = 8 * kMNs;      // 64 rows (re/im, 32 l_x)
constexpr uint32_t kA2Bytes = 16 * kMNs;     // 128 rows l_y
constexpr uint32_t kA1Bytes = 16 * kMNs;     // 128 rows (pol, y)
constexpr uint32_t kPolBytes = 8 * kMNs;     // 64 rows of one pol
constexpr uint32_t kB2Ks = 2064;             // MN-major B2: K-group stride (16 groups + 16 B pad)
constexpr uint32_t kB2MNs = 128;             // MN-major B2: MN-group stride
constexpr uint32_t kB2Bytes = 16 * kB2Ks;
constexpr uint32_t kOffA2 = kB1Bytes;
constexpr uint32_t kOffA1 = kOffA2 + kA2Bytes;
constexpr uint32_t kOffB2 = kOffA1 + 2 * kA1Bytes;
constexpr uint32_t kOffE = kOffB2 + kB2Bytes;
constexpr uint32_t kD2Col = 128;             // TMEM: D1 at 0 / 64, D2 at 128 / 256

// Header of a station's gather blob (N = 128): per rank the byte offset,
// size, tiles and entries of its gather table (GatherLayout), and the owner
// rank of each 8-row group of the box.
struct Blob128 {
    uint32_t off[kRanks], bytes[kRanks];
    int32_t ntile[kRanks], nent[kRanks];
    uint8_t owner[8];
    int32_t box_w, box_h;       // kernel box of the station (cells)
    uint8_t pad[48];
};
static_assert(sizeof(Blob128) == 128, "blob header");

struct Params {
    const int8_t *volt;
    float *img;
    const TcStation *stations;
    const uint8_t *dft;
    const long long *cta_begin;   // per group
    long long len, total;
    int C, T;
    int ne_max;
    uint32_t vstage;
    int direct, accumulate, use_tma, guard;
    float *partials;
    unsigned *status;
};

__device__ __forceinline__ void bar_front() { asm volatile("bar.sync 1, 224;" ::: "memory"); }

template <bool BF>
__global__ void __cluster_dims__(kRanks, 1, 1) __launch_bounds__(kThreads, 1) epic_tc128_kernel(const Params p) {
    // operand type of both MMA operands: FP16, or BF16 when BF
    constexpr uint32_t kIdesc1 = tc::idesc_f16_as(BF, 128, 64, 0, 0);
    constexpr uint32_t kIdesc2 = tc::idesc_f16_as(BF, 128, 128, 0, 1);
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mb_v[kStages];
    __shared__ __align__(8) uint64_t mb_a1[2], mb_a1free[2], mb_d1[2], mb_a2, mb_b2free, mb_full[2], mb_empty[2];
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t rank = tc::cluster_rank();
    const int group = blockIdx.x / kRanks;
    uint8_t *sB1 = smem;
    uint8_t *sA2 = smem + kOffA2;
    uint8_t *sA1 = smem + kOffA1;
    uint8_t *sB2 = smem + kOffB2;
    uint2 *sE = reinterpret_cast<uint2 *>(smem + kOffE);   // [2][ne_max]: X, Y as half2
    const uint32_t off_v = kOffE + 2u * 8u * ((p.ne_max + 1) & ~1);
    int8_t *sV = reinterpret_cast<int8_t *>(smem + off_v);
    uint8_t *sT = smem + off_v + kStages * p.vstage;

    // ---- set-up: this CTA's stage-1 DFT columns and the stage-2 DFT matrix
    for (int i = tid; i < (int)(kB1Bytes / 16); i += kThreads)
        reinterpret_cast<int4 *>(sB1)[i] = __ldg(reinterpret_cast<const int4 *>(p.dft + rank * kB1Bytes) + i);
    for (int i = tid; i < (int)(kA2Bytes / 16); i += kThreads)
        reinterpret_cast<int4 *>(sA2)[i] = __ldg(reinterpret_cast<const int4 *>(p.dft + kRanks * kB1Bytes) + i);
    if (tid == 0) {
        for (int s = 0; s < kStages; s++) tc::mbar_init(&mb_v[s], 1);
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&mb_a1[b], 1);
            tc::mbar_init(&mb_a1free[b], kRanks);
            tc::mbar_init(&mb_d1[b], 1);
            tc::mbar_init(&mb_full[b], 1);
            tc::mbar_init(&mb_empty[b], kEpi);
        }
        tc::mbar_init(&mb_a2, 128);
        tc::mbar_init(&mb_b2free, 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot, 512);
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::cluster_sync();                    // peers' barriers exist before any remote arrival
    tc::fence_after();
    const uint32_t tmem = tmem_slot;

    const long long s0 = p.cta_begin ? p.cta_begin[group] : (long long)group * p.len;
    const long long s1 = p.cta_begin ? p.cta_begin[group + 1] : min(s0 + p.len, p.total);
    const int nsteps = (int)max(0ll, s1 - s0);

    if (warp < kMmaWarp) {
        // ================================================================ front
        int cur_station = -1, ne = 0, ntile = 0;
        int a1_st0 = -1, a1_st1 = -1;          // station whose cells buffer 0 / 1 holds
        uint32_t own_mask = 0, incoming = 0;
        uint32_t box_mask = 0, copy_bytes = 0;    // groups inside the box; bytes of a group's box columns
        bool dead = false;                     // a wait of this thread gave up: send nothing more
        const uint32_t *s_cell = nullptr;
        const int32_t *s_base = nullptr, *s_warp = nullptr;
        const float2 *s_w = nullptr;
        const uint16_t *s_e = nullptr;

        auto prepare = [&](int stn, int b) {
            if (stn == cur_station && (b ? a1_st1 : a1_st0) == stn) return;
            bar_front();
            if (stn != cur_station) {
                const TcStation st = p.stations[stn];
                const Blob128 *hd = reinterpret_cast<const Blob128 *>(st.table);
                const uint32_t off = hd->off[rank], bytes = hd->bytes[rank];
                for (int k = tid; k < (int)(bytes / 16); k += kFront)
                    reinterpret_cast<int4 *>(sT)[k] = __ldg(reinterpret_cast<const int4 *>(st.table + off) + k);
                const GatherLayout gl = gather_layout(hd->ntile[rank], hd->nent[rank]);
                s_cell = reinterpret_cast<const uint32_t *>(sT + gl.off_cell);
                s_base = reinterpret_cast<const int32_t *>(sT + gl.off_base);
                s_warp = reinterpret_cast<const int32_t *>(sT + gl.off_warp);
                s_w = reinterpret_cast<const float2 *>(sT + gl.off_w);
                s_e = reinterpret_cast<const uint16_t *>(sT + gl.off_e);
                ntile = hd->ntile[rank];
                ne = st.ne;
                own_mask = 0;
                for (int g = 0; g < 8; g++)
                    if (hd->owner[g] == rank) own_mask |= 1u << g;
                box_mask = 0;
                for (int g = 0; g < 8; g++)
                    if (8 * g < hd->box_h) box_mask |= 1u << g;
                // K-groups (8 values: 4 cells of (re, im)) that hold box columns
                copy_bytes = (uint32_t)((2 * hd->box_w + 7) / 8) * kKs;
                incoming = (uint32_t)__popc(box_mask & ~own_mask) * 2u * copy_bytes;
                cur_station = stn;
            }
            if ((b ? a1_st1 : a1_st0) != stn) {
                // zero what no other CTA writes into this copy: own groups, groups
                // outside the box, and the columns past the box of every group
                uint8_t *A = sA1 + b * kA1Bytes;
                for (int k = tid; k < (int)(16 * kGroupBytes / 16); k += kFront) {
                    const uint32_t byte = (uint32_t)k * 16u;
                    const int g = (byte / kGroupBytes) & 7;
                    const uint32_t in_group = byte % kGroupBytes;
                    if ((own_mask & (1u << g)) || !(box_mask & (1u << g)) || in_group >= copy_bytes)
                        reinterpret_cast<int4 *>(A)[k] = make_int4(0, 0, 0, 0);
                }
                (b ? a1_st1 : a1_st0) = stn;
            }
            bar_front();
        };
        auto stage_volt = [&](const TcStep &s, int i) {
            const int8_t *V;
            uint32_t delta;
            const int8_t *src = tc_aligned_src(s.src, p.guard, delta);
            if (p.use_tma) {
                tc::mbar_wait(&mb_v[i % kStages], (uint32_t)((i / kStages) & 1), p.status);
                V = sV + (i % kStages) * p.vstage + delta;
            } else {
                int8_t *dst = sV + (i % kStages) * p.vstage;
                for (int b = tid; b < 4 * ne; b += kFront) dst[b] = src[b];
                bar_front();
                V = dst;
            }
            uint2 *E = sE + (size_t)(i & 1) * ((p.ne_max + 1) & ~1);
            const char2 *v2 = reinterpret_cast<const char2 *>(V);
            for (int a = tid; a < ne; a += kFront) {
                const char2 x = v2[a], y = v2[ne + a];
                E[a] = make_uint2(tc::pack_half2((float)x.x, (float)x.y), tc::pack_half2((float)y.x, (float)y.y));
            }
            bar_front();
        };
        auto grid_step = [&](int i) {
            uint8_t *A = sA1 + (i & 1) * kA1Bytes;
            const uint2 *E = sE + (size_t)(i & 1) * ((p.ne_max + 1) & ~1);
            for (int t = s_warp[warp]; t < s_warp[warp + 1]; t++) {
                float2 g0 = make_float2(0.f, 0.f), g1 = g0;
                const int qe = s_base[t + 1];
                // (re, im) += conj(W~) e per pol as packed FMAs, the roundings of
                // fmaf(w.x, x.x, fmaf(-w.y, x.y, re)) and fmaf(w.x, x.y, fmaf(w.y, x.x, im))
                auto mac = [&](const float2 w, const uint2 e) {
                    const float2 x = __half22float2(*reinterpret_cast<const __half2 *>(&e.x));
                    const float2 y = __half22float2(*reinterpret_cast<const __half2 *>(&e.y));
                    const float2 wr = make_float2(w.x, w.x), wi = make_float2(-w.y, w.y);
                    g0 = __ffma2_rn(wr, x, __ffma2_rn(wi, make_float2(x.y, x.x), g0));
                    g1 = __ffma2_rn(wr, y, __ffma2_rn(wi, make_float2(y.y, y.x), g1));
                };
                // the lane's slots q, q + 32, ...: four at a time with every
                // shared-memory load issued before the first use
                int q = s_base[t] + lane;
                for (; q + 96 < qe; q += 128) {
                    float2 w[4];
                    int en[4];
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        w[j] = s_w[q + 32 * j];
                        en[j] = s_e[q + 32 * j];
                    }
                    uint2 e[4];
#pragma unroll
                    for (int j = 0; j < 4; j++) e[j] = E[en[j]];
#pragma unroll
                    for (int j = 0; j < 4; j++) mac(w[j], e[j]);
                }
                for (; q < qe; q += 32) mac(s_w[q], E[s_e[q]]);
                const uint32_t off = s_cell[t * 32 + lane];
                if (off != 0xffffffffu) {
                    *reinterpret_cast<uint32_t *>(A + off) = tc::pack2<BF>(g0.x, g0.y);
                    *reinterpret_cast<uint32_t *>(A + off + kPolBytes) = tc::pack2<BF>(g1.x, g1.y);
                }
            }
        };
        // warp 6: the box columns of the own in-box row groups of G -> the
        // three other CTAs, one bulk copy per lane (peer, group, pol); then
        // this CTA's own arrival, expecting the bytes the others send
        auto send = [&](int i) {
            const int b = i & 1;
            uint8_t *A = sA1 + b * kA1Bytes;
            const uint32_t mine = own_mask & box_mask;
            const int n_own = __popc(mine);
            if (!dead)
                for (int c = lane; c < (kRanks - 1) * n_own * 2; c += 32) {
                    const int pol = c & 1, k = (c >> 1) % n_own, pi = (c >> 1) / n_own;
                    const uint32_t peer = (uint32_t)pi + (pi >= (int)rank ? 1u : 0u);
                    int g = -1;
                    for (int x = 0, seen = 0; x < 8; x++)
                        if (mine & (1u << x)) {
                            if (seen == k) g = x;
                            seen++;
                        }
                    const uint32_t off = (uint32_t)pol * kPolBytes + (uint32_t)g * kGroupBytes;
                    tc::bulk_s2peer(tc::peer_addr(tc::smem_u32(A + off), peer), A + off, copy_bytes,
                                    tc::peer_addr(tc::smem_u32(&mb_a1[b]), peer));
                }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive_expect_tx(&mb_a1[b], incoming);
        };
        // warps 0-3: D1 row (pol, y) -> column (y, re/im) of B2 for the
        // rows (pol, out re/im, l_x): out re <- (H_r, -H_i), out im <- (H_i, H_r)
        auto convert = [&](int i) {
            const int pol = warp >> 1, y = 32 * (warp & 1) + lane;
            const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(i & 1) * 64u;
#pragma unroll
            for (int hh = 0; hh < 2; hh++) {               // l_x in [16 hh, 16 hh + 16)
                uint32_t hr[16], hi[16];
                tc::tmem_ld16(base + 16 * hh, hr);
                tc::tmem_ld16(base + 32 + 16 * hh, hi);
                tc::tmem_wait_ld();
#pragma unroll
                for (int c_in = 0; c_in < 2; c_in++) {
                    const int kappa = 2 * y + c_in;
#pragma unroll
                    for (int c_out = 0; c_out < 2; c_out++) {
#pragma unroll
                        for (int h = 0; h < 2; h++) {        // 8 columns l_x -> one 16-byte row
                            float v[8];
#pragma unroll
                            for (int e = 0; e < 8; e++) {
                                const float r = __uint_as_float(hr[8 * h + e]), im = __uint_as_float(hi[8 * h + e]);
                                v[e] = c_out == 0 ? (c_in == 0 ? r : -im) : (c_in == 0 ? im : r);
                            }
                            const int n2 = pol * 64 + c_out * 32 + 16 * hh + 8 * h;
                            uint4 u;
                            u.x = tc::pack2<BF>(v[0], v[1]);
                            u.y = tc::pack2<BF>(v[2], v[3]);
                            u.z = tc::pack2<BF>(v[4], v[5]);
                            u.w = tc::pack2<BF>(v[6], v[7]);
                            *reinterpret_cast<uint4 *>(sB2 + tc::off_mnmajor(n2, kappa, kB2Ks, kB2MNs)) = u;
                        }
                    }
                }
            }
        };
        TcWalker wk;
        wk.init(p.volt, p.stations, p.C, p.T, s0, s1);
        for (int i = -1; i < nsteps; i++) {
            if (i + 1 < nsteps) {
                const int j = i + 1, b = j & 1;
                const TcStep s = wk.next(1);
                // G buffer b was last read by the stage-1 MMAs of step j - 2 in every CTA
                if (j >= 2 && !tc::mbar_wait_cluster(&mb_a1free[b], (uint32_t)(((j >> 1) - 1) & 1), p.status))
                    dead = true;
                prepare(s.stn, b);
                stage_volt(s, j);
                grid_step(j);
                tc::fence_proxy_async();
                bar_front();
                if (warp == kSendWarp) send(j);
            }
            if (i >= 0 && warp < 4) {
                tc::mbar_wait(&mb_d1[i & 1], (uint32_t)((i >> 1) & 1), p.status);
                if (i >= 1) tc::mbar_wait(&mb_b2free, (uint32_t)((i - 1) & 1), p.status);
                tc::fence_after();
                convert(i);
                tc::fence_proxy_async();
                tc::fence_before();
                tc::mbar_arrive(&mb_a2);
            }
        }
    } else if (warp == kMmaWarp) {
        // ================================================================ MMA + TMA
        if (lane == 0) {
            const uint32_t b1 = tc::smem_u32(sB1), a2 = tc::smem_u32(sA2), b2 = tc::smem_u32(sB2);
            int n_loaded = 0;
            TcWalker ld;
            ld.init(p.volt, p.stations, p.C, p.T, s0, s1);
            auto issue_load = [&]() {
                if (n_loaded >= nsteps || !p.use_tma) return;
                const TcStep s = ld.next(1);
                uint32_t delta;
                const int8_t *src = tc_aligned_src(s.src, p.guard, delta);
                const uint32_t bytes = (delta + 4u * s.ne + 15u) & ~15u;
                const int sg = n_loaded % kStages;
                tc::mbar_arrive_expect_tx(&mb_v[sg], bytes);
                tc::bulk_g2s(sV + sg * p.vstage, src, bytes, &mb_v[sg]);
                n_loaded++;
            };
            for (int q = 0; q < kStages; q++) issue_load();
            for (int k = -1; k < nsteps; k++) {
                if (k >= 0) {                      // stage 2 of step k
                    tc::mbar_wait(&mb_a2, (uint32_t)(k & 1), p.status);
                    const int slot = k & 1;
                    if (k >= 2) tc::mbar_wait(&mb_empty[slot], (uint32_t)(((k >> 1) - 1) & 1), p.status);
                    tc::fence_after();
                    const uint32_t d = tmem + kD2Col + (uint32_t)slot * 128u;
#pragma unroll
                    for (int s = 0; s < 8; s++)
                        tc::mma_f16(d, tc::desc(a2 + s * 2 * kKs, kKs, kMNs), tc::desc(b2 + s * 2 * kB2Ks, kB2Ks, kB2MNs),
                                    kIdesc2, s > 0);
                    tc::mma_commit(&mb_full[slot]);
                    tc::mma_commit(&mb_b2free);
                }
                if (k + 1 < nsteps) {              // stage 1 of step k+1
                    const int i = k + 1;
                    tc::mbar_wait_cluster(&mb_a1[i & 1], (uint32_t)((i >> 1) & 1), p.status);
                    issue_load();
                    tc::fence_after();
                    const uint32_t a = tc::smem_u32(sA1 + (i & 1) * kA1Bytes);
                    const uint32_t d = tmem + (uint32_t)(i & 1) * 64u;
#pragma unroll
                    for (int s = 0; s < 8; s++)
                        tc::mma_f16(d, tc::desc(a + s * 2 * kKs, kKs, kMNs), tc::desc(b1 + s * 2 * kKs, kKs, kMNs),
                                    kIdesc1, s > 0);
                    tc::mma_commit(&mb_d1[i & 1]);
                    // every CTA waits for this only before step i + 2
                    if (i + 2 < nsteps) tc::mma_commit_multicast(&mb_a1free[i & 1], (uint16_t)((1u << kRanks) - 1));
                }
            }
        }
    } else {
        // ============================================================= epilogue
        const int q = warp & 3, h = (warp - 8) >> 2;
        const int ly = 32 * q + lane;
        const int lx0 = 32 * (int)rank + 16 * h;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        // packed accumulators: pw[t] = (|X|^2, |Y|^2), cx[t] = (Re, Im) X conj(Y)
        float2 pw[16], cx[16];
#pragma unroll
        for (int t = 0; t < 16; t++) pw[t] = cx[t] = make_float2(0.f, 0.f);
        int seg = 0;
        long long cur_blk = -1;
        auto flush = [&](int stn, int c, int sgm) {
            float *dst = p.direct ? p.img + p.stations[stn].img_off + (size_t)c * 4 * kNN
                                  : p.partials + ((size_t)group * 2 + sgm) * 4 * kNN;
            // plane pl: component c (0 = .x, 1 = .y) of the pairs in a
            auto put = [&](int pl, const float2 (&a)[16], int c) {
                float4 *d4 = reinterpret_cast<float4 *>(dst + (size_t)pl * kNN + (size_t)ly * kN + lx0);
#pragma unroll
                for (int v = 0; v < 4; v++) {
                    float4 o = c ? make_float4(a[4 * v].y, a[4 * v + 1].y, a[4 * v + 2].y, a[4 * v + 3].y)
                                 : make_float4(a[4 * v].x, a[4 * v + 1].x, a[4 * v + 2].x, a[4 * v + 3].x);
                    if (p.direct && p.accumulate) {
                        const float4 old = d4[v];
                        o.x += old.x;
                        o.y += old.y;
                        o.z += old.z;
                        o.w += old.w;
                    }
                    d4[v] = o;
                }
            };
            put(0, pw, 0);
            put(1, pw, 1);
            put(2, cx, 0);
            put(3, cx, 1);
#pragma unroll
            for (int t = 0; t < 16; t++) pw[t] = cx[t] = make_float2(0.f, 0.f);
        };
        TcWalker wk;
        wk.init(p.volt, p.stations, p.C, p.T, s0, s1);
        int cur_stn = 0, cur_chan = 0;
        for (int k = 0; k < nsteps; k++) {
            const TcStep s = wk.next(1);
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
            const int slot = k & 1;
            tc::mbar_wait(&mb_full[slot], (uint32_t)((k >> 1) & 1), p.status);
            tc::fence_after();
            const uint32_t col = kD2Col + (uint32_t)slot * 128u + 16u * h;
#pragma unroll
            for (int qt = 0; qt < 4; qt++) {                // 4 columns l_x at a time
                uint32_t ar[4], ai[4], br[4], bi[4];
                tc::tmem_ld4(tmem + lane_base + col + 4 * qt, ar);         // X re
                tc::tmem_ld4(tmem + lane_base + col + 4 * qt + 32, ai);    // X im
                tc::tmem_ld4(tmem + lane_base + col + 4 * qt + 64, br);    // Y re
                tc::tmem_ld4(tmem + lane_base + col + 4 * qt + 96, bi);    // Y im
                tc::tmem_wait_ld();
                if (qt == 3) {
                    tc::fence_before();
                    tc::mbar_arrive(&mb_empty[slot]);
                }
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const int t = 4 * qt + e;
                    const float a_r = __uint_as_float(ar[e]), a_i = __uint_as_float(ai[e]);
                    const float b_r = __uint_as_float(br[e]), b_i = __uint_as_float(bi[e]);
                    // |X|^2 = fmaf(a_r, a_r, fmaf(a_i, a_i, .)), |Y|^2 likewise;
                    // Re X conj(Y) = fmaf(a_r, b_r, fmaf(a_i, b_i, .)),
                    // Im X conj(Y) = fmaf(a_i, b_r, fmaf(-a_r, b_i, .)): packed pairs
                    const float2 re = make_float2(a_r, b_r), im = make_float2(a_i, b_i);
                    pw[t] = __ffma2_rn(re, re, __ffma2_rn(im, im, pw[t]));
                    cx[t] = __ffma2_rn(make_float2(a_r, a_i), make_float2(b_r, b_r),
                                       __ffma2_rn(make_float2(a_i, -a_r), make_float2(b_i, b_i), cx[t]));
                }
            }
        }
        if (cur_blk >= 0) flush(cur_stn, cur_chan, seg);
    }

    tc::fence_before();
    __syncthreads();
    tc::cluster_sync();                    // no copy or arrival targets this CTA any more
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

uint32_t vstage_bytes(int ne_max) { return (4u * ne_max + 16u + 15u) & ~15u; }

}  // namespace

size_t epic_tc128_smem(int ne_max, uint32_t table_max) {
    return kOffE + 16ull * ((ne_max + 1) & ~1) + (size_t)kStages * vstage_bytes(ne_max) + table_max;
}

// Gather blob of one station for the N = 128 kernel: the box's 8-row groups
// dealt to the four ranks (largest entry count first, to the least loaded
// rank), then one gather table per rank with the cells of its groups.
void epic_tc128_build_blob(int box_w, int box_h, const std::vector<int32_t> &cstart,
                           const std::vector<int32_t> &elem, const std::vector<float2> &w,
                           std::vector<uint8_t> &out, uint32_t &max_rank_bytes, long long &max_rank_entries) {
    long long cnt[8] = {0};
    for (int y = 0; y < box_h; y++)
        for (int x = 0; x < box_w; x++) cnt[y / 8] += cstart[y * box_w + x + 1] - cstart[y * box_w + x];
    int order[8];
    for (int g = 0; g < 8; g++) order[g] = g;
    std::stable_sort(order, order + 8, [&](int a, int b) { return cnt[a] > cnt[b]; });
    long long load[kRanks] = {0};
    int ngroups[kRanks] = {0};
    uint8_t owner[8];
    for (int k = 0; k < 8; k++) {
        int best = 0;
        for (int r = 1; r < kRanks; r++)
            if (load[r] < load[best] || (load[r] == load[best] && ngroups[r] < ngroups[best])) best = r;
        owner[order[k]] = (uint8_t)best;
        load[best] += cnt[order[k]];
        ngroups[best]++;
    }
    Blob128 hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.owner, owner, 8);
    hd.box_w = box_w;
    hd.box_h = box_h;
    std::vector<std::vector<uint8_t>> tabs(kRanks);
    max_rank_bytes = 0;
    max_rank_entries = 0;
    for (int r = 0; r < kRanks; r++) {
        // CSR restricted to the rank's rows (other cells empty)
        std::vector<int32_t> cs(cstart.size(), 0);
        std::vector<int32_t> el;
        std::vector<float2> ww;
        for (int y = 0; y < box_h; y++)
            for (int x = 0; x < box_w; x++) {
                const int c = y * box_w + x;
                if (owner[y / 8] == r)
                    for (int k = cstart[c]; k < cstart[c + 1]; k++) {
                        el.push_back(elem[k]);
                        ww.push_back(w[k]);
                    }
                cs[c + 1] = (int32_t)el.size();
            }
        // warp 6 sends the rows to the other CTAs instead of gridding
        epic_tc_build_gather(box_w, box_h, cs, el, ww, kKs, kMNs, tabs[r], hd.ntile[r], hd.nent[r], kGatherWarps - 1);
        hd.bytes[r] = (uint32_t)tabs[r].size();
        max_rank_bytes = std::max(max_rank_bytes, hd.bytes[r]);
        max_rank_entries = std::max<long long>(max_rank_entries, hd.nent[r]);
    }
    uint32_t off = sizeof(Blob128);
    for (int r = 0; r < kRanks; r++) {
        hd.off[r] = off;
        off += hd.bytes[r];
    }
    out.assign(off, 0);
    memcpy(out.data(), &hd, sizeof(hd));
    for (int r = 0; r < kRanks; r++) memcpy(out.data() + hd.off[r], tabs[r].data(), tabs[r].size());
}

hai_status epic_tc128_run(hai_ctx *ctx, const TcLaunch &l, cudaStream_t st) {
    const size_t smem = epic_tc128_smem(l.ne_max, l.table_max);
    if (smem + kStaticSmem > (size_t)ctx->smem_optin)
        return hai_fail(HAI_ERR_UNSUPPORTED, "epic fp16 (N = 128): shared memory need exceeds the device limit");
    const void *dft = epic_tc_dft(ctx, 128, l.bf16 != 0);
    if (!dft) return hai_fail(HAI_ERR_INVALID_ARG, "epic tensor cores (N = 128): DFT operand not prepared");
    if (!l.no_attr) {
        const hai_status s = epic_tc128_set_attr(ctx);
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
    p.vstage = vstage_bytes(l.ne_max);
    p.direct = l.direct;
    p.accumulate = l.accumulate;
    p.guard = l.guard;
    p.use_tma = l.guard || (((uintptr_t)l.volt & 15) == 0 && (4 * l.ne_max) % 16 == 0 && l.n_station == 1);
    p.partials = l.partials;
    p.status = ctx->d_status;
    const int pidx = prof_begin(ctx, st);
    if (l.bf16) epic_tc128_kernel<true><<<l.n_cta * kRanks, kThreads, smem, st>>>(p);
    else epic_tc128_kernel<false><<<l.n_cta * kRanks, kThreads, smem, st>>>(p);
    prof_end(ctx, pidx, st);
    prof_count(ctx, 1);
    HAI_CUDA_TRY(cudaGetLastError());
    return HAI_OK;
}

hai_status epic_tc128_set_attr(hai_ctx *ctx) {
    HAI_CUDA_TRY(hai_allow_dyn_smem(epic_tc128_kernel<false>, ctx->smem_optin));
    HAI_CUDA_TRY(hai_allow_dyn_smem(epic_tc128_kernel<true>, ctx->smem_optin));
    return HAI_OK;
}

// Clusters of four of this kernel that can be resident at once.
int epic_tc128_max_groups(hai_ctx *ctx, int ne_max, uint32_t table_max) {
    const size_t smem = epic_tc128_smem(ne_max, table_max);
    if (smem + kStaticSmem > (size_t)ctx->smem_optin) return 0;
    if (epic_tc128_set_attr(ctx) != HAI_OK) return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kRanks * 64, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = kRanks;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, epic_tc128_kernel<false>, &cfg) != cudaSuccess) return 0;
    return n;
}
