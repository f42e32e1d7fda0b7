// Correlator (Eq. intra-station visibilities): V^{pq}_{ab} = sum_t E^p_a conj(E^q_b)
// for all element pairs a >= b, on tcgen05 tensor cores with exact integer
// results.
//
// Per channel the voltages form a real matrix X[m][k] with rows m = (pol,
// element) and columns k = (sample, re/im).  For rows (elements a) and
// columns (elements b):
//   Re V = sum_k X_a[k] X_b[k],   Im V = sum_k X_a[k] X'_b[k],
// where X'_b = (-Im, Re) per sample, so B = [X_b ; X'_b] gives both parts in
// one product.  int8 values are exact in FP16, products are at most 2^14 in
// magnitude, and an FP32 sum of 1024 of them (512 samples) stays an exact
// integer (|sum| <= 2^24): the tensor cores accumulate one 512-sample block
// in TMEM, the epilogue rounds it to int32 (exact) and adds it to integer
// sums held in registers, and after the last block writes (or adds) the
// tile's visibilities once.  |V| <= 2^15 T, so int32 holds any T <= 65535.
//
// Two kernels per batch of channels and samples (sized to the context's
// workspace):
//   pack:  int8 -> fp16 operand images, K-major in the tensor cores' tile
//          order: one 16 KB image (128 rows x 64 K = 32 samples) per
//          (channel, k block, column block J) holding [X ; X'] of the 64 / P
//          elements of column block J, both pols, rows (x', pol, element),
//          transposed through shared memory;
//   gemm:  persistent, one work item per (row block I, pair of column blocks
//          2JP, 2JP+1, channel) with a >= b somewhere in it.  The A operand
//          of row block I (128 / P elements, rows (half, pol, element)) is the
//          X halves of images 2I and 2I+1, so it needs no images of its own;
//          B is images 2JP and 2JP+1, adjacent in the workspace.  Per k block
//          three bulk copies (8 + 8 + 32 KB) fill one stage of a 4-stage ring
//          and one thread issues four MMAs of M = 128, N = 256, K = 16 (one
//          commit per k block: a commit-and-wait round trip costs about as
//          much as four MMAs of N = 256, so narrower MMAs would leave the
//          tensor pipe idle) into one of two 256-column TMEM accumulators,
//          alternating per 512-sample block so that the epilogue of a block
//          overlaps the MMAs of the next.  Eight epilogue warps (two per TMEM
//          lane quadrant, one per column block of the pair) drain them.
#include <string.h>

#include <algorithm>

#include "hai_internal.h"
#include "tc.cuh"

namespace {

constexpr int kChunkT = 512;            // samples per exact FP32 block
constexpr int kKbT = 32;                // samples per k block (K = 64)
constexpr int kKbPerChunk = kChunkT / kKbT;
constexpr int kStages = 4;
constexpr uint32_t kLBO = 128;          // K-major: K-group stride
constexpr uint32_t kSBO = 1024;         // K-major: MN-group stride
constexpr uint32_t kImg = 16384;        // 128 rows x 64 K fp16
constexpr uint32_t kHalf = kImg / 2;    // rows 0..63 of an image
constexpr uint32_t kStage = 3 * kImg;   // A (16 KB) + B (32 KB)
constexpr uint32_t kIdesc = tc::idesc_f16(128, 256, 0, 0);
constexpr int kThreads = 320;           // warp 0 loads, warp 1 MMA, warps 2-9 epilogue
constexpr int kEpiThreads = 256;
constexpr uint32_t kTmemCols = 512;     // two 256-column FP32 accumulators

struct CorrGeo {
    int T, ne, P;
    int em, E;                   // elements per row block; per column block (= per 64-row half)
    int nbi, nbj;                // row / column blocks per channel
    int nimg;                    // images per (channel, k block): max(nbj rounded up to even, 2 nbi)
    int tiles_per_chan;
};

// (I, JP) of the k-th tile of a channel (row block I, column blocks 2JP and
// 2JP+1) with some a >= b, row-block major.
__device__ __forceinline__ void decode_tile(const CorrGeo &g, int k, int &I, int &JP) {
    const int njp_all = g.nimg / 2;
    for (I = 0; I < g.nbi; I++) {
        const int amax = min(g.ne - 1, (I + 1) * g.em - 1);
        const int njp = min(njp_all, amax / (2 * g.E) + 1);
        if (k < njp) {
            JP = k;
            return;
        }
        k -= njp;
    }
    I = JP = 0;
}

// image J of (channel cb, k block kb) of a batch holding nkb k blocks per channel
__host__ __device__ __forceinline__ size_t img_index(const CorrGeo &g, int nkb, int cb, int kb, int J) {
    return ((size_t)cb * nkb + kb) * g.nimg + J;
}

// One CTA per (channel, k block, group of kPackJ column blocks): the 32
// samples x P pols x kPackJ * 64 / P elements of the group are read once,
// coalesced, into shared memory ([sample][pol][element], 32 KB), and written
// out as kPackJ images, one thread per 16-byte K group (4 samples) of one
// image row, lanes over rows so that stores fill whole 128-byte row groups.
constexpr int kPackJ = 8;
constexpr int kPackCols = kPackJ * 64;       // P x elements of a group

__global__ void __launch_bounds__(256) corr_pack_kernel(const int8_t *__restrict__ volt, CorrGeo g, int c0, int kb0,
                                                        int nkb, int vec16, uint8_t *__restrict__ ws) {
    __shared__ __align__(16) char2 tile[kKbT][kPackCols];
    const int njg = (g.nimg + kPackJ - 1) / kPackJ;
    const int kb = blockIdx.x / njg, jg = blockIdx.x % njg, cb = blockIdx.y;
    const int ge = kPackJ * g.E;                 // elements of the group
    const int a0 = jg * ge;
    const int8_t *vc = volt + (size_t)(c0 + cb) * g.T * g.P * g.ne * 2;
    const int tb = (kb0 + kb) * kKbT;
    // load: rows (t, pol) of ge elements; 16-byte vectors where the rows allow
    if (vec16 && a0 + ge <= g.ne) {
        const int nv = ge / 8;                   // 8 elements per 16 bytes
        for (int i = threadIdx.x; i < kKbT * g.P * nv; i += blockDim.x) {
            const int v = i % nv, tp = i / nv, t = tp / g.P, pol = tp % g.P;
            uint4 x = make_uint4(0, 0, 0, 0);
            if (tb + t < g.T)
                x = *reinterpret_cast<const uint4 *>(vc + (((size_t)(tb + t) * g.P + pol) * g.ne + a0 + 8 * v) * 2);
            *reinterpret_cast<uint4 *>(&tile[t][pol * ge + 8 * v]) = x;
        }
    } else {
        for (int i = threadIdx.x; i < kKbT * g.P * ge; i += blockDim.x) {
            const int e = i % ge, tp = i / ge, t = tp / g.P, pol = tp % g.P;
            char2 x = make_char2(0, 0);
            if (tb + t < g.T && a0 + e < g.ne)
                x = reinterpret_cast<const char2 *>(vc)[((size_t)(tb + t) * g.P + pol) * g.ne + a0 + e];
            tile[t][pol * ge + e] = x;
        }
    }
    __syncthreads();
    const int nj = min(kPackJ, g.nimg - jg * kPackJ);
    for (int i = threadIdx.x; i < nj * 1024; i += blockDim.x) {
        const int r = i & 127, kg = (i >> 7) & 7, jl = i >> 10;
        const int rr = r & 63, pol = rr / g.E;
        const int col = pol * ge + jl * g.E + rr % g.E;
        uint32_t h2[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const char2 v = tile[4 * kg + j][col];
            h2[j] = r >= 64 ? tc::pack_half2(-(float)v.y, (float)v.x) : tc::pack_half2((float)v.x, (float)v.y);
        }
        uint8_t *dst = ws + img_index(g, nkb, cb, kb, jg * kPackJ + jl) * kImg + tc::off_kmajor(r, 8 * kg, kLBO, kSBO);
        *reinterpret_cast<uint4 *>(dst) = make_uint4(h2[0], h2[1], h2[2], h2[3]);
    }
}

struct GemmParams {
    const uint8_t *ws;
    CorrGeo g;
    int c0, ncb;                 // channels of this batch
    int nkb;                     // k blocks of this batch (per channel)
    int add;                     // add to vis (else overwrite)
    int32_t *vis;
    unsigned *status;
};

template <int P>
__global__ void __launch_bounds__(kThreads, 1) corr_gemm_kernel(const GemmParams p) {
    constexpr int E = 64 / P;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], accf[2], acce[2];
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const CorrGeo g = p.g;
    const int nitems = g.tiles_per_chan * p.ncb;
    const int nchunk = (p.nkb + kKbPerChunk - 1) / kKbPerChunk;
    if (tid == 0) {
        for (int s = 0; s < kStages; s++) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&accf[b], 1);
            tc::mbar_init(&acce[b], kEpiThreads);
        }
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc(&tslot, kTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tslot;
    // The loader and MMA loops run on one thread each and sit on the critical
    // path: stage and parity are toggled, not divided, pointers and
    // descriptors advance by additions.
    if (warp == 0) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 1;                       // first pass over the ring waits on nothing
            bool wrapped = false;
            const size_t kb_stride = (size_t)g.nimg * kImg;
            for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
                int I, JP;
                decode_tile(g, w % g.tiles_per_chan, I, JP);
                const uint8_t *base = p.ws + img_index(g, p.nkb, w / g.tiles_per_chan, 0, 0) * kImg;
                const uint8_t *pa0 = base + (size_t)(2 * I) * kImg, *pa1 = pa0 + kImg;
                const uint8_t *pb = base + (size_t)(2 * JP) * kImg;
                for (int kb = 0; kb < p.nkb; kb++) {
                    if (wrapped) tc::mbar_wait(&empty[s], ph, p.status);
                    uint8_t *st = smem + (size_t)s * kStage;
                    tc::mbar_arrive_expect_tx(&full[s], kStage);
                    tc::bulk_g2s(st, pa0, kHalf, &full[s]);
                    tc::bulk_g2s(st + kHalf, pa1, kHalf, &full[s]);
                    tc::bulk_g2s(st + kImg, pb, 2 * kImg, &full[s]);
                    pa0 += kb_stride;
                    pa1 += kb_stride;
                    pb += kb_stride;
                    if (++s == kStages) {
                        s = 0;
                        ph ^= 1u;
                        wrapped = true;
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;                       // full[] parity
            uint32_t acc_ph = 3u, acc_used = 0u;   // per buffer (bit b): acce[] parity, buffer used before
            int b = 0;
            // descriptors of stage 0; a stage is kStage bytes = kStage >> 4 in the address field
            const uint64_t da0 = tc::desc(tc::smem_u32(smem), kLBO, kSBO);
            const uint64_t db0 = tc::desc(tc::smem_u32(smem) + kImg, kLBO, kSBO);
            constexpr uint64_t kStageD = kStage >> 4, kStepD = (2 * kLBO) >> 4;
            for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
                for (int ch = 0; ch < nchunk; ch++) {
                    if ((acc_used >> b) & 1u) tc::mbar_wait(&acce[b], (acc_ph >> b) & 1u, p.status);
                    acc_ph ^= 1u << b;
                    acc_used |= 1u << b;
                    tc::fence_after();
                    const uint32_t d = tmem + (uint32_t)(b * 256);
                    const int nk = min(kKbPerChunk, p.nkb - ch * kKbPerChunk);
                    for (int kb = 0; kb < nk; kb++) {
                        tc::mbar_wait(&full[s], ph, p.status);
                        tc::fence_after();
                        const uint64_t da = da0 + (uint64_t)s * kStageD, db = db0 + (uint64_t)s * kStageD;
                        tc::mma_f16(d, da, db, kIdesc, kb > 0 ? 1u : 0u);
                        tc::mma_f16(d, da + kStepD, db + kStepD, kIdesc, 1u);
                        tc::mma_f16(d, da + 2 * kStepD, db + 2 * kStepD, kIdesc, 1u);
                        tc::mma_f16(d, da + 3 * kStepD, db + 3 * kStepD, kIdesc, 1u);
                        tc::mma_commit(&empty[s]);
                        if (++s == kStages) {
                            s = 0;
                            ph ^= 1u;
                        }
                    }
                    tc::mma_commit(&accf[b]);
                    b ^= 1;
                }
            }
        }
    } else {
        // epilogue, warps 2-9: TMEM lane quadrant q = warp % 4 (row m), column
        // block hs of the pair; 64 (b, q) outputs, their int32 sums in registers
        const int q = warp & 3, hs = (warp - 2) >> 2, m = q * 32 + lane;
        const int h = m >> 6, rr = m & 63;
        const int pol = rr / E;
        const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(hs * 128);
        const long long nbl = (long long)g.ne * (g.ne + 1) / 2;
        long long grp = 0;
        for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
            int I, JP;
            decode_tile(g, w % g.tiles_per_chan, I, JP);
            const int J = 2 * JP + hs;
            const int c = p.c0 + w / g.tiles_per_chan;
            const int a = I * (2 * E) + h * E + rr % E;
            int sre[64], sim[64];
#pragma unroll
            for (int k = 0; k < 64; k++) sre[k] = sim[k] = 0;
            for (int ch = 0; ch < nchunk; ch++, grp++) {
                const int b = (int)(grp & 1);
                tc::mbar_wait(&accf[b], (uint32_t)((grp >> 1) & 1), p.status);
                tc::fence_after();
                const uint32_t tacc = lane_base + (uint32_t)(b * 256);
#pragma unroll
                for (int n0 = 0; n0 < 64; n0 += 16) {
                    uint32_t vr[16], vi[16];
                    tc::tmem_ld16(tacc + (uint32_t)n0, vr);
                    tc::tmem_ld16(tacc + 64u + (uint32_t)n0, vi);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int k = 0; k < 16; k++) {
                        sre[n0 + k] += __float2int_rn(__uint_as_float(vr[k]));
                        sim[n0 + k] += __float2int_rn(__uint_as_float(vi[k]));
                    }
                }
                tc::fence_before();
                tc::mbar_arrive(&acce[b]);
            }
            if (a < g.ne) {
                int2 *row = reinterpret_cast<int2 *>(p.vis) + (((size_t)c * nbl + (long long)a * (a + 1) / 2) * P + pol) * P;
#pragma unroll
                for (int n0 = 0; n0 < 64; n0 += 16) {
#pragma unroll
                    for (int k = 0; k < 16; k++) {
                        const int n = n0 + k, qq = n / E, bb = J * E + n % E;
                        if (bb > a || bb >= g.ne) continue;
                        int2 *o = row + (size_t)bb * (P * P) + qq;
                        int2 v = make_int2(sre[n], sim[n]);
                        if (p.add) {
                            const int2 old = *o;
                            v.x += old.x;
                            v.y += old.y;
                        }
                        *o = v;
                    }
                    asm volatile("" ::: "memory");   // keep the read-modify-writes in groups of 16
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

extern "C" hai_status hai_correlate(hai_ctx *ctx, const int8_t *volt, int C, int T, int N, int P,
                                    int32_t *vis, int accumulate, void *stream) {
    if (!ctx) return hai_fail(HAI_ERR_INVALID_ARG, "hai_correlate: ctx is NULL");
    if (C < 0 || T < 0 || N <= 0 || (P != 1 && P != 2) || (accumulate != 0 && accumulate != 1))
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_correlate: bad size, polarisation count or flag");
    if (T > 65535) return hai_fail(HAI_ERR_OVERFLOW_RISK, "hai_correlate: T > 65535 may overflow int32");
    if (N > 65535) return hai_fail(HAI_ERR_UNSUPPORTED, "hai_correlate: N > 65535");
    CorrGeo g;
    g.T = T;
    g.ne = N;
    g.P = P;
    g.em = 128 / P;
    g.E = 64 / P;
    g.nbi = (N + g.em - 1) / g.em;
    g.nbj = (N + g.E - 1) / g.E;
    g.nimg = std::max((g.nbj + 1) & ~1, 2 * g.nbi);
    const size_t chunk_bytes = (size_t)kKbPerChunk * g.nimg * kImg;   // one channel, one 512-sample block
    if (chunk_bytes > kCorrWorkspaceBytes)
        return hai_fail(HAI_ERR_UNSUPPORTED, "hai_correlate: N too large for the operand workspace");
    if (C == 0) return HAI_OK;
    if (!vis || (T > 0 && !volt)) return hai_fail(HAI_ERR_INVALID_ARG, "hai_correlate: NULL buffer");
    if (hai_fault_injected("launch")) return hai_fail(HAI_ERR_CUDA, "hai_correlate: injected launch failure");
    HAI_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nbl = (size_t)N * (N + 1) / 2;
    if (T == 0) {
        if (!accumulate) HAI_CUDA_TRY(cudaMemsetAsync(vis, 0, sizeof(int32_t) * 2 * P * P * nbl * C, st));
        return HAI_OK;
    }
    if (((uintptr_t)vis) & 7) return hai_fail(HAI_ERR_INVALID_ARG, "hai_correlate: vis must be 8-byte aligned");
    if (((uintptr_t)volt) & 1) return hai_fail(HAI_ERR_INVALID_ARG, "hai_correlate: volt must be 2-byte aligned");
    const hai_status wst = hai_workspace(ctx);
    if (wst != HAI_OK) return wst;
    int tpc = 0;
    for (int I = 0; I < g.nbi; I++) {
        const int amax = std::min(N - 1, (I + 1) * g.em - 1);
        tpc += std::min(g.nimg / 2, amax / (2 * g.E) + 1);
    }
    g.tiles_per_chan = tpc;
    // batches: as many 512-sample blocks per channel as fit, then as many channels
    const int nchunk_all = (T + kChunkT - 1) / kChunkT;
    const int chunks_per_batch = (int)std::min<size_t>(nchunk_all, ctx->corr_ws_bytes / chunk_bytes);
    const size_t chan_bytes = chunk_bytes * chunks_per_batch;
    const int chans_per_batch = (int)std::min<size_t>(
        {(size_t)C, (size_t)65535, ctx->corr_ws_bytes / chan_bytes, (size_t)(INT32_MAX / tpc)});
    const size_t smem = (size_t)kStages * kStage;
    auto gemm = P == 2 ? corr_gemm_kernel<2> : corr_gemm_kernel<1>;
    HAI_CUDA_TRY(cudaFuncSetAttribute(gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    uint8_t *ws = static_cast<uint8_t *>(ctx->d_corr_ws);
    // rows of the voltage array start on 16-byte boundaries when 2 N is a multiple of 16
    const int vec16 = (N % 8 == 0 && ((uintptr_t)volt & 15) == 0) ? 1 : 0;
    const int pidx = prof_begin(ctx, st);
    for (int ch0 = 0; ch0 < nchunk_all; ch0 += chunks_per_batch) {
        const int kb0 = ch0 * kKbPerChunk;
        const int t1 = std::min(T, (ch0 + chunks_per_batch) * kChunkT);
        const int nkb = (t1 - kb0 * kKbT + kKbT - 1) / kKbT;
        for (int c0 = 0; c0 < C; c0 += chans_per_batch) {
            const int ncb = std::min(chans_per_batch, C - c0);
            const int njg = (g.nimg + kPackJ - 1) / kPackJ;
            corr_pack_kernel<<<dim3(nkb * njg, ncb), 256, 0, st>>>(volt, g, c0, kb0, nkb, vec16, ws);
            GemmParams gp;
            gp.ws = ws;
            gp.g = g;
            gp.c0 = c0;
            gp.ncb = ncb;
            gp.nkb = nkb;
            gp.add = (ch0 > 0 || accumulate) ? 1 : 0;
            gp.vis = vis;
            gp.status = ctx->d_status;
            gemm<<<std::min(tpc * ncb, ctx->num_sms), kThreads, smem, st>>>(gp);
            prof_count(ctx, 2);
        }
    }
    prof_end(ctx, pidx, st);
    HAI_CUDA_TRY(cudaGetLastError());
    return HAI_OK;
}
