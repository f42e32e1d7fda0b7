// Correlator (Eq. intra-station visibilities): V^{pq}_{ab} = sum_t E^p_a conj(E^q_b)
// for all element pairs a >= b, on tcgen05 tensor cores with exact integer
// results.
//
// Per channel the voltages form a real matrix X[m][k] with rows m = (pol,
// element) and columns k = (sample, re/im).  For a tile of rows (elements
// a) and columns (elements b):
//   Re V = sum_k X_a[k] X_b[k],   Im V = sum_k X_a[k] X'_b[k],
// where X'_b = (-Im, Re) per sample, so one MMA with B = [X_b ; X'_b]
// (N = 128) yields both parts.  int8 values are exact in FP16, products are
// below 2^14, and the FP32 accumulator holds every partial sum exactly while
// it stays below 2^24, i.e. for up to 512 samples; every 512 samples the
// epilogue moves the accumulator into int32 registers (exact) and the MMA
// restarts.  |V| <= 2^15 T, so int32 holds any T <= 65535.
//
// CTA = 16 warps, persistent over (channel, row block I, column block J)
// tiles that touch the lower triangle a >= b:
//   warps 0-6  producers: 16-byte int8 loads (prefetched one stage ahead),
//              int8 -> fp16 by a bit trick, MN-major operand stages in smem;
//   warp 7     one thread issues the MMAs (4 per 32-sample stage);
//   warps 8-15 epilogue: TMEM -> int32 accumulators, then the lower-triangle
//              visibilities are written.
// Tile: rows M = 128 = P x (128/P) elements, columns 2 x P x (64/P) elements.
#include <string.h>

#include <algorithm>

#include "hai_internal.h"
#include "tc.cuh"

namespace {

constexpr int kThreads = 512;
constexpr int kProd = 224;              // warps 0-6
constexpr int kMmaWarp = 7;
constexpr int kEpi = 256;               // warps 8-15
constexpr int kStageT = 32;             // samples per stage (K = 64)
constexpr int kChunkT = 512;            // samples per exact FP32 block
constexpr int kStages = 4;
constexpr uint32_t kKs = 2064;          // MN-major: K-group stride (16 MN groups + 16 B)
constexpr uint32_t kMNs = 128;          // MN-major: MN-group stride
constexpr uint32_t kOpBytes = 8 * kKs;  // one operand stage (128 rows x 64 K)
constexpr uint32_t kIdesc = tc::idesc_f16(128, 128, 1, 1);

struct CorrParams {
    const int8_t *volt;
    int C, T, ne, P;
    int em, en;                  // elements per row block / column block
    int nbi, nbj;                // row / column blocks per channel
    int tiles_per_chan;
    long long ntiles;
    int32_t *vis;
    int accumulate;
    int vec;                     // 16-byte loads are aligned
    unsigned *status;
};

// (I, J) of the k-th lower-triangle tile of a channel, row-block major.
__device__ __forceinline__ void decode_tile(const CorrParams &p, int k, int &I, int &J) {
    for (I = 0; I < p.nbi; I++) {
        const int amax = min(p.ne - 1, (I + 1) * p.em - 1);
        const int nj = min(p.nbj, amax / p.en + 1);
        if (k < nj) {
            J = k;
            return;
        }
        k -= nj;
    }
    I = J = 0;
}

// int8 (re, im) x 8 in 16 bytes -> fp16 re[8] and im[8] packed in uint4s.
// half(1024 + u) has bits 0x6400 + u for 0 <= u < 1024, and u = x + 128 is
// the int8 with its sign bit flipped; subtracting 1152 leaves x exactly.
__device__ __forceinline__ void int8x16_to_half(const int4 raw, uint4 &re, uint4 &im) {
    const uint32_t w[4] = {(uint32_t)raw.x ^ 0x80808080u, (uint32_t)raw.y ^ 0x80808080u,
                           (uint32_t)raw.z ^ 0x80808080u, (uint32_t)raw.w ^ 0x80808080u};
    const __half2 bias = __floats2half2_rn(1152.f, 1152.f);
    uint32_t r[4], m[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        // word k holds (re, im) of elements 2k and 2k+1: bytes re0 im0 re1 im1
        const uint32_t pr = __byte_perm(w[k], 0x64646464u, 0x4240);   // re0, 0x64, re1, 0x64
        const uint32_t pi = __byte_perm(w[k], 0x64646464u, 0x4341);   // im0, 0x64, im1, 0x64
        __half2 hr = __hsub2(*reinterpret_cast<const __half2 *>(&pr), bias);
        __half2 hi = __hsub2(*reinterpret_cast<const __half2 *>(&pi), bias);
        r[k] = *reinterpret_cast<uint32_t *>(&hr);
        m[k] = *reinterpret_cast<uint32_t *>(&hi);
    }
    re = make_uint4(r[0], r[1], r[2], r[3]);
    im = make_uint4(m[0], m[1], m[2], m[3]);
}

__global__ void __launch_bounds__(kThreads, 1) corr_kernel(const CorrParams p) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mb_full[kStages], mb_empty[kStages];
    __shared__ __align__(8) uint64_t mb_dfull[2], mb_dempty[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t *sA = smem;                               // [kStages][kOpBytes]
    uint8_t *sB = smem + kStages * kOpBytes;

    if (tid == 0) {
        for (int s = 0; s < kStages; s++) {
            tc::mbar_init(&mb_full[s], kProd);
            tc::mbar_init(&mb_empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&mb_dfull[b], 1);
            tc::mbar_init(&mb_dempty[b], kEpi);
        }
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot, 256);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_slot;

    const int nstage = (p.T + kStageT - 1) / kStageT;          // stages per tile
    const int per_chunk = kChunkT / kStageT;                   // stages per exact block
    const int nchunk = (nstage + per_chunk - 1) / per_chunk;   // blocks per tile
    const int sample_bytes = p.P * p.ne * 2;

    if (warp < kMmaWarp) {
        // ============================================================ producers
        // work items of a stage: A (rows): P x 32 samples x em/8 groups,
        // B (columns): P x 32 samples x en/8 groups
        const int ga = p.em / 8, gb = p.en / 8;
        const int na = p.P * kStageT * ga, nb = p.P * kStageT * gb;
        const int nitem = na + nb;
        constexpr int kMaxItems = 4;                           // per thread per stage
        long long gs = 0;                                      // global stage counter
        for (long long tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x) {
            const int c = (int)(tile / p.tiles_per_chan);
            int I, J;
            decode_tile(p, (int)(tile % p.tiles_per_chan), I, J);
            const int8_t *vc = p.volt + (size_t)c * p.T * sample_bytes;
            // item -> (pol, sample, 8-element group); each warp's 32 items are
            // 8 consecutive samples x 4 consecutive groups, so global loads
            // fill 32-byte sectors and the 16-byte smem stores of a phase land
            // in distinct bank groups
            auto item_src = [&](int it, int st, int &pol, int &t, int &a0, bool &is_b) {
                is_b = it >= na;
                const int r = is_b ? it - na : it;
                const int gq = (is_b ? gb : ga) / 4;
                const int li = r & 31, blk = r >> 5;
                const int gqi = blk % gq, tb = (blk / gq) % (kStageT / 8);
                pol = blk / (gq * (kStageT / 8));
                t = st * kStageT + tb * 8 + (li & 7);
                a0 = (is_b ? J * p.en : I * p.em) + (gqi * 4 + (li >> 3)) * 8;
            };
            auto load = [&](int it, int st) -> int4 {
                int pol, t, a0;
                bool is_b;
                item_src(it, st, pol, t, a0, is_b);
                if (t >= p.T) return make_int4(0, 0, 0, 0);
                const int8_t *src = vc + (size_t)t * sample_bytes + (size_t)pol * p.ne * 2 + (size_t)a0 * 2;
                if (p.vec && a0 + 8 <= p.ne) return __ldg(reinterpret_cast<const int4 *>(src));
                uint32_t wv[4];                               // ragged edge: byte loads
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    wv[k] = 0;
#pragma unroll
                    for (int j = 0; j < 4; j++)
                        if (a0 + (4 * k + j) / 2 < p.ne) wv[k] |= (uint32_t)(uint8_t)src[4 * k + j] << (8 * j);
                }
                return make_int4((int)wv[0], (int)wv[1], (int)wv[2], (int)wv[3]);
            };
            int4 cur[kMaxItems], nxt[kMaxItems];
#pragma unroll
            for (int k = 0; k < kMaxItems; k++) {
                const int it = tid + k * kProd;
                cur[k] = it < nitem ? load(it, 0) : make_int4(0, 0, 0, 0);
            }
            for (int st = 0; st < nstage; st++, gs++) {
#pragma unroll
                for (int k = 0; k < kMaxItems; k++) {          // prefetch the next stage
                    const int it = tid + k * kProd;
                    nxt[k] = (it < nitem && st + 1 < nstage) ? load(it, st + 1) : make_int4(0, 0, 0, 0);
                }
                const int slot = (int)(gs % kStages);
                if (gs >= kStages) tc::mbar_wait(&mb_empty[slot], (uint32_t)(((gs / kStages) - 1) & 1), p.status);
                uint8_t *A = sA + slot * kOpBytes, *B = sB + slot * kOpBytes;
#pragma unroll
                for (int k = 0; k < kMaxItems; k++) {
                    const int it = tid + k * kProd;
                    if (it >= nitem) continue;
                    int pol, t, a0;
                    bool is_b;
                    item_src(it, st, pol, t, a0, is_b);
                    uint4 re, im;
                    int8x16_to_half(cur[k], re, im);
                    const int tl = t - st * kStageT;
                    const int kre = 2 * tl, kim = 2 * tl + 1;
                    if (!is_b) {
                        const int m = pol * p.em + (a0 - I * p.em);
                        *reinterpret_cast<uint4 *>(A + tc::off_mnmajor(m, kre, kKs, kMNs)) = re;
                        *reinterpret_cast<uint4 *>(A + tc::off_mnmajor(m, kim, kKs, kMNs)) = im;
                    } else {
                        const int n = pol * p.en + (a0 - J * p.en);
                        const uint4 nim = make_uint4(im.x ^ 0x80008000u, im.y ^ 0x80008000u,
                                                     im.z ^ 0x80008000u, im.w ^ 0x80008000u);
                        *reinterpret_cast<uint4 *>(B + tc::off_mnmajor(n, kre, kKs, kMNs)) = re;
                        *reinterpret_cast<uint4 *>(B + tc::off_mnmajor(n, kim, kKs, kMNs)) = im;
                        *reinterpret_cast<uint4 *>(B + tc::off_mnmajor(n + 64, kre, kKs, kMNs)) = nim;
                        *reinterpret_cast<uint4 *>(B + tc::off_mnmajor(n + 64, kim, kKs, kMNs)) = re;
                    }
                }
                tc::fence_proxy_async();
                tc::mbar_arrive(&mb_full[slot]);
#pragma unroll
                for (int k = 0; k < kMaxItems; k++) cur[k] = nxt[k];
            }
        }
    } else if (warp == kMmaWarp) {
        // ============================================================ MMA
        if (lane == 0) {
            long long gs = 0, gc = 0;                          // stage and block counters
            for (long long tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x) {
                for (int ch = 0; ch < nchunk; ch++, gc++) {
                    const int b = (int)(gc & 1);
                    if (gc >= 2) tc::mbar_wait(&mb_dempty[b], (uint32_t)(((gc >> 1) - 1) & 1), p.status);
                    tc::fence_after();
                    const uint32_t d = tmem + (uint32_t)b * 128u;
                    const int s_end = min(nstage, (ch + 1) * per_chunk);
                    for (int st = ch * per_chunk; st < s_end; st++, gs++) {
                        const int slot = (int)(gs % kStages);
                        tc::mbar_wait(&mb_full[slot], (uint32_t)((gs / kStages) & 1), p.status);
                        tc::fence_after();
                        const uint32_t a = tc::smem_u32(sA + slot * kOpBytes), bb = tc::smem_u32(sB + slot * kOpBytes);
#pragma unroll
                        for (int s = 0; s < 4; s++)
                            tc::mma_f16(d, tc::desc(a + s * 2 * kKs, kKs, kMNs), tc::desc(bb + s * 2 * kKs, kKs, kMNs),
                                        kIdesc, (st > ch * per_chunk || s > 0) ? 1u : 0u);
                        tc::mma_commit(&mb_empty[slot]);
                    }
                    tc::mma_commit(&mb_dfull[b]);
                }
            }
        }
    } else {
        // ============================================================ epilogue
        const int q = warp & 3, h = (warp - 8) >> 2;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        const int m = q * 32 + lane;                           // tile row of this thread
        const int pol = m / p.em;
        long long gc = 0;
        const long long nbl = (long long)p.ne * (p.ne + 1) / 2;
        for (long long tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x) {
            const int c = (int)(tile / p.tiles_per_chan);
            int I, J;
            decode_tile(p, (int)(tile % p.tiles_per_chan), I, J);
            int acc_r[32], acc_i[32];
#pragma unroll
            for (int k = 0; k < 32; k++) acc_r[k] = acc_i[k] = 0;
            for (int ch = 0; ch < nchunk; ch++, gc++) {
                const int b = (int)(gc & 1);
                tc::mbar_wait(&mb_dfull[b], (uint32_t)((gc >> 1) & 1), p.status);
                tc::fence_after();
#pragma unroll
                for (int half = 0; half < 2; half++) {
                    uint32_t rr[16], ri[16];
                    const uint32_t col = (uint32_t)b * 128u + (uint32_t)(32 * h + 16 * half);
                    tc::tmem_ld16(tmem + lane_base + col, rr);
                    tc::tmem_ld16(tmem + lane_base + col + 64, ri);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int k = 0; k < 16; k++) {
                        acc_r[16 * half + k] += __float2int_rn(__uint_as_float(rr[k]));
                        acc_i[16 * half + k] += __float2int_rn(__uint_as_float(ri[k]));
                    }
                }
                tc::fence_before();
                tc::mbar_arrive(&mb_dempty[b]);
            }
            // lower-triangle outputs of this thread's row (element a, pol)
            const int a = I * p.em + (m - pol * p.em);
            if (a < p.ne) {
#pragma unroll
                for (int k = 0; k < 32; k++) {
                    const int n = 32 * h + k;                  // column 0..63
                    const int qq = n / p.en;
                    const int bidx = J * p.en + (n - qq * p.en);
                    if (bidx > a || bidx >= p.ne) continue;
                    const long long bl = (long long)a * (a + 1) / 2 + bidx;
                    int2 *o = reinterpret_cast<int2 *>(p.vis) + (((size_t)c * nbl + bl) * p.P + pol) * p.P + qq;
                    int2 v = make_int2(acc_r[k], acc_i[k]);
                    if (p.accumulate) {
                        const int2 old = *o;
                        v.x += old.x;
                        v.y += old.y;
                    }
                    *o = v;
                }
            }
        }
    }

    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

}  // namespace

extern "C" hai_status hai_correlate(hai_ctx *ctx, const int8_t *volt, int C, int T, int N, int P,
                                    int32_t *vis, int accumulate, void *stream) {
    if (!ctx) return hai_fail(HAI_ERR_INVALID_ARG, "hai_correlate: ctx is NULL");
    if (C < 0 || T < 0 || N <= 0 || (P != 1 && P != 2) || (accumulate != 0 && accumulate != 1))
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_correlate: bad size, polarisation count or flag");
    if (T > 65535) return hai_fail(HAI_ERR_OVERFLOW_RISK, "hai_correlate: T > 65535 may overflow int32");
    if (N > 65535) return hai_fail(HAI_ERR_UNSUPPORTED, "hai_correlate: N > 65535");
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
    CorrParams p;
    p.volt = volt;
    p.C = C;
    p.T = T;
    p.ne = N;
    p.P = P;
    p.em = 128 / P;
    p.en = 64 / P;
    p.nbi = (N + p.em - 1) / p.em;
    p.nbj = (N + p.en - 1) / p.en;
    int tpc = 0;
    for (int I = 0; I < p.nbi; I++) {
        const int amax = std::min(N - 1, (I + 1) * p.em - 1);
        tpc += std::min(p.nbj, amax / p.en + 1);
    }
    p.tiles_per_chan = tpc;
    p.ntiles = (long long)tpc * C;
    p.vis = vis;
    p.accumulate = accumulate;
    p.vec = ((N % 8) == 0) && ((((uintptr_t)volt) & 15) == 0);
    p.status = ctx->d_status;
    const size_t smem = 2 * (size_t)kStages * kOpBytes;
    if (smem > (size_t)ctx->smem_optin) return hai_fail(HAI_ERR_UNSUPPORTED, "hai_correlate: shared memory");
    HAI_CUDA_TRY(cudaFuncSetAttribute(corr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (int)std::min<long long>(p.ntiles, ctx->num_sms);
    const int pidx = prof_begin(ctx, st);
    corr_kernel<<<grid, kThreads, smem, st>>>(p);
    prof_end(ctx, pidx, st);
    prof_count(ctx, 1);
    HAI_CUDA_TRY(cudaGetLastError());
    return HAI_OK;
}
