// Voltage beamformer (Eq. intra-station BF) with diagonal polarisation
// weights, B^p_k(t) = sum_a conj(w^p_{k,a}) E^p_a(t), exact in int32, with an
// optional requantisation to int8 fused into the epilogue.
//
// Per (station s, channel c, tile of 128 samples) and polarisation p the beams
// are one real GEMM on tcgen05 tensor cores:
//   D_p[t][n] = sum_kappa A_p[t][kappa] B_p[n][kappa],  kappa = (element, re/im)
// with A_p the voltages (int8 widened to fp16, exact) and B_p the weights:
// row n = 2k holds (w_r, w_i) per element (real part of conj(w) E), row 2k+1
// holds (-w_i, w_r) (imaginary part).  Products are below 2^14 and an output
// sums 2 N_e of them, so for N_e <= 512 every FP32 partial sum is an integer
// below 2^24: exact.
//
// CTA = 13 warps, persistent over a contiguous range of (s, c, tile) units:
//   warps 0-7  producers: cp.async 16-byte copies of the voltage rows of a
//              64-element chunk (zero-filled past T) into a 5-deep int8 ring
//              (4 chunks, 64 KB, in flight per SM to cover HBM latency), then
//              fp16 widening into a 2-deep K-major A ring; every thread owns
//              four fixed (row, 16-byte group) items of a chunk for the copies
//              and four for the widening, their offsets computed once; the
//              station's weights are widened into B when the station changes;
//   warp 8     one thread issues the MMAs (8 per chunk);
//   warps 9-12 epilogue: TMEM -> int32, optional requantisation; each thread
//              assembles its sample's [k][p][re, im] row from both pols and
//              writes it with 16-byte stores (rows are contiguous per unit).
#include "hai_internal.h"
#include "tc.cuh"

namespace {

constexpr int kThreads = 416;
constexpr int kProd = 256;             // warps 0-7
constexpr int kMmaWarp = 8;
constexpr int kEpi = 128;              // warps 9-12
constexpr int kItems = 4;              // (row, 16-byte group) items per producer thread and chunk
constexpr int kTile = 128;             // samples per unit (MMA M)
constexpr int kChunkE = 64;            // elements per K chunk (128 real K)
constexpr int kI8Stages = 5;           // int8 landing ring: 4 chunks in flight
constexpr int kAhead = kI8Stages - 1;
constexpr int kAStages = 2;            // fp16 operand ring
constexpr uint32_t kI8Bytes = kTile * kChunkE * 2;   // int8 chunk: 128 rows x 128 B
constexpr uint32_t kAKs = 128;         // A: K-group stride
constexpr uint32_t kAMNs = 2048;       // A: row-group stride (16 K groups)
constexpr uint32_t kABytes = 16 * kAMNs;             // 32 KB fp16 chunk

struct BfParams {
    const int8_t *volt;
    const int8_t *w;
    int S, C, T, K, ne, P;
    int tiles;                 // sample tiles per (s, c)
    long long nunits, per_cta;
    int shift;                 // < 0: int32 output
    void *beams;
    unsigned long long *nsat;
    unsigned *status;
};

__device__ __forceinline__ void cp_async16(void *dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc::smem_u32(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void bar_prod() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// 16 int8 -> 16 fp16 (two 8-value K groups), exact: bits 0x6400 + (x ^ 0x80) minus 1152
__device__ __forceinline__ void widen16(const int4 raw, uint4 &lo, uint4 &hi) {
    const uint32_t w[4] = {(uint32_t)raw.x ^ 0x80808080u, (uint32_t)raw.y ^ 0x80808080u,
                           (uint32_t)raw.z ^ 0x80808080u, (uint32_t)raw.w ^ 0x80808080u};
    const __half2 bias = __floats2half2_rn(1152.f, 1152.f);
    uint32_t o[8];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const uint32_t p0 = __byte_perm(w[k], 0x64646464u, 0x4140);   // bytes 0, 1
        const uint32_t p1 = __byte_perm(w[k], 0x64646464u, 0x4342);   // bytes 2, 3
        __half2 h0 = __hsub2(*reinterpret_cast<const __half2 *>(&p0), bias);
        __half2 h1 = __hsub2(*reinterpret_cast<const __half2 *>(&p1), bias);
        o[2 * k] = *reinterpret_cast<uint32_t *>(&h0);
        o[2 * k + 1] = *reinterpret_cast<uint32_t *>(&h1);
    }
    lo = make_uint4(o[0], o[1], o[2], o[3]);
    hi = make_uint4(o[4], o[5], o[6], o[7]);
}

__device__ __forceinline__ int requant(int x, int shift, int &sat) {
    int m = x < 0 ? -x : x;
    if (shift > 0) m = (m + (1 << (shift - 1))) >> shift;
    if (m > 127) {
        m = 127;
        sat++;
    }
    return x < 0 ? -m : m;
}

__global__ void __launch_bounds__(kThreads, 1) bf_kernel(const BfParams p) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mb_full[kAStages], mb_empty[kAStages], mb_dfull[2], mb_dempty[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nchunk = (p.ne + kChunkE - 1) / kChunkE;        // per polarisation
    const int ne_pad = nchunk * kChunkE;                      // B covers whole chunks, zero-padded
    const uint32_t bmns = (uint32_t)ne_pad * 32u;             // B: row-group stride (2 ne_pad / 8 groups)
    const uint32_t bbytes = (uint32_t)(2 * p.K / 8) * bmns;   // B of one polarisation
    uint8_t *sI8 = smem;                                      // [kI8Stages][kI8Bytes]
    uint8_t *sA = smem + kI8Stages * kI8Bytes;                // [kAStages][kABytes]
    uint8_t *sB = sA + kAStages * kABytes;                    // [P][bbytes]
    const int ncols = 2 * p.K;                                // MMA N per polarisation
    const uint32_t dcols = (uint32_t)(p.P * ncols);           // TMEM columns per unit

    if (tid == 0) {
        for (int s = 0; s < kAStages; s++) {
            tc::mbar_init(&mb_full[s], kProd);
            tc::mbar_init(&mb_empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&mb_dfull[b], 1);
            tc::mbar_init(&mb_dempty[b], kEpi);
        }
        tc::mbar_fence_init();
    }
    uint32_t alloc = 32;
    while (alloc < 2 * dcols) alloc <<= 1;
    if (warp == 0) tc::tmem_alloc(&tmem_slot, alloc);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_slot;
    const long long u0 = (long long)blockIdx.x * p.per_cta;
    const long long u1 = min(p.nunits, u0 + p.per_cta);
    const size_t row_bytes = (size_t)p.ne * 2;                 // one (t, p) row of voltages
    const uint32_t idesc = tc::idesc_f16(128, ncols, 0, 0);

    if (warp < kMmaWarp) {
        // ============================================================ producers
        long long gq = 0;                                      // chunk counter (stages)
        int cur_s = -1;
        // chunks of the CTA in order: (unit = (station, channel, tile), pol,
        // element chunk), walked by counters (no 64-bit divisions per chunk);
        // one walker for the copies issued kAhead chunks early, one for the
        // chunk being widened
        struct Walk {
            int s, c, tile, pol, kc;
        };
        auto walk_init = [&](Walk &w) {
            w.s = (int)(u0 / ((long long)p.C * p.tiles));
            w.c = (int)((u0 / p.tiles) % p.C);
            w.tile = (int)(u0 % p.tiles);
            w.pol = 0;
            w.kc = 0;
        };
        auto walk_next = [&](Walk &w) {
            if (++w.kc < nchunk) return;
            w.kc = 0;
            if (++w.pol < p.P) return;
            w.pol = 0;
            if (++w.tile < p.tiles) return;
            w.tile = 0;
            if (++w.c < p.C) return;
            w.c = 0;
            ++w.s;
        };
        const long long nq = (u1 - u0) * p.P * nchunk;
        const uint32_t t_stride = (uint32_t)(p.P * row_bytes);  // bytes between samples of one pol
        Walk wi, wc;
        walk_init(wi);
        walk_init(wc);
        static_assert(kTile * 8 == kItems * kProd, "items per chunk");
        // copy items: row tc0 + 32 j, group gc (16 bytes of row t stored at
        // group g ^ (t & 7): conflict-free reads below)
        const int tc0 = tid >> 3, gc = tid & 7;
        const uint32_t src0 = (uint32_t)tc0 * t_stride + (uint32_t)gc * 16;
        const uint32_t dst0 = (uint32_t)tc0 * 128 + (uint32_t)((gc ^ (tc0 & 7)) * 16);
        // widening items: row tw0 + 32 j, group gw
        const int tw0 = (tid & 7) + 8 * (tid >> 6), gw = (tid >> 3) & 7;
        const uint32_t rd0 = (uint32_t)tw0 * 128 + (uint32_t)((gw ^ (tw0 & 7)) * 16);
        const uint32_t wr0 = (uint32_t)(tw0 >> 3) * kAMNs + (uint32_t)(tw0 & 7) * 16 + (uint32_t)(2 * gw) * kAKs;
        auto issue = [&](long long q) {                        // cp.async of chunk q into its int8 stage
            if (q < nq) {
                const int t0 = wi.tile * kTile;
                const int8_t *base = p.volt + ((((size_t)wi.s * p.C + wi.c) * p.T + t0) * p.P + wi.pol) * row_bytes +
                                     (size_t)wi.kc * kChunkE * 2;
                uint8_t *dst = sI8 + (q % kI8Stages) * kI8Bytes + dst0;
                const int t_valid = p.T - t0 - tc0;
                const bool g_ok = gc * 8 < p.ne - wi.kc * kChunkE;
#pragma unroll
                for (int j = 0; j < kItems; j++) {
                    const bool ok = g_ok && 32 * j < t_valid;
                    const int8_t *src = ok ? base + src0 + (size_t)(32 * j) * t_stride : p.volt;
                    cp_async16(dst + 32 * 128 * j, src, ok ? 16u : 0u);
                }
                walk_next(wi);
            }
            cp_async_commit();
        };
        for (int q = 0; q < kAhead; q++) issue(q);
        for (long long q = 0; q < nq; q++, gq++) {
            const int s = wc.s;
            walk_next(wc);
            issue(q + kAhead);             // its ring slot was drained at the end of iteration q - 1
            cp_async_wait<kAhead>();
            const int slot = (int)(gq % kAStages);
            if (gq >= kAStages) tc::mbar_wait(&mb_empty[slot], (uint32_t)(((gq / kAStages) - 1) & 1), p.status);
            if (s != cur_s) {
                // new station: every MMA issued so far has completed (the empty
                // barrier of the previous chunk), so B can be rewritten
                if (gq >= 1) {
                    const long long pq = gq - 1;
                    tc::mbar_wait(&mb_empty[pq % kAStages], (uint32_t)((pq / kAStages) & 1), p.status);
                }
                for (int it = tid; it < (int)(p.P * bbytes / 16); it += kProd)
                    reinterpret_cast<uint4 *>(sB)[it] = make_uint4(0, 0, 0, 0);
                bar_prod();
                for (int it = tid; it < p.P * p.K * p.ne; it += kProd) {   // (pol, beam, element)
                    const int a = it % p.ne, kk = (it / p.ne) % p.K, pp = it / (p.ne * p.K);
                    const char2 wv = reinterpret_cast<const char2 *>(p.w)[(((size_t)s * p.K + kk) * p.P + pp) * p.ne + a];
                    const __half wr = __int2half_rn(wv.x), wi = __int2half_rn(wv.y), nwi = __int2half_rn(-(int)wv.y);
                    uint8_t *B = sB + pp * bbytes;
                    // row 2kk: (wr, wi); row 2kk+1: (-wi, wr)
                    *reinterpret_cast<__half2 *>(B + tc::off_kmajor(2 * kk, 2 * a, kAKs, bmns)) = __halves2half2(wr, wi);
                    *reinterpret_cast<__half2 *>(B + tc::off_kmajor(2 * kk + 1, 2 * a, kAKs, bmns)) = __halves2half2(nwi, wr);
                }
                cur_s = s;
            }
            bar_prod();                                        // int8 stage landed for all threads
            const uint8_t *src = sI8 + (q % kI8Stages) * kI8Bytes + rd0;
            uint8_t *A = sA + slot * kABytes + wr0;
#pragma unroll
            for (int j = 0; j < kItems; j++) {                 // rows tw0 + 32 j: A row groups + 4 j
                const int4 raw = *reinterpret_cast<const int4 *>(src + 32 * 128 * j);
                uint4 lo, hi;
                widen16(raw, lo, hi);
                *reinterpret_cast<uint4 *>(A + 4 * kAMNs * j) = lo;
                *reinterpret_cast<uint4 *>(A + 4 * kAMNs * j + kAKs) = hi;
            }
            tc::fence_proxy_async();
            tc::mbar_arrive(&mb_full[slot]);
            bar_prod();                                        // int8 stage may be refilled
        }
        cp_async_wait<0>();
    } else if (warp == kMmaWarp) {
        // ============================================================ MMA
        if (lane == 0) {
            long long gq = 0, gu = 0;
            for (long long u = u0; u < u1; u++, gu++) {
                const int b = (int)(gu & 1);
                if (gu >= 2) tc::mbar_wait(&mb_dempty[b], (uint32_t)(((gu >> 1) - 1) & 1), p.status);
                tc::fence_after();
                for (int pol = 0; pol < p.P; pol++) {
                    const uint32_t d = tmem + (uint32_t)b * dcols + (uint32_t)pol * ncols;
                    const uint32_t bb = tc::smem_u32(sB + pol * bbytes);
                    for (int kc = 0; kc < nchunk; kc++, gq++) {
                        const int slot = (int)(gq % kAStages);
                        tc::mbar_wait(&mb_full[slot], (uint32_t)((gq / kAStages) & 1), p.status);
                        tc::fence_after();
                        const uint32_t a = tc::smem_u32(sA + slot * kABytes);
#pragma unroll
                        for (int s = 0; s < 8; s++)
                            tc::mma_f16(d, tc::desc(a + s * 2 * kAKs, kAKs, kAMNs),
                                        tc::desc(bb + (kc * 16 + s * 2) * kAKs, kAKs, bmns), idesc,
                                        (kc > 0 || s > 0) ? 1u : 0u);
                        tc::mma_commit(&mb_empty[slot]);
                    }
                }
                tc::mma_commit(&mb_dfull[b]);
            }
        }
    } else {
        // ============================================================ epilogue
        const int q = warp & 3;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        const int t_local = q * 32 + lane;
        long long gu = 0;
        int sat = 0;
        for (long long u = u0; u < u1; u++, gu++) {
            const int b = (int)(gu & 1);
            tc::mbar_wait(&mb_dfull[b], (uint32_t)((gu >> 1) & 1), p.status);
            tc::fence_after();
            const int s = (int)(u / ((long long)p.C * p.tiles));
            const int c = (int)((u / p.tiles) % p.C);
            const int t = (int)(u % p.tiles) * kTile + t_local;
            const size_t row = (((size_t)s * p.C + c) * p.T + t) * p.K * p.P * 2;   // [s][c][t][k][p][2]
            // 8 beams at a time: both pols' (re, im) of beams k0..k0+7, in output order
            for (int c0 = 0; c0 < ncols; c0 += 16) {
                int v[2][16];
#pragma unroll
                for (int pol = 0; pol < 2; pol++) {
                    if (pol < p.P) {
                        uint32_t r[16];
                        tc::tmem_ld16(tmem + lane_base + (uint32_t)b * dcols + (uint32_t)(pol * ncols + c0), r);
                        tc::tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 16; j++) v[pol][j] = __float2int_rn(__uint_as_float(r[j]));
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; j++) v[pol][j] = 0;
                    }
                }
                if (t >= p.T) continue;
                const int k0 = c0 >> 1;
                if (p.shift < 0) {
                    int32_t *o = reinterpret_cast<int32_t *>(p.beams) + row + (size_t)k0 * p.P * 2;
                    if (p.P == 2) {
#pragma unroll
                        for (int j = 0; j < 8; j++)             // beam k0 + j: X (re, im), Y (re, im)
                            reinterpret_cast<int4 *>(o)[j] = make_int4(v[0][2 * j], v[0][2 * j + 1], v[1][2 * j],
                                                                       v[1][2 * j + 1]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; j++)
                            reinterpret_cast<int4 *>(o)[j] = make_int4(v[0][4 * j], v[0][4 * j + 1], v[0][4 * j + 2],
                                                                       v[0][4 * j + 3]);
                    }
                } else {
                    uint32_t wds[8];                             // P = 2: 8 words; P = 1: 4
#pragma unroll
                    for (int j = 0; j < 8; j++) {                // beam k0 + j
                        const uint32_t b0 = (uint8_t)requant(v[0][2 * j], p.shift, sat);
                        const uint32_t b1 = (uint8_t)requant(v[0][2 * j + 1], p.shift, sat);
                        if (p.P == 2) {
                            const uint32_t b2 = (uint8_t)requant(v[1][2 * j], p.shift, sat);
                            const uint32_t b3 = (uint8_t)requant(v[1][2 * j + 1], p.shift, sat);
                            wds[j] = b0 | (b1 << 8) | (b2 << 16) | (b3 << 24);
                        } else {
                            const uint32_t h = b0 | (b1 << 8);
                            if (j & 1) wds[j >> 1] |= h << 16;
                            else wds[j >> 1] = h;
                        }
                    }
                    int8_t *o = reinterpret_cast<int8_t *>(p.beams) + row + (size_t)k0 * p.P * 2;
                    if (p.P == 2) {                              // 32 bytes
                        reinterpret_cast<uint4 *>(o)[0] = make_uint4(wds[0], wds[1], wds[2], wds[3]);
                        reinterpret_cast<uint4 *>(o)[1] = make_uint4(wds[4], wds[5], wds[6], wds[7]);
                    } else {                                     // P = 1: 16 bytes
                        reinterpret_cast<uint4 *>(o)[0] = make_uint4(wds[0], wds[1], wds[2], wds[3]);
                    }
                }
            }
            tc::fence_before();
            tc::mbar_arrive(&mb_dempty[b]);
        }
        if (p.nsat) {
            for (int o = 16; o; o >>= 1) sat += __shfl_xor_sync(0xffffffffu, sat, o);
            if (lane == 0 && sat) atomicAdd(p.nsat, (unsigned long long)sat);
        }
    }

    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, alloc);
}

}  // namespace

extern "C" hai_status hai_beamform(hai_ctx *ctx, const int8_t *volt, const int8_t *w, int S, int C, int T, int K,
                                   int N, int P, int requant_shift, void *beams, long long *n_saturated,
                                   void *stream) {
    if (!ctx) return hai_fail(HAI_ERR_INVALID_ARG, "hai_beamform: ctx is NULL");
    if (S < 0 || C < 0 || T < 0 || K <= 0 || N <= 0 || (P != 1 && P != 2) || requant_shift > 30)
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_beamform: bad size, polarisation count or shift");
    if (N % 8 != 0 || N > 512 || (2 * K) % 16 != 0 || K > 64)
        return hai_fail(HAI_ERR_UNSUPPORTED,
                        "hai_beamform: this build needs N a multiple of 8 and <= 512 (exact FP32 block), "
                        "K a multiple of 8 and <= 64");
    if ((long long)S * C * T == 0) return HAI_OK;
    if (!volt || !w || !beams) return hai_fail(HAI_ERR_INVALID_ARG, "hai_beamform: NULL buffer");
    if ((((uintptr_t)volt) & 15) != 0 || (((uintptr_t)beams) & 15) != 0)
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_beamform: volt and beams must be 16-byte aligned");
    if (hai_fault_injected("launch")) return hai_fail(HAI_ERR_CUDA, "hai_beamform: injected launch failure");
    HAI_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    BfParams p;
    p.volt = volt;
    p.w = w;
    p.S = S;
    p.C = C;
    p.T = T;
    p.K = K;
    p.ne = N;
    p.P = P;
    p.tiles = (T + kTile - 1) / kTile;
    p.nunits = (long long)S * C * p.tiles;
    const int grid = (int)std::min<long long>(p.nunits, ctx->num_sms);
    p.per_cta = (p.nunits + grid - 1) / grid;
    p.shift = requant_shift;
    p.beams = beams;
    p.nsat = reinterpret_cast<unsigned long long *>(n_saturated);
    p.status = ctx->d_status;
    const size_t bbytes = (size_t)(2 * K / 8) * ((N + kChunkE - 1) / kChunkE * kChunkE) * 32;
    const size_t smem = kI8Stages * kI8Bytes + kAStages * kABytes + (size_t)P * bbytes;
    if (smem > (size_t)ctx->smem_optin)
        return hai_fail(HAI_ERR_UNSUPPORTED, "hai_beamform: weights of one station exceed shared memory");
    HAI_CUDA_TRY(cudaFuncSetAttribute(bf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int pidx = prof_begin(ctx, st);
    bf_kernel<<<grid, kThreads, smem, st>>>(p);
    prof_end(ctx, pidx, st);
    prof_count(ctx, 1);
    HAI_CUDA_TRY(cudaGetLastError());
    return HAI_OK;
}
