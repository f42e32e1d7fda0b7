// sm_103a building blocks written as inline PTX: tcgen05 MMA (kind::f16,
// FP32 accumulation in tensor memory), TMEM allocation and loads, mbarriers
// with bounded waits, and TMA bulk copies.
//
// Shared-memory operand descriptors use the no-swizzle canonical layouts:
// a "core matrix" is 8 rows of 16 contiguous bytes.  K-major: rows are
// M/N indices and the 16 bytes hold 8 consecutive K values.  MN-major: rows
// are K indices and the 16 bytes hold 8 consecutive M/N values.  In both
// the descriptor's leading byte offset is the distance between core matrices
// adjacent along K and the stride byte offset the distance between core
// matrices adjacent along M/N.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "hai_internal.h"

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (mn, k) of a 16-bit operand, K-major no-swizzle.
__host__ __device__ __forceinline__ uint32_t off_kmajor(int mn, int k, uint32_t k_stride,
                                                       uint32_t mn_stride) {
    return (uint32_t)(mn >> 3) * mn_stride + (uint32_t)(k >> 3) * k_stride + (mn & 7) * 16 + (k & 7) * 2;
}

// Byte offset of element (mn, k) of a 16-bit operand, MN-major no-swizzle.
__host__ __device__ __forceinline__ uint32_t off_mnmajor(int mn, int k, uint32_t k_stride,
                                                        uint32_t mn_stride) {
    return (uint32_t)(k >> 3) * k_stride + (uint32_t)(mn >> 3) * mn_stride + (k & 7) * 16 + (mn & 7) * 2;
}

// Shared-memory matrix descriptor (no swizzle, descriptor version 1).
__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t k_stride, uint32_t mn_stride) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((k_stride >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((mn_stride >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16 with FP16 A and B, FP32 accumulator.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, int a_mn_major, int b_mn_major) {
    return (1u << 4) | ((uint32_t)a_mn_major << 15) | ((uint32_t)b_mn_major << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// The same with both A and B in BF16 (A format bits 7-9 and B format bits
// 10-12 set to 1).  One MMA never mixes FP16 and BF16 operands.
__host__ __device__ constexpr uint32_t idesc_f16_as(bool bf16, int M, int N, int a_mn_major, int b_mn_major) {
    return idesc_f16(M, N, a_mn_major, b_mn_major) | (bf16 ? ((1u << 7) | (1u << 10)) : 0u);
}

// D[tmem] (+)= A * B^T, issued by one thread.
__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

// Arrive on the mbarrier once all MMAs issued so far by this thread complete.
__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Make generic-proxy shared-memory writes visible to the async proxy (MMA, TMA).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------------- TMEM
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 lanes x 4 consecutive 32-bit columns.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}

// 32 lanes x 8 consecutive 32-bit columns.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

// 32 lanes x 16 consecutive 32-bit columns: thread i of the warp receives
// lane (quadrant base + i), columns taddr.col .. +15.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// the inverse of tmem_ld16: thread i writes lane (quadrant base + i),
// columns taddr.col .. +15
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
        ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
          "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t *m) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(m)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *m, uint32_t bytes) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
                     smem_u32(m)),
                 "r"(bytes)
                 : "memory");
}

// Test the phase; the hardware may suspend the thread for a short while
// (hint: 20 us) while the phase is incomplete.
__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t *m, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(m)), "r"(parity), "r"(20000u)
        : "memory");
    return done;
}

// Bounded wait for the phase with the given parity to complete.  Polls
// try_wait (which may suspend the thread in hardware until the phase flips)
// and reads the device status word only once every 2^14 cycles of waiting,
// so a wait that ends within a few microseconds never leaves the SM.  Gives
// up after `limit` SM cycles (default 2^32, about two seconds; checked at the
// same 2^14-cycle points), or at the next check once another wait of the
// launch has given up, flagging HAI_DEV_TIMEOUT in the status word and
// returning false; the caller carries on so that every thread still reaches
// every barrier and the kernel ends.
constexpr long long kWaitLimitCycles = 1ll << 32;

__device__ __forceinline__ bool mbar_wait(uint64_t *m, uint32_t parity, unsigned *status,
                                          long long limit = kWaitLimitCycles) {
    if (mbar_try_wait(m, parity)) return true;
    const long long t0 = clock64();
    long long next_check = 1ll << 14;
    for (;;) {
        if (mbar_try_wait(m, parity)) return true;
        const long long dt = clock64() - t0;
        if (dt > next_check) {
            if (*reinterpret_cast<volatile unsigned *>(status) & HAI_DEV_TIMEOUT) return false;
            if (dt > limit) {
                atomicOr(status, (unsigned)HAI_DEV_TIMEOUT);
                return false;
            }
            next_check = dt + (1ll << 14);
            __nanosleep(128);
        }
    }
}

// ---------------------------------------------------------------- TMA bulk copy
// Global -> shared copy of `bytes` (multiple of 16, both addresses 16-byte
// aligned) completing on the mbarrier's transaction count.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *m) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(m))
        : "memory");
}

// One 32-byte store to global memory (32-byte aligned address).
__device__ __forceinline__ void st_global_v8(void *p, uint4 lo, uint4 hi) {
    asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(lo.x), "r"(lo.y), "r"(lo.z),
                 "r"(lo.w), "r"(hi.x), "r"(hi.y), "r"(hi.z), "r"(hi.w)
                 : "memory");
}

// Prefetch `bytes` (multiple of 16, 16-byte aligned) of global memory into L2,
// so that a later bulk copy of them is an L2 hit.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------- clusters
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Every thread of every CTA of the cluster arrives and waits.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release;\n barrier.cluster.wait.acquire;" ::: "memory");
}

// Shared-memory address of the same variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t peer_addr(uint32_t local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}

// 32-bit and 128-bit stores to shared memory of any CTA of the cluster
// (cluster address from peer_addr).
__device__ __forceinline__ void st_cluster(uint32_t addr, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void st_cluster_v4(uint32_t addr, uint4 v) {
    asm volatile("st.shared::cluster.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w)
                 : "memory");
}

// Make this thread's generic-proxy writes to cluster shared memory visible
// to the async proxy (the tensor cores of the CTAs that own it).
__device__ __forceinline__ void fence_proxy_async_cluster() {
    asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
}

// Arrive (release at cluster scope) on an mbarrier of any CTA of the cluster.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t mbar_cluster) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(mbar_cluster) : "memory");
}

// Local shared -> shared of another CTA of the cluster, `bytes` (multiple of
// 16, 16-byte aligned), completing on that CTA's mbarrier (cluster address).
__device__ __forceinline__ void bulk_s2peer(uint32_t dst_cluster, const void *src, uint32_t bytes,
                                            uint32_t mbar_cluster) {
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst_cluster),
        "r"(smem_u32(src)), "r"(bytes), "r"(mbar_cluster)
        : "memory");
}

// Arrive on the mbarrier at the same offset in every CTA of `mask` once all
// MMAs issued so far by this thread complete.
__device__ __forceinline__ void mma_commit_multicast(uint64_t *mbar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(mbar)),
        "h"(mask)
        : "memory");
}

// try_wait with cluster-scope acquire, for phases completed by other CTAs;
// no suspend-time hint, so the poll returns after the hardware's own short
// wait rather than sleeping through a remote completion.
__device__ __forceinline__ uint32_t mbar_try_wait_cluster(uint64_t *m, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(m)), "r"(parity)
        : "memory");
    return done;
}

__device__ __forceinline__ bool mbar_wait_cluster(uint64_t *m, uint32_t parity, unsigned *status) {
    if (mbar_try_wait_cluster(m, parity)) return true;
    const long long t0 = clock64();
    long long next_check = 1ll << 14;
    for (;;) {
        if (mbar_try_wait_cluster(m, parity)) return true;
        const long long dt = clock64() - t0;
        if (dt > next_check) {
            if (*reinterpret_cast<volatile unsigned *>(status) & HAI_DEV_TIMEOUT) return false;
            if (dt > (1ll << 32)) {
                atomicOr(status, (unsigned)HAI_DEV_TIMEOUT);
                return false;
            }
            next_check = dt + (1ll << 14);
            __nanosleep(128);
        }
    }
}

__device__ __forceinline__ uint32_t pack_half2(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ uint32_t pack_bf162(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// Two values rounded to the 16-bit operand type (FP16, or BF16 if BF) and
// packed (a in the low half).
template <bool BF>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    if constexpr (BF) return pack_bf162(a, b);
    else return pack_half2(a, b);
}

// x rounded to the operand type, as a float.
template <bool BF>
__device__ __forceinline__ float round_op(float x) {
    if constexpr (BF) return __bfloat162float(__float2bfloat16_rn(x));
    else return __half2float(__float2half_rn(x));
}

// Split operands: hi = the two values rounded to the operand type, lo = their
// remainders x - hi rounded to it (hi + lo carries ~2x the type's bits).
template <bool BF>
__device__ __forceinline__ void pack2_split(float a, float b, uint32_t &hi, uint32_t &lo) {
    hi = pack2<BF>(a, b);
    lo = pack2<BF>(a - round_op<BF>(a), b - round_op<BF>(b));
}

}  // namespace tc
