// Inline-PTX wrappers shared by the tensor-core kernels: mbarriers with
// bounded waits, TMA (tiled and plain bulk) copies, TMEM allocation, the
// kind::f16 tcgen05 MMA (BF16 operands, FP32 accumulation) with its
// shared-memory descriptors for K-major tiles of 64-byte rows (64-byte swizzle)
// and of 32-byte rows (32-byte swizzle), TMEM loads, and the three-term BF16
// split.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace {

constexpr int KSTEP = 32;                 // BF16 K elements per 64-byte swizzle row
constexpr int ROWB = 2 * KSTEP;           // bytes per operand row in shared memory
// Waits of the pipeline give up after a limit passed to the kernel (the
// context's setting, ~2 s of clock cycles by default); the waits of the clean-up
// that lets a CTA's own copies and MMAs finish before it frees TMEM and exits
// always use this fixed bound, however short the pipeline limit is.
constexpr long long CLEANUP_WAIT_LIMIT = 4000000000LL;  // clock cycles (~2 s)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// One test of a barrier phase.  While the phase is incomplete the thread may be suspended in
// hardware until it completes or MBAR_SUSPEND_NS pass (measured: waking on completion instead
// of polling takes ~4 % off the chi0 kernel); callers check their time limit between tests.
constexpr uint32_t MBAR_SUSPEND_NS = 10000000;
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(MBAR_SUSPEND_NS)
        : "memory");
    return ok != 0;
}
// Bounded wait by one thread.  Returns false after `limit` clock cycles (which
// also raises the CTA abort flag and the global status) or when another role
// aborted.
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* status, long long limit,
                          bool honour_abort = true) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (honour_abort && *abort_flag) return false;
        if (clock64() - t0 > limit) {
            *abort_flag = 1;
            atomicExch(status, 1);
            return false;
        }
    }
}
// warp-uniform version: lane 0 waits, the result is broadcast
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* status,
                                          long long limit) {
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort_flag, status, limit) ? 1 : 0;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
            "r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// L2 prefetch of one tensor box (no shared memory, no barrier; completes on its own)
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"((uint64_t)map), "r"(x), "r"(y)
                 : "memory");
}
// L2 prefetch of a contiguous range (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_prefetch(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"((uint64_t)src), "r"(bytes) : "memory");
}

// plain bulk copy global -> shared (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// 32 TMEM lanes x 8 columns of 32-bit data into 8 registers per thread (no wait)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
// 32 TMEM lanes x 16 columns of 32-bit data into 16 registers per thread (no wait)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Per-warpgroup register budgets (all four warps of a warpgroup execute the same one): the
// registers a warpgroup gives back can be taken by another; the sum over the warpgroups must
// stay within the registers the block was launched with.
template <uint32_t N> __device__ __forceinline__ void regs_dec() {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(N));
}
template <uint32_t N> __device__ __forceinline__ void regs_inc() {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(N));
}

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;              // leading-dimension offset (unused for swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;     // stride between 8-row groups
    d |= (uint64_t)1 << 46;              // descriptor version
    d |= (uint64_t)4 << 61;              // 64-byte swizzle
    return d;
}
// byte offset of the 16-byte chunk j of row r in a 64-byte-swizzled K-major tile
__device__ __forceinline__ uint32_t sw64_off(int r, int j) {
    return (uint32_t)r * ROWB + ((uint32_t)(j ^ ((r >> 1) & 3)) << 4);
}
// Shared-memory matrix descriptor: K-major, 32-byte swizzle (rows of 32 bytes = 16 BF16), 8-row
// groups 256 bytes apart.
__device__ __forceinline__ uint64_t sw32_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;              // leading-dimension offset (unused for swizzled K-major)
    d |= (uint64_t)(256 >> 4) << 32;     // stride between 8-row groups
    d |= (uint64_t)1 << 46;              // descriptor version
    d |= (uint64_t)6 << 61;              // 32-byte swizzle
    return d;
}
// byte offset of the 16-byte chunk j (0, 1) of row r in a 32-byte-swizzled K-major tile
__device__ __forceinline__ uint32_t sw32_off(int r, int j) {
    return (uint32_t)r * 32u + ((uint32_t)(j ^ ((r >> 2) & 1)) << 4);
}
// kind::f16 instruction descriptor: BF16 x BF16 -> FP32 (A and B type fields 1 = BF16), both
// operands K-major
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}
// (a, b) -> three packed BF16 pairs with a = a0 + a1 + a2, b = b0 + b1 + b2 (each term the
// round-to-nearest BF16 of what the earlier terms leave)
__device__ __forceinline__ void split3(float a, float b, uint32_t& p0, uint32_t& p1, uint32_t& p2) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    p0 = *reinterpret_cast<uint32_t*>(&h);
    const float ra = a - hf.x, rb = b - hf.y;
    __nv_bfloat162 m = __floats2bfloat162_rn(ra, rb);
    const float2 mf = __bfloat1622float2(m);
    p1 = *reinterpret_cast<uint32_t*>(&m);
    p2 = pack_bf16(ra - mf.x, rb - mf.y);
}
__device__ __forceinline__ float2 bf2(uint32_t u) {
    return __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&u));
}
// the terms of (xi, -xr) from those of (xr, xi): swap the halves, negate the new high half
__device__ __forceinline__ uint32_t perm_im(uint32_t re) { return __byte_perm(re, 0u, 0x1032) ^ 0x80000000u; }

}  // namespace
