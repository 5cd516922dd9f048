// gc_ptx.cuh -- inline-PTX helpers for Blackwell bulk copies (TMA, 1-D) and
// shared-memory mbarriers.
#pragma once
#include <stdint.h>

__device__ __forceinline__ uint32_t gc_smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void gc_mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(gc_smem_u32(bar)), "r"(count)
                 : "memory");
}

// make barrier initialisation visible to the asynchronous (bulk-copy) proxy
__device__ __forceinline__ void gc_fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's generic-proxy shared-memory accesses before later
// asynchronous-proxy writes to the same memory
__device__ __forceinline__ void gc_fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void gc_mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(gc_smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared, completion counted on `bar` (bytes and
// addresses 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void gc_bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            gc_smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(gc_smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool gc_mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(gc_smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of `bar`, taken by a whole warp (all 32
// lanes call it with the same barrier and parity); false if the limit ran
// out.  The lanes agree after every poll, so they all
// return true together or all false together, and a warp that gives up
// leaves no lane behind at a later full-mask shuffle or __syncwarp.  Once the
// phase has completed every lane's poll sees it, so the agreement costs at
// most one extra poll.
__device__ __forceinline__ bool gc_mbar_wait_bounded_warp(uint64_t *bar, uint32_t parity,
                                                          uint32_t limit)
{
    for (uint32_t i = 0; i < limit; ++i)
        if (__all_sync(0xffffffffu, gc_mbar_try_wait(bar, parity))) return true;
    return false;
}

// 1/sqrt(x) by the hardware approximation (rsqrt.approx, relative error
// below 2^-22) in its flush-to-zero form: the interaction kernel's arguments
// are r^2 + eps^2 >= eps^2 > 0, never subnormal.
__device__ __forceinline__ float gc_rsqrt(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/x by the hardware approximation (rcp.approx, relative error below
// 2^-22) in its flush-to-zero form; the LJ kernel's r^2 is never subnormal.
__device__ __forceinline__ float gc_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Exact float -> double widening on the integer pipe (IEEE 754 binary32 ->
// binary64: rebias the exponent by 1023 - 127, move the 23 fraction bits to
// the top of the 52; a subnormal float is normalised first).  Same value as
// the hardware conversion for every finite input and infinities; NaNs stay
// NaN.  The per-id accumulation widens two floats per row component, and on
// this GPU the FP64 pipe, not memory, bounds that step.
__device__ __forceinline__ double gc_f2d(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t sign = u & 0x80000000u;
    const uint32_t e = (u >> 23) & 0xFFu;
    uint32_t m = u & 0x7FFFFFu;
    uint32_t hi;
    if (e != 0u && e != 255u) {
        hi = sign | ((e + 896u) << 20) | (m >> 3);
    } else if (e == 255u) {
        hi = sign | 0x7FF00000u | (m >> 3) | (m ? 0x80000u : 0u);   // inf, quiet NaN
    } else if (m == 0u) {
        hi = sign;                                                  // signed zero
    } else {
        const uint32_t lz = (uint32_t)__clz((int)m) - 8u;           // to bring the top bit to bit 23
        m = (m << lz) & 0x7FFFFFu;
        hi = sign | ((897u - lz) << 20) | (m >> 3);
    }
    return __hiloint2double((int)hi, (int)(m << 29));
}
