// Shared device helpers of libjac: storage element types, PTX wrappers for
// mbarriers, TMA tensor copies, L2 cache policies and cache-hinted stores, and
// bounded waits.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/jacobi.h"

namespace jac {

// Layout of the first 256 bytes of every sweep workspace.
struct WsHeader {
    int errword;          // JAC_OK or JAC_ETIMEOUT, written by kernels
    unsigned counter;     // CTAs finished (last one reduces and resets)
    unsigned gbar;        // grid barrier between sweeps of one launch
    unsigned pad0;
    double residual;      // default destination of the residual
};
constexpr size_t kWsHeaderBytes = 256;

// Upper bound of a device-side wait before it gives up (nanoseconds).  A
// launch may ask for a shorter bound on the waits that depend on the
// progress of other warps or CTAs (SweepArgs::wait_ns); the waits that only
// let a CTA's own copies land before it exits always keep this one.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Wait for the phase with the given parity to complete; gives up after
// limit_ns and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  unsigned long long limit_ns = kWaitLimitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Order this thread's generic-proxy global accesses with later async-proxy
// (TMA) accesses, in both directions.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }


// Wait until *p >= target (acquire); false after limit_ns.
__device__ __forceinline__ bool wait_counter_bounded(const unsigned *p, unsigned target,
                                                     unsigned long long limit_ns = kWaitLimitNs)
{
    if (ld_acquire_gpu(p) >= target) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (true) {
        __nanosleep(64);
        if (ld_acquire_gpu(p) >= target) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// The workspace error word as it stands (an atomic read, so that the last
// CTA of a launch sees every other CTA's abort).
__device__ __forceinline__ bool workspace_failed(WsHeader *h) { return atomicOr(&h->errword, 0) != 0; }

// 3-D tiled TMA load global -> shared, completion counted on `bar`.
__device__ __forceinline__ void tma_load_3d(void *smem_dst, const CUtensorMap *map, uint64_t *bar, int x, int y,
                                            int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// L2 cache policies for the copies and stores (createpolicy), by mode:
// 0 = normal priority everywhere; 1 = keep the state in L2 (state copies and
// stores evict_last, the streamed coefficients evict_first).
__device__ __forceinline__ uint64_t l2_policy(int evict)
{
    uint64_t p;
    if (evict > 0) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    else if (evict < 0) asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    else asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// 3-D tiled TMA load with an L2 cache policy.
__device__ __forceinline__ void tma_load_3d_hint(void *smem_dst, const CUtensorMap *map, uint64_t *bar, int x, int y,
                                                 int z, uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%3, %4, %5}], [%2], %6;" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z), "l"(policy)
        : "memory");
}

__device__ __forceinline__ void st_v4_hint(float *p, float a, float b, float c, float d, uint64_t policy)
{
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(a), "f"(b), "f"(c),
                 "f"(d), "l"(policy)
                 : "memory");
}

__device__ __forceinline__ void st_v2d_hint(double *p, double a, double b, uint64_t policy)
{
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(p), "d"(a), "d"(b), "l"(policy)
                 : "memory");
}

// Storage element type of array `which` under precision `prec` (host side).
inline size_t elem_bytes(jac_prec prec, int which)
{
    if (prec == JAC_F64) return 8;
    if (prec == JAC_F32) return 4;
    return (which == JAC_P || which == JAC_WRK1) ? 4 : 2;
}

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace jac
