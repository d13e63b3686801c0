// ptx.cuh -- inline-PTX helpers for sm_103a kernels: mbarriers, 1-D bulk
// copies (TMA, cp.async.bulk), proxy fences and bounded waits.
//
// Every wait here is bounded. A wait that runs out sets a bit in the
// caller's device error word and returns false. The host turns that into
// TC_ETIMEOUT. No kernel traps or spins forever.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tc {

// Device error word bits.
enum : int { ERR_TIMEOUT_TMA = 1, ERR_TIMEOUT_MMA = 2, ERR_BAD_ARGS = 4 };

// Limit of a bounded wait, in nanoseconds of %globaltimer.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

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

// Makes the mbarrier initialisation visible to the async proxy (TMA, tcgen05).
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Orders this thread's generic-proxy shared-memory accesses before later
// async-proxy accesses (a TMA write into the same buffer).
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Plain arrive (no transaction bytes): completes the phase of a count-1 barrier.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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

// Iteration backstop of every bounded wait, beside its time limit: a wait
// also ends after this many polls (at least seconds), even if %globaltimer
// were not to advance.
constexpr uint32_t kWaitMaxPolls = 1u << 30;

// Polls mbarrier `bar` for phase `parity` until the phase completes (true), or
// limit_ns of %globaltimer or kWaitMaxPolls polls have passed, or *abort
// (checked every 256 polls) is nonzero (false). On a timeout, ORs errbit into
// *err (err may be NULL); on an abort, leaves *err to the role that failed.
__device__ __forceinline__ bool mbar_wait_limited(uint64_t *bar, uint32_t parity, int *err, int errbit,
                                                  unsigned long long limit_ns, const volatile int *abort = nullptr)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const unsigned long long t0 = globaltimer_ns();
    for (uint32_t it = 0; it < kWaitMaxPolls; ++it) {
        if (mbar_try_wait(bar, parity))
            return true;
        if ((it & 255u) == 255u) {
            if (abort && *abort)
                return false;
            if (globaltimer_ns() - t0 > limit_ns)
                break;
        }
    }
    if (err)
        atomicOr(err, errbit);
    return false;
}

// The kernels' waits: at most kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *err, int errbit)
{
    return mbar_wait_limited(bar, parity, err, errbit, kWaitLimitNs);
}

// 1-D bulk copy global -> shared, completing `bytes` of transaction count on
// `bar`. dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace tc
