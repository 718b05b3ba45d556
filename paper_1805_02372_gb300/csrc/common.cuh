// Shared device helpers of the sm_103a Toeplitz-hash library: bit access, TMA
// bulk copies with mbarriers and bounded waits, device status words.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace pa {

// Bounded waits are limited in time (the global nanosecond timer), not in polls: one
// mbarrier poll may suspend the thread for a hardware-chosen interval. A wait gives up
// after kWaitNs and reports PA_ERR_TIMEOUT; a wait that only lets copies already in
// flight land before the kernel returns is limited to kDrainNs.
constexpr uint64_t kWaitNs = 4000000000ull;
constexpr uint64_t kDrainNs = 500000000ull;

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void set_status(int *status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// ---- mbarrier + bulk async copy (TMA engine, non-tensor form) ----

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// Global -> shared bulk copy completing on bar. dst, src 16-byte aligned; bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Wait for phase completion with an iteration limit. On timeout the status word
// records PA_ERR_TIMEOUT, and a second bounded wait gives copies still in flight
// time to land before the caller returns. Returns true when the phase completed.
// Polls the phase until it completes or `limit_ns` have passed since the first poll.
__device__ __forceinline__ bool mbar_wait_for(uint64_t *bar, uint32_t phase, uint64_t limit_ns) {
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try_wait(bar, phase)) return true;
        if ((i & 15u) == 15u && global_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, int *status) {
    if (mbar_wait_for(bar, phase, kWaitNs)) return true;
    set_status(status, PA_ERR_TIMEOUT);
    mbar_wait_for(bar, phase, kDrainNs);
    return false;
}

// ---- counters between CTAs of one launch ----

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool wait_count(const uint32_t *c, uint32_t target, int *status, int *flag) {
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint64_t t0 = global_ns();
        while (ld_acquire(c) < target) {
            if (global_ns() - t0 > kWaitNs) {
                set_status(status, PA_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        *flag = ok;
    }
    __syncthreads();
    return *flag != 0;
}

// Release of a CTA's global writes to the CTAs that wait on counter c: the barrier orders
// every thread's writes before thread 0's GPU-scope fence, which (being cumulative) orders
// them before the counter increment; a waiter's acquire load of the counter then sees them
// (the pattern of a grid-wide barrier: one fence per CTA, not one per thread).
__device__ __forceinline__ void signal_count(uint32_t *c) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(c, 1u);
    }
}

// signal_count for `count` consecutive counters (one barrier and fence for all of them)
__device__ __forceinline__ void signal_counts(uint32_t *c, uint32_t count) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        for (uint32_t i = 0; i < count; ++i) atomicAdd(c + i, 1u);
    }
}

// ---- bit helpers ----

__device__ __forceinline__ uint64_t ceil_div_dev(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

// 32 bits of a packed string starting at bit position `bit` (may be negative:
// positions < 0 read as 0). `words` is the number of valid 32-bit words; positions
// past them read as 0.
__device__ __forceinline__ uint32_t bits32_at(const uint32_t *__restrict__ v, uint64_t words,
                                              int64_t bit) {
    int64_t w = bit >> 5;  // arithmetic shift: floor division
    uint32_t sh = static_cast<uint32_t>(bit & 31);
    uint32_t lo = (w >= 0 && static_cast<uint64_t>(w) < words) ? __ldg(v + w) : 0u;
    uint32_t hi = (w + 1 >= 0 && static_cast<uint64_t>(w + 1) < words) ? __ldg(v + w + 1) : 0u;
    return __funnelshift_r(lo, hi, sh);
}

}  // namespace pa
