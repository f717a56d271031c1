// Bulk asynchronous copies global -> shared memory completed on an mbarrier
// (sm_90 and later; used here for sm_103a).  One thread arms the barrier
// with the byte count it expects and issues the copies; the copy engine
// counts the bytes down and completes the barrier's phase, which the
// consumers wait on with try_wait.parity.  Every wait is bounded: after a
// time limit it gives up and the kernel records SPMV_ERR_TIMEOUT in a device
// status word instead of spinning forever.
#pragma once

#include <stdint.h>

namespace spmv {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned arrivals) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(arrivals) : "memory");
}

// makes initialised barriers visible to the copy engine (async proxy)
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// the calling thread's arrival, announcing `bytes` of copies to come
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// bytes (a multiple of 16) from 16-byte aligned global src to 16-byte aligned
// shared dst, counted on bar
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
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

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// waits for the phase of the given parity to complete; false once `limit_ns`
// nanoseconds have passed without it
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

// orders this thread's earlier shared-memory accesses before later copies of
// the copy engine into the same shared memory
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// device status word bits (reported by spmv_check)
constexpr unsigned STATUS_TIMEOUT = 1u;
constexpr unsigned STATUS_BOUNDS = 2u;

// time a kernel waits for a copy before it gives up: one second, far beyond
// any copy's completion time
constexpr uint64_t MBAR_WAIT_NS = 1000000000ull;

}  // namespace spmv
