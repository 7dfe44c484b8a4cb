// mbarrier.cuh -- shared-memory barriers, bulk copies and bounded waits used
// by the kernels that move data with the asynchronous copy engine (TMA).
//
// Every wait on an mbarrier is bounded in time: a wait that gives up sets a
// flag shared by the CTA and the context's status word (read back by
// spec_ctx_check as SPEC_ETIMEOUT), so that a copy or product that never
// completes ends in an error status instead of a kernel that never returns.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace spec {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make the initialised barriers visible to the asynchronous proxy
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

struct Guard {
    volatile int* abort;       // shared: set by the first wait that gives up
    unsigned* status;          // global: the context's status word
    uint64_t timeout_ns;
};

// Wait for the phase of `bar` with parity `parity`, at most timeout_ns; on
// a timeout flag the CTA and the context.  Returns false if the CTA aborts.
__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity, const Guard& g) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gtime();
    while (!mbar_try_wait(bar, parity)) {
        if (*g.abort) return false;
        if (gtime() - t0 > g.timeout_ns) {
            *g.abort = 1;
            atomicOr(g.status, 1u);
            return false;
        }
    }
    return true;
}

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to this CTA's shared memory, counted on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

}  // namespace spec
