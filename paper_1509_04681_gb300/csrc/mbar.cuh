// mbarrier and bulk-copy (TMA) helpers shared by the tensor-core contraction and the sweeps.
// Every wait has a wall-clock deadline, so that no kernel can spin forever on a copy that
// never lands.
#pragma once

#include "common.cuh"

namespace cggm {

constexpr uint64_t kMbarWaitNs = 1000000000ull;  // 1 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: true when the phase completed, false (and *err set) at the deadline or,
// with give_up_on_err, as soon as another thread of the kernel has recorded a failure.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, int *err,
                                          bool give_up_on_err = true) {
    if (mbar_try(b, parity)) return true;
    const uint64_t t0 = global_ns();
    for (unsigned it = 1;; it++) {
        if (mbar_try(b, parity)) return true;
        if ((it & 255u) == 0) {
            if (give_up_on_err && *(volatile int *)err != 0) return false;
            if (global_ns() - t0 > kMbarWaitNs) {
                atomicCAS(err, 0, (int)DEV_TIMEOUT);
                return false;
            }
        }
    }
}

// Orders this thread's earlier generic-proxy accesses (and those made visible to it) before
// its later async-proxy (TMA) operations.
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async;" ::: "memory");
}

// Untiled bulk copy global -> shared of `bytes` (both addresses 16-byte aligned, bytes a
// multiple of 16), completing on mbar with that many transaction bytes.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(mbar))
        : "memory");
}

}  // namespace cggm
