// Bulk asynchronous copies (TMA, cp.async.bulk) from global to shared memory
// with mbarrier completion, for operators that stream through the SMs once
// per product.  Every wait is bounded: a copy that does not complete within
// the limit reports failure instead of hanging.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nnqp {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}

// Makes initialised mbarriers visible to the async proxy (the bulk copies).
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrives on b and announces `bytes` of bulk-copy transactions for its phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}

// Orders this thread's earlier generic-proxy accesses of shared memory (the
// reads of a buffer slot) before later async-proxy writes into it.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// L2 policy for data read once per product: evict first, so that the
// vectors the product gathers stay in L2.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// bytes (a multiple of 16; both addresses 16-byte aligned) from global src to
// shared dst, completing as transactions on mbarrier b.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, uint64_t *b,
                                              uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(b)), "l"(policy)
        : "memory");
}

// Waits until the phase of b with the given parity has completed; gives up
// after about 2^22 polls (each poll may suspend the thread for a while).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *b, unsigned parity) {
    for (int it = 0; it < (1 << 22); ++it) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_addr(b)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace nnqp
