// Bulk (TMA engine) copies from global to shared memory completed on an
// mbarrier, with a bounded wait (the dedispersion kernels), and 8-byte
// asynchronous copies with zero fill (the double-buffered FFT and plane
// kernels).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pss {

constexpr int WAIT_LIMIT = 1 << 22;  // polls before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Wait for the phase of `parity` to complete: up to WAIT_LIMIT blocking polls
// (try_wait), or, with test_polls > 0 (a context's short limit for tests),
// that many non-blocking polls (test_wait); false when they run out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int test_polls = 0) {
    const uint32_t a = smem_u32(bar);
    if (test_polls > 0) {
        for (int i = 0; i < test_polls; ++i) {
            uint32_t ok;
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                : "=r"(ok)
                : "r"(a), "r"(parity)
                : "memory");
            if (ok) return true;
        }
        return false;
    }
    for (int i = 0; i < WAIT_LIMIT; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// 8-byte global -> shared copy; src_bytes < 8 fills the rest with zeros
// (src_bytes 0 reads nothing)
__device__ __forceinline__ void cp_async8(void* dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

}  // namespace pss
