// Tensor-memory-accelerator (TMA) loads and mbarriers for the column passes
// (inline PTX, sm_90+ forms that sm_103a keeps).
//
// A column tile (SLOTS columns x its rows) is a 3-D box of the W1/W2 array,
// copied by one cp.async.bulk.tensor into shared memory; completion is
// signalled on an mbarrier through its transaction count.  Waits are bounded:
// a wait that runs out reports false, and the caller records a timeout in
// the plan's status word instead of spinning forever.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pgb {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make the initialised barrier visible to the async (TMA) proxy
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this CTA's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) writes to the same buffer
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// One poll: suspends for at most kMbarPollNs (the explicit time hint bounds
// each poll, so max_polls bounds the whole wait in time as well).
constexpr unsigned kMbarPollNs = 1000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kMbarPollNs)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity` of bar to complete (at most about
// max_polls microseconds).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int max_polls) {
    for (int i = 0; i < max_polls; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// 3-D tiled TMA load of the box at coordinates (c0, c1, c2) into dst,
// completing transaction bytes on bar.  c0 * element size must be a
// multiple of 16 bytes; dst 128-byte aligned.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

// Host: encode a 3-D FP32 tensor map (dims and box in elements, strides of
// dims 1 and 2 in bytes) through the driver entry point.
cudaError_t tma_encode_3d_f32(CUtensorMap* map, const void* base, const unsigned long long dims[3],
                              const unsigned long long strides[2], const unsigned box[3]);

}  // namespace pgb
