// rt_stage.cuh -- staging of the scene table into shared memory: one TMA bulk copy
// (cp.async.bulk, completion counted on an mbarrier) or a cooperative copy by all
// threads.  Every wait is bounded; on expiry the CTA flags the device error word,
// waits (bounded again) for its own copy to land, and tells the caller to return.
#pragma once

#include "rt_device.cuh"

namespace rtd {

constexpr uint32_t kErrStageTimeout = 1u;
constexpr uint32_t kErrQueueTimeout = 2u;
constexpr uint32_t kWaitLimit = 1u << 24;  // try_wait polls before giving up

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity` of the barrier.  Returns false on expiry.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit = kWaitLimit) {
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Copy `bytes` (multiple of 16, both addresses 16-byte aligned) from global src to
// shared dst.  staging == 1: TMA bulk copy issued by thread 0; otherwise all
// threads copy 16-byte words.  `bar` is a shared mbarrier initialised by the
// caller (count 1) and `phase` its current parity (flipped here on use).  All
// threads of the CTA must call.  Returns false when the CTA must return.
__device__ __forceinline__ bool stage_to_smem(void* dst, const void* src, uint32_t bytes, int staging,
                                              uint64_t* bar, uint32_t& phase, uint32_t* err_word) {
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nth = blockDim.x * blockDim.y;
    if (staging == 1) {
        if (tid == 0) {
            mbar_arrive_expect_tx(bar, bytes);
            bulk_copy_g2s(dst, src, bytes, bar);
        }
        const bool ok = mbar_wait_bounded(bar, phase);
        if (!ok) {
            if (tid == 0) atomicOr(err_word, kErrStageTimeout);
            mbar_wait_bounded(bar, phase);  // let the copy in flight land before leaving
        }
        phase ^= 1u;
        // A CTA leaves only as a whole.
        return __syncthreads_and(ok) != 0;
    }
    const float4* s = reinterpret_cast<const float4*>(src);
    float4* d = reinterpret_cast<float4*>(dst);
    for (uint32_t i = tid; i < bytes / 16; i += nth) d[i] = __ldg(s + i);
    __syncthreads();
    return true;
}

}  // namespace rtd
