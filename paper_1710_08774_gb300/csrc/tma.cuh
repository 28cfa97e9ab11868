// tma.cuh -- tensor-memory-accelerator (TMA) staging for the streaming
// kernels: mbarrier completion, tiled tensor copies (cp.async.bulk.tensor)
// and contiguous bulk copies (cp.async.bulk) from this GPU's global memory
// into the CTA's shared memory, and the host-side tensor-map encoding.
//
// Every wait on an mbarrier is bounded: after kTmaSpinLimit polls it records
// a timeout in the caller's error word and returns, so a copy that never
// completes ends the kernel with an error status instead of a hang.  No
// multicast, no clusters: each CTA copies into its own shared memory.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace hfav {

constexpr unsigned kTmaSpinLimit = 1u << 24;   // polls of one wait (each may suspend briefly)

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make the initialised barriers visible to the asynchronous (TMA) proxy
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this thread's earlier generic-proxy accesses of shared memory before
// its later asynchronous-proxy (TMA) writes there
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase with the given parity; false (and *err set) on timeout
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, unsigned* err) {
    for (unsigned n = 0; n < kTmaSpinLimit; ++n)
        if (mbar_try_wait(bar, parity)) return true;
    if (err) atomicOr(err, 1u);
    return false;
}

// 3D tiled tensor copy of the map's box at element coordinates (x, y, z)
// into shared memory, completing `bytes` of the barrier's transaction count
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
// contiguous bulk copy (both addresses 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Host: encode a 3D tiled tensor map over an array of `es`-byte elements
// (FP32 or FP64) with extents dims[3] (innermost first), byte strides of
// dims 1 and 2, and a box of box[3] elements; out-of-range elements read as
// zero.  Returns false (nothing encoded) when the driver entry point is
// missing or the arguments break its rules (base / strides 16-byte aligned,
// box inner extent a multiple of 16 bytes, box dims <= 256).
bool encode_tensor_map_3d(CUtensorMap* map, const void* base, int es, const uint64_t dims[3],
                          const uint64_t strides_bytes[2], const uint32_t box[3]);

}  // namespace hfav
