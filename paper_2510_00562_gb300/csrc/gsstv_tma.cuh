// Tensor-memory-accelerator (TMA) helpers: host-side tensor-map encoding and
// the device-side PTX for bulk tensor loads completed through mbarriers.
//
// Every wait on an mbarrier is bounded: after kMbarSpinLimit failed polls the
// caller gets `false` and is expected to flag a timeout, drain its own loads
// (again bounded) and return, so that no kernel of this library can hang the
// device.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gsstv {

constexpr unsigned kMbarSpinLimit = 1u << 24;

// ---------------------------------------------------------------------------
// device side
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// makes the initialised barriers visible to the async (TMA) proxy
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
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

// Bounded wait for phase `parity` of `bar` to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    for (unsigned k = 0; k < kMbarSpinLimit; ++k)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (TMA) writes to the same shared memory
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Brings a tensor map held in global memory into the TMA unit's descriptor
// cache ahead of its first use.
__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// 3-D tiled bulk tensor load global -> shared, completion counted on `bar`.
// The innermost coordinate x must be a multiple of 16 bytes / element size;
// other coordinates may be negative or beyond the tensor (zero fill).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// Encodes a 3-D tiled map over `ncubes` stacked pitched cubes of `elem_bytes`
// elements: dims (n2, n1, n3 * ncubes), row pitch p2 elements, box
// (box_x, box_y, 1), zero fill outside.  Returns 0 on success.
int tma_encode_cubes(CUtensorMap* map, const void* base, int elem_bytes, int n1, int n2, int n3,
                     int p2, int ncubes, int box_x, int box_y);

}  // namespace gsstv
