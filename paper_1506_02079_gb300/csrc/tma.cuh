// Tensor-memory-accelerator (TMA) plumbing: host-side encoding of 2-D tiled tensor maps and
// device-side inline PTX for bulk tensor loads completed on shared-memory mbarriers.
//
// Every wait on an mbarrier is bounded: after kWaitLimit polls the caller gets `false`,
// records an error flag for the host, and must not touch the slot's data.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace emfuse {

// ---------------------------------------------------------------- host
// 2-D tensor map over a row-pitched array: `nx` x `ny` elements of `elem_bytes` (4 or 8),
// row pitch `pitch` elements (a multiple of 16 bytes), base 16-byte aligned, boxes of
// box_x x box_y elements; out-of-range elements read as zero.
int encode_tensor_map_2d(CUtensorMap* out, const void* base, int elem_bytes, int64_t nx, int64_t ny,
                         int64_t pitch, int box_x, int box_y);
// 3-D tensor map over a stack of nz planes of ny rows (row pitch `pitch` elements), element
// type uint8 (elem_bytes 1) or float32 (4); boxes of box_x x box_y x 1.
int encode_tensor_map_3d(CUtensorMap* out, const void* base, int elem_bytes, int64_t nx, int64_t ny,
                         int64_t nz, int64_t pitch, int box_x, int box_y);

// ---------------------------------------------------------------- device
constexpr int kWaitLimit = 1 << 20;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Make initialised barriers visible to the async (TMA) proxy.
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Order this thread's earlier generic-proxy accesses of shared memory before later
// async-proxy (TMA) writes to it.
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Warp-uniform bounded wait for phase `parity` of barrier `bar`.
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < kWaitLimit; ++it)
        if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
    return false;
}

// 2-D tiled bulk tensor load of the box at element coordinates (x, y) into shared memory,
// completing `bytes` of transaction count on `bar`.  x * element size must be a multiple of
// 16 bytes; coordinates may lie outside the tensor (zero fill).
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Explicit shared-memory vector loads (a generic pointer into the ring would otherwise be
// compiled to generic loads).
__device__ __forceinline__ void lds4(uint32_t addr, float (&v)[4]) {
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                 : "r"(addr));
}
__device__ __forceinline__ void lds4(uint32_t addr, double (&v)[4]) {
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v[0]), "=d"(v[1]) : "r"(addr));
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v[2]), "=d"(v[3]) : "r"(addr + 16));
}
__device__ __forceinline__ void lds2(uint32_t addr, float& a, float& b) {
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(a), "=f"(b) : "r"(addr));
}
__device__ __forceinline__ void lds2(uint32_t addr, double& a, double& b) {
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(a), "=d"(b) : "r"(addr));
}
__device__ __forceinline__ float lds1(uint32_t addr, float) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ double lds1(uint32_t addr, double) {
    double v;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(addr));
    return v;
}

}  // namespace emfuse
