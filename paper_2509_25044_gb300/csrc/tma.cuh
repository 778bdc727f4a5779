// tma.cuh -- Tensor Memory Accelerator helpers for sm_103a, as inline PTX:
// tiled 4-D tensor loads and plain bulk copies from global memory into
// shared memory, completed on an mbarrier through its transaction count, and
// the host-side construction of a tiled tensor map (through the driver entry
// point, so the library does not link the driver library directly).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "umma.cuh"

namespace regk {
namespace tma {

// the mbarrier's pending phase completes after this arrival and `bytes` of
// asynchronous copies
__device__ __forceinline__ void expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(umma::smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

// box of a 4-D tiled tensor map at coordinates (c0 innermost .. c3) -> shared
// memory; out-of-range elements read as zero.  c0 * element size must be a
// multiple of 16 bytes; the other coordinates may be negative.
__device__ __forceinline__ void load_4d(void *smem_dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                        uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(umma::smem_addr(smem_dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(umma::smem_addr(mbar))
        : "memory");
}

// box of a 3-D tiled tensor map at (c0 innermost, c1, c2) -> shared memory,
// same rules as load_4d
__device__ __forceinline__ void load_3d(void *smem_dst, const CUtensorMap *map, int c0, int c1, int c2,
                                        uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(umma::smem_addr(smem_dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(umma::smem_addr(mbar))
        : "memory");
}

// contiguous bytes global -> shared (both 16-byte aligned, bytes % 16 == 0)
__device__ __forceinline__ void load_bulk(void *smem_dst, const void *src, uint32_t bytes, uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            umma::smem_addr(smem_dst)),
        "l"((uint64_t)src), "r"(bytes), "r"(umma::smem_addr(mbar))
        : "memory");
}

// Host: a 4-D tiled tensor map over a BF16 array with dims[0] innermost
// (dims[0] * 2 bytes a multiple of 16) and the given box.  Returns false if
// the driver entry point is missing or rejects the description.
bool make_map_bf16_4d(CUtensorMap *map, const void *base, const uint64_t dims[4], const uint32_t box[4]);

// Host: a tiled tensor map of rank 3 or 4 over a dense FP32 (dt = REG_F32) or
// BF16 (REG_BF16) array, dims[0] innermost, no swizzle, zero fill outside the
// array.  Every stride (dims[0] * element size, ...) must be a multiple of 16
// bytes and box[0] * element size a multiple of 16.  Returns false if the
// driver entry point is missing or rejects the description.
bool make_map(CUtensorMap *map, const void *base, int dt, int rank, const uint64_t *dims, const uint32_t *box);

}  // namespace tma
}  // namespace regk
