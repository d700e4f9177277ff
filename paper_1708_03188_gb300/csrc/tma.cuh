// tma.cuh - tensor-memory-accelerator (TMA) building blocks of the streaming transform kernels:
// tiled tensor loads (cp.async.bulk.tensor) completing on an mbarrier, 1-D bulk loads, and the
// host-side encoding of a tensor map through the driver entry point (no link against the
// driver library is needed: the runtime hands out the function pointer).
//
// Every copy here reads this GPU's own memory into this CTA's shared memory (no multicast).
// A tiled load may start at any coordinate along the outer dimensions; the innermost
// coordinate (in elements) times the element size is kept a multiple of 16 bytes by the
// callers (tile starts are multiples of 16 complex values).  Out-of-range parts of a box read
// as zero.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "tc.cuh"

namespace sgm {
namespace tma {

// 2-D tiled load: box at (c0 innermost, c1) into dst, completion counted on bar
__device__ __forceinline__ void load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          tc::smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(tc::smem_addr(bar))
      : "memory");
}

// 3-D tiled load: box at (c0 innermost, c1, c2)
__device__ __forceinline__ void load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(tc::smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(tc::smem_addr(bar))
      : "memory");
}

// prefetch the tensor map descriptor into the constant cache
__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

}  // namespace tma

// Host: encode a tiled tensor map (row-major, no swizzle, no interleave, zero fill).
//   dims[0] innermost (elements), strides[i] = byte stride of dims[i + 1], box[i] elements.
// Returns cudaSuccess or the error of the entry-point lookup / an invalid-value error when the
// driver rejects the description.
cudaError_t encode_tiled_map(CUtensorMap* map, CUtensorMapDataType dtype, int rank, const void* base,
                             const uint64_t* dims, const uint64_t* strides, const uint32_t* box);

}  // namespace sgm
