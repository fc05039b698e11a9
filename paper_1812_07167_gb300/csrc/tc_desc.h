// Encodings of the sm_100-family (tcgen05) tensor-core operand descriptors,
// written from the field tables of NVIDIA's public PTX ISA documentation
// (sections "Shared memory descriptor" and "Instruction descriptor" of the
// tcgen05 chapter).  Host and device code share them; a host test decodes
// every field again from these numbers.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define TC_HD __host__ __device__
#else
#define TC_HD
#endif

namespace hps {
namespace tc {

// Shared-memory matrix descriptor (64 bits):
//   bits  0-13  start address >> 4
//   bits 16-29  leading-dimension byte offset >> 4 (unused for K-major
//               operands in a swizzled layout whose K step fits one atom)
//   bits 32-45  stride-dimension byte offset >> 4: distance between
//               consecutive groups of 8 rows (M or N)
//   bits 46-48  fixed constant 0b001
//   bits 49-51  matrix base offset (0: atoms aligned to their repeat)
//   bit  52     leading-dimension stride mode (0: relative byte offset)
//   bits 61-63  swizzle: 0 none, 1 128-byte with 32-byte atoms, 2 128-byte,
//               4 64-byte, 6 32-byte
// This is the K-major operand with 128-byte swizzling: rows of 64 bf16
// (128 bytes), 8-row atoms of 1024 bytes stored back to back, the layout a
// TMA copy with CU_TENSOR_MAP_SWIZZLE_128B and a 128-byte inner box writes.
TC_HD constexpr uint64_t smem_desc_sw128_kmajor(uint32_t smem_addr) {
  return (uint64_t)((smem_addr & 0x3FFFFu) >> 4) |  // start address
         ((uint64_t)1u << 16) |                      // LBO (unused here)
         ((uint64_t)(1024u >> 4) << 32) |            // SBO = 8 rows x 128 B
         ((uint64_t)1u << 46) |                      // fixed 0b001
         ((uint64_t)2u << 61);                       // 128-byte swizzle
}

// Instruction descriptor of tcgen05.mma .kind::f16 (32 bits):
//   bits  0-1  sparsity selector (0)      bit 2  sparsity (0 = dense)
//   bit   3    saturate (0)               bits 4-5  D type: 0 f16, 1 f32
//   bits  7-9  A type: 0 f16, 1 bf16      bits 10-12  B type: 0 f16, 1 bf16
//   bit  13    negate A                   bit 14  negate B
//   bit  15    A major-ness (0 = K-major) bit 16  B major-ness (0 = K-major)
//   bits 17-22 N >> 3                     bits 24-28  M >> 4
//   bits 30-31 maximum shift (.ws only; 0)
TC_HD constexpr uint32_t idesc_bf16_f32(int M, int N, bool negate_a) {
  return (1u << 4) |                           // D: f32
         (1u << 7) |                           // A: bf16
         (1u << 10) |                          // B: bf16
         ((negate_a ? 1u : 0u) << 13) |        // -A
         ((uint32_t)(N >> 3) << 17) |          // N
         ((uint32_t)(M >> 4) << 24);           // M
}

}  // namespace tc
}  // namespace hps
