// lp_tcgen05.h -- encoders of the two descriptors that tcgen05.mma takes,
// usable on the host (tests) and on the device.  Field layouts as given in the
// PTX ISA for sm_100-family tensor cores:
//
// Shared-memory matrix descriptor (64 bits):
//   bits  0..13  matrix start address >> 4 (shared-memory byte address)
//   bits 16..29  leading-dimension byte offset >> 4
//   bits 32..45  stride-dimension byte offset >> 4
//   bits 46..48  fixed constant 0b001
//   bits 49..51  matrix base offset (0: the swizzle pattern starts at the
//                1024-byte aligned address the tiles are placed at)
//   bit  52      leading-dimension stride mode (0: relative byte offset)
//   bits 61..63  swizzling mode: 0 none, 1 128-byte with 32-byte atoms,
//                2 128-byte, 4 64-byte, 6 32-byte
//
// Instruction descriptor of .kind::f16 (32 bits):
//   bits  0..1   sparsity selector (0), bit 2 sparsity (0: dense),
//   bit   3      saturate (0)
//   bits  4..5   D format: 0 F16, 1 F32
//   bits  7..9   A format: 0 F16, 1 BF16
//   bits 10..12  B format: 0 F16, 1 BF16
//   bits 13, 14  negate A, negate B
//   bits 15, 16  A major, B major: 0 = K-major
//   bits 17..22  N >> 3
//   bits 24..28  M >> 4
//   bits 30..31  maximum shift (weight-stationary only; 0)
#pragma once

#include <cstdint>

namespace lpb {
namespace tc {

enum SmemSwizzle : uint32_t { kSwizzleNone = 0, kSwizzle128B = 2, kSwizzle64B = 4, kSwizzle32B = 6 };

__host__ __device__ constexpr uint64_t smem_desc(uint32_t start_addr, uint32_t lbo_bytes, uint32_t sbo_bytes,
                                                 uint32_t swizzle) {
    return (uint64_t)((start_addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46) | ((uint64_t)(swizzle & 7u) << 61);
}

// BF16 A and B, both K-major, FP32 accumulator, dense, M x N per instruction
// (K = 16 per instruction for 16-bit inputs).
__host__ __device__ constexpr uint32_t idesc_bf16_f32(uint32_t M, uint32_t N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// Shapes valid for cta_group::1 kind::f16 with M = 128: N a multiple of 16 in [16, 256].
__host__ __device__ constexpr bool valid_m128_n(uint32_t N) { return N >= 16 && N <= 256 && N % 16 == 0; }

}  // namespace tc
}  // namespace lpb
