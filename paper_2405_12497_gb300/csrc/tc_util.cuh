// tc_util.cuh -- small tcgen05 helpers (sm_103a): shared-memory matrix and
// instruction descriptors, the canonical no-swizzle core-matrix layout, and a
// bounded mbarrier wait.
#pragma once

#include <stdint.h>

namespace rbq {

constexpr uint32_t kWaitLimit = 1u << 26;  // try_wait polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K)
// byte offset, stride (M/N) byte offset, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3fff) | ((uint64_t)((lbo >> 4) & 0x3fff) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3fff) << 32) | (1ull << 46);
}

// Instruction descriptor: FP32 accumulator, A/B format (1 = BF16 for
// kind::f16, 2 = TF32 for kind::tf32), both K-major, N >> 3, M >> 4.
__device__ __forceinline__ uint32_t make_idesc(uint32_t fmt, int m, int n) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

// Offset of (row r, 16-byte chunk c) in a staged tile of R rows: core
// matrices are 128 contiguous bytes; consecutive 8-row groups are 128 bytes
// apart (SBO), consecutive chunks along K are R/8 * 128 bytes apart (LBO).
__device__ __forceinline__ uint32_t core_off(int r, int c, int R) {
  return (uint32_t)((c * (R >> 3) + (r >> 3)) * 128 + (r & 7) * 16);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          uint32_t limit = kWaitLimit) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

}  // namespace rbq
