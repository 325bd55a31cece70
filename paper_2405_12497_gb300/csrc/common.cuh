// common.cuh -- device helpers shared by the library's kernels (sm_103a).
//
// Numerics contract (identical results on every launch shape):
//   canonical FP32 dot        s = 0; for i ascending: s = fma(a_i, b_i, s)
//   canonical FP32 sq. dist.  s = 0; for i ascending: t = a_i - b_i; s = fma(t, t, s)
//   every other FP32/FP64 step is one IEEE round-to-nearest operation, written
//   with the __f*_rn / __d*_rn intrinsics so the compiler never contracts or
//   reorders it.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rbq {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;

// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw, SC'11):
// ten rounds of two 32x32->64 multiplies; the key is bumped by the Weyl
// constants between rounds. Counter words (c0, c1, c2, c3), key = seed.
struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                                            uint32_t c3) {
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return U4{c0, c1, c2, c3};
}

// Stream tags (fourth counter word) of the library's random draws.
enum : uint32_t { kTagKmeansInit = 1, kTagGauss = 2, kTagQuant = 3, kTagSample = 4 };

// Total order of floats as unsigned keys (negatives below positives).
__device__ __forceinline__ uint32_t float_key(float f) {
  uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// The probe filter's error bound eps_c of a centroid's approximate score
// (derived where probe_select_kernel is defined).
// eps_c as a quadratic in ||c|| with per-query coefficients: squared
// distances 1.05 [2a ||q|| ||c|| + b (||q|| + ||c||)^2], b = (2d + 8) 2^-23,
// = ||c|| (kb ||c|| + ka) + kg; inner products 1.05 (a + (d + 8) 2^-22)
// ||q|| ||c||. (Evaluated in FP32: a few units of rounding, inside the 5%.)
struct ProbeEps {
  float ka, kb, kg;
  __device__ __forceinline__ ProbeEps(int ip_metric, float nq, int d) {
    const float a = 0x1.0p-10f + (float)(d + 2) * 0x1.0p-21f;
    if (ip_metric) {
      ka = 1.05f * (a + (float)(d + 8) * 0x1.0p-22f) * nq;
      kb = 0.0f;
      kg = 0.0f;
    } else {
      const float b = (float)(2 * d + 8) * 0x1.0p-23f;
      ka = 1.05f * (2.0f * a + 2.0f * b) * nq;
      kb = 1.05f * b;
      kg = 1.05f * b * nq * nq;
    }
  }
  __device__ __forceinline__ float operator()(float nc) const {
    return __fmaf_rn(nc, __fmaf_rn(kb, nc, ka), kg);
  }
};

// Ascending bitonic sort of n (power of two) 64-bit keys in shared memory by
// the whole block. Caller synchronizes before; returns synchronized.
__device__ __forceinline__ void block_bitonic_sort_u64(unsigned long long* a, int n) {
  for (int size = 2; size <= n; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < (n >> 1); t += blockDim.x) {
        const int lo = 2 * t - (t & (stride - 1));
        const int hi = lo + stride;
        const bool up = ((lo & size) == 0);
        const unsigned long long x = a[lo], y = a[hi];
        if ((x > y) == up) {
          a[lo] = y;
          a[hi] = x;
        }
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ void block_bitonic_sort_u32(uint32_t* a, int n) {
  for (int size = 2; size <= n; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < (n >> 1); t += blockDim.x) {
        const int lo = 2 * t - (t & (stride - 1));
        const int hi = lo + stride;
        const bool up = ((lo & size) == 0);
        const uint32_t x = a[lo], y = a[hi];
        if ((x > y) == up) {
          a[lo] = y;
          a[hi] = x;
        }
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

__device__ __forceinline__ float warp_min_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

}  // namespace rbq
