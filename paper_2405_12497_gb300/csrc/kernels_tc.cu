// kernels_tc.cu -- tensor-core (tcgen05) query rotation P^{-1}[q_r; 0] in
// BF16 or TF32 with FP32 accumulation (the precision modes of the query
// rotation of §3.3; the FP32 canonical path lives in kernels_gemm.cu).
//
// C[M x N] = A[M x K] * B[N x K]^T with A = the raw queries (FP32 in global
// memory, rounded to BF16/TF32 while staged), B = P^T rows (one per output
// coordinate, K-major, stored pre-rounded in the index). One CTA = 4 warps,
// a 128-row M tile and an N tile of up to 256 columns accumulated in TMEM;
// K advances in stages of 128 bytes per row (64 BF16 or 32 TF32 elements)
// staged in shared memory in the canonical no-swizzle core-matrix layout
// (8 rows x 16 bytes per core matrix). One thread issues the MMAs and
// commits them to an mbarrier; every wait is bounded and reports a timeout
// through the error word instead of hanging.
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"
#include "tc_util.cuh"

namespace rbq {
namespace {

constexpr int kTcThreads = 128;
constexpr int kTcM = 128;           // rows per CTA (one per TMEM lane)
constexpr int kStageBytes = 128;    // bytes per row per K stage

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// MODE 0: BF16 operands (kind::f16); MODE 1: TF32 operands (kind::tf32).
template <int MODE>
__global__ void __launch_bounds__(kTcThreads) rotate_tc_kernel(const float* __restrict__ Q,
                                                               int64_t M, int K,
                                                               const void* __restrict__ Bg,
                                                               int Kp, int N, int NT,
                                                               float* __restrict__ C, int* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint32_t s_taddr;
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ int s_fail;
  uint8_t* sA = smem;                      // kTcM rows x 128 B
  uint8_t* sB = smem + kTcM * kStageBytes; // NT rows x 128 B
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t m0 = (int64_t)blockIdx.x * kTcM;
  const int n0 = blockIdx.y * NT;
  const int ncols = NT <= 32 ? 32 : (NT <= 64 ? 64 : (NT <= 128 ? 128 : 256));
  constexpr int esize = MODE == 0 ? 2 : 4;
  constexpr int kEl = kStageBytes / esize;  // elements per row per stage
  constexpr int kInstr = MODE == 0 ? 16 : 8; // K per MMA instruction

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_taddr)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&s_bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = s_taddr;
  const uint32_t bar = smem_u32(&s_bar);
  const uint32_t idesc = make_idesc(MODE == 0 ? 1u : 2u, kTcM, NT);
  const uint32_t lboA = (kTcM / 8) * 128, lboB = (NT / 8) * 128;
  uint32_t phase = 0;
  bool ok = true;

  for (int k0 = 0; k0 < K && ok; k0 += kEl) {
    // stage A: 128 rows x kEl elements, rounded to the operand type
    for (int u = tid; u < kTcM * 8; u += kTcThreads) {
      const int r = u >> 3, c = u & 7;
      const int64_t gm = m0 + r;
      const int kb = k0 + c * (16 / esize);
      uint4 pk;
      if (MODE == 0) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e)
          v[e] = (gm < M && kb + e < K) ? __ldg(Q + gm * K + kb + e) : 0.0f;
        __nv_bfloat162 h0 = __floats2bfloat162_rn(v[0], v[1]);
        __nv_bfloat162 h1 = __floats2bfloat162_rn(v[2], v[3]);
        __nv_bfloat162 h2 = __floats2bfloat162_rn(v[4], v[5]);
        __nv_bfloat162 h3 = __floats2bfloat162_rn(v[6], v[7]);
        pk.x = *reinterpret_cast<uint32_t*>(&h0);
        pk.y = *reinterpret_cast<uint32_t*>(&h1);
        pk.z = *reinterpret_cast<uint32_t*>(&h2);
        pk.w = *reinterpret_cast<uint32_t*>(&h3);
      } else {
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
          v[e] = (gm < M && kb + e < K) ? to_tf32(__ldg(Q + gm * K + kb + e)) : 0.0f;
        pk = make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]),
                        __float_as_uint(v[3]));
      }
      *reinterpret_cast<uint4*>(sA + core_off(r, c, kTcM)) = pk;
    }
    // stage B: NT rows of P^T (already in the operand type, K padded to Kp)
    const uint8_t* Bb = static_cast<const uint8_t*>(Bg);
    for (int u = tid; u < NT * 8; u += kTcThreads) {
      const int r = u >> 3, c = u & 7;
      const int gn = n0 + r;
      uint4 pk = make_uint4(0, 0, 0, 0);
      if (gn < N) pk = __ldg(reinterpret_cast<const uint4*>(Bb + ((int64_t)gn * Kp + k0) * esize) + c);
      *reinterpret_cast<uint4*>(sB + core_off(r, c, NT)) = pk;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
      for (int s = 0; s < kEl / kInstr; ++s) {
        const uint32_t chunk = (uint32_t)(s * (kInstr * esize / 16));
        const uint64_t da = make_desc(a0 + chunk * lboA, lboA, 128);
        const uint64_t db = make_desc(b0 + chunk * lboB, lboB, 128);
        const uint32_t acc = (k0 > 0 || s > 0) ? 1u : 0u;
        if (MODE == 0)
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(taddr),
              "l"(da), "l"(db), "r"(idesc), "r"(acc));
        else
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(taddr),
              "l"(da), "l"(db), "r"(idesc), "r"(acc));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
          : "memory");
    }
    if (!mbar_wait(bar, phase)) {  // the MMAs did not complete in time
      s_fail = 1;
      ok = false;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    ok = ok && !s_fail;
  }
  // epilogue: warp w reads TMEM lanes 32w..32w+31 (= tile rows)
  if (ok) {
    const int64_t row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < NT; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (row < M) {
        const int gb = n0 + c0;
        if (gb + 16 <= N && (N & 3) == 0) {  // whole chunk: four 16-byte stores
          float4* dst = reinterpret_cast<float4*>(C + row * N + gb);
#pragma unroll
          for (int v = 0; v < 4; ++v)
            dst[v] = make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]),
                                 __uint_as_float(r[4 * v + 2]), __uint_as_float(r[4 * v + 3]));
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int gn = gb + e;
            if (gn < N) C[row * N + gn] = __uint_as_float(r[e]);
          }
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 2);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// P^T rounded to the operand type, K-major, K padded to a multiple of 64.
__global__ void pack_pt_kernel(const float* __restrict__ P32, int d, int dpad, int Kp,
                               __nv_bfloat16* __restrict__ ptb, float* __restrict__ ptf) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)dpad * Kp) return;
  const int n = (int)(i / Kp), k = (int)(i % Kp);
  const float v = (k < d) ? P32[(int64_t)k * dpad + n] : 0.0f;
  ptb[i] = __float2bfloat16_rn(v);
  ptf[i] = to_tf32(v);
}

// Centroid rows rounded to TF32 (K-major, zero-padded to Kp), and the FP32
// norms ||c||^2 (ascending fold) and ||c|| that scale the probe filter's
// error bound. One thread per (centroid, column); column 0 also folds the
// norm.
__global__ void pack_centroids_kernel(const float* __restrict__ C, int K, int d, int Kp,
                                      float* __restrict__ ctf, float* __restrict__ cn2,
                                      float* __restrict__ cnorm) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)K * Kp) return;
  const int c = (int)(i / Kp), k = (int)(i % Kp);
  const float* row = C + (int64_t)c * d;
  ctf[i] = (k < d) ? to_tf32(row[k]) : 0.0f;
  if (k == 0) {
    float s2 = 0.0f;
    for (int t = 0; t < d; ++t) s2 = __fmaf_rn(row[t], row[t], s2);
    cn2[c] = s2;
    cnorm[c] = __fsqrt_rn(s2);
  }
}

}  // namespace

int pack_centroids(rabitq_index* X, cudaStream_t s) {
  const int64_t total = (int64_t)X->K * X->kp;
  pack_centroids_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
      X->centroids, X->K, X->d, X->kp, X->ctf, X->cn2, X->cnorm);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

int centroid_dot_tc(const rabitq_index* X, const float* Q, int64_t M, float* out, int* err,
                    cudaStream_t s) {
  if (M <= 0) return RABITQ_OK;
  const int N = X->K;
  const int NT = 256;
  const int ntiles = (N + NT - 1) / NT;
  const size_t smem = 100 * 1024;  // at most two CTAs (256 TMEM columns each) per SM
  dim3 grid((unsigned)((M + kTcM - 1) / kTcM), (unsigned)ntiles);
  RBQ_CUDA(cudaFuncSetAttribute(rotate_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  rotate_tc_kernel<1><<<grid, kTcThreads, smem, s>>>(Q, M, X->d, X->ctf, X->kp, N, NT, out, err);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

int pack_pt(rabitq_index* X, cudaStream_t s) {
  const int64_t total = (int64_t)X->dpad * X->kp;
  pack_pt_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(X->P32, X->d, X->dpad, X->kp,
                                                                 reinterpret_cast<__nv_bfloat16*>(X->ptb),
                                                                 X->ptf);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

int rotate_tc(const rabitq_index* X, const float* Q, int64_t M, int mode, float* out, int* err,
              cudaStream_t s) {
  if (M <= 0) return RABITQ_OK;
  const int N = X->dpad;
  const int NT = N >= 256 ? 256 : N;  // N is a multiple of 64
  const int ntiles = (N + NT - 1) / NT;
  // request enough shared memory that at most two CTAs share an SM, so the
  // TMEM they allocate (<= 256 columns each) always fits the SM's 512
  const size_t smem = 100 * 1024;
  dim3 grid((unsigned)((M + kTcM - 1) / kTcM), (unsigned)ntiles);
  if (mode == RABITQ_ROT_BF16) {
    RBQ_CUDA(cudaFuncSetAttribute(rotate_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    rotate_tc_kernel<0><<<grid, kTcThreads, smem, s>>>(Q, M, X->d, X->ptb, X->kp, N, NT, out, err);
  } else {
    RBQ_CUDA(cudaFuncSetAttribute(rotate_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    rotate_tc_kernel<1><<<grid, kTcThreads, smem, s>>>(Q, M, X->d, X->ptf, X->kp, N, NT, out, err);
  }
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

}  // namespace rbq
