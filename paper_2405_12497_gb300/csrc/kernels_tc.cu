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
//
// The probe scores of all K centroids (§4's probe, made exact by the bound
// in probe_select) run in probe_dot_kernel: both operands are stored
// pre-tiled in the core-matrix layout (the centroids in the index, the
// queries by query_prep_kernel per search), so that every K stage of a
// 128 x 256 output tile is two contiguous bulk copies. One producer warp
// fills a ring of stages, one thread issues the MMAs into one of two TMEM
// accumulators, and two groups of eight warps turn the accumulators'
// products into the filter's upper-bound keys.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tc_util.cuh"

namespace rbq {
namespace {

constexpr int kTcThreads = 128;
constexpr int kTcM = 128;           // rows per CTA (one per TMEM lane)
constexpr int kStageBytes = 128;    // bytes per row per K stage

inline __host__ __device__ size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

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

// ---- probe scores (products and the filter's keys)
constexpr int kPdM = 128;                        // queries per tile (TMEM lanes)
constexpr int kPdN = 256;                        // centroids per tile (TMEM columns)
constexpr int kPdStages = 3;                     // ring of K stages
constexpr int kPdA = kPdM * kStageBytes;         // 16 KB: one A stage
constexpr int kPdB = kPdN * kStageBytes;         // 32 KB: one B stage
constexpr int kPdEpiG = 8;                       // warps of an epilogue group (one accumulator)
constexpr int kPdEpi = 2 * kPdEpiG;              // epilogue warps: two groups
constexpr int kPdThreads = (kPdEpi + 2) * 32;    // then the producer warp and the MMA warp
constexpr int kPdCols = kPdN / 2;                // columns per epilogue warp
constexpr size_t kPdSmem = (size_t)kPdStages * (kPdA + kPdB);
constexpr int kPdEl = kStageBytes / 4;           // TF32 elements per row per stage

// Offset (floats) of element (row r, column k) of a matrix stored pre-tiled:
// tiles of R rows, each a run of K stages of R rows x 32 TF32 in the
// core-matrix layout (the shared-memory image of one stage).
__device__ __forceinline__ int64_t tiled_off(int64_t r, int k, int R, int nks) {
  const int64_t tile = r / R;
  const int rr = (int)(r % R), st = k / kPdEl, kk = k % kPdEl;
  return ((tile * nks + st) * (int64_t)(R * kStageBytes) + core_off(rr, kk >> 2, R)) / 4 + (kk & 3);
}

// Centroids rounded to TF32 in tiles of kPdN rows (rows past K and columns
// past d are zero), and the FP32 norms ||c||^2 (ascending fold) and ||c||
// that scale the probe filter's error bound. One thread per element of the
// padded matrix; column 0 also folds the norm.
__global__ void pack_centroids_kernel(const float* __restrict__ C, int K, int d, int Kp,
                                      int64_t rows, float* __restrict__ ctf,
                                      float* __restrict__ cn2, float* __restrict__ cnorm) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= rows * Kp) return;
  const int64_t c = i / Kp;
  const int k = (int)(i % Kp);
  const float* row = C + c * d;
  ctf[tiled_off(c, k, kPdN, Kp / kPdEl)] = (c < K && k < d) ? to_tf32(row[k]) : 0.0f;
  if (k == 0 && c < K) {
    float s2 = 0.0f;
    for (int t = 0; t < d; ++t) s2 = __fmaf_rn(row[t], row[t], s2);
    cn2[c] = s2;
    cnorm[c] = __fsqrt_rn(s2);
  }
}

// max_c ||c|| (one block).
__global__ void max_norm_kernel(const float* __restrict__ cnorm, int K, float* __restrict__ out) {
  __shared__ float wmax[32];
  float m = 0.0f;
  for (int c = threadIdx.x; c < K; c += blockDim.x) m = fmaxf(m, cnorm[c]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wmax[w]);
    *out = m;
  }
}

// One warp per query row (rows past M: zeros): the row rounded to TF32 in
// tiles of kPdM rows, its FP32 ||q||^2 (lane-strided partial folds, then a
// fixed butterfly; the bound needs an FP32 value of the norm, not the
// canonical fold) and the initial range of its keys.
__global__ void query_prep_kernel(const float* __restrict__ Q, int64_t M, int d, int Kp,
                                  int64_t rows, float* __restrict__ qt, float* __restrict__ nq2,
                                  uint32_t* __restrict__ kmin, uint32_t* __restrict__ kmax) {
  const int64_t m = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (m >= rows) return;
  const int nks = Kp / kPdEl;
  float part = 0.0f;
  for (int k = lane; k < Kp; k += 32) {
    const float v = (m < M && k < d) ? __ldg(Q + m * d + k) : 0.0f;
    part = __fmaf_rn(v, v, part);
    qt[tiled_off(m, k, kPdM, nks)] = to_tf32(v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part = __fadd_rn(part, __shfl_xor_sync(0xffffffffu, part, o));
  if (lane == 0 && m < M) {
    nq2[m] = part;
    kmin[m] = 0xffffffffu;
    kmax[m] = 0u;
  }
}

// Bounded wait that also gives up once another role of the CTA has failed.
__device__ __forceinline__ bool pd_wait(uint32_t bar, uint32_t parity, volatile int* fail,
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
    if ((it & 255) == 255 && *fail) return false;
  }
  return false;
}

// The products Qt Ct^T (M x N) over tiles (m, n), m-major, turned into the
// probe filter's keys: keys[m][c] = key of U_c, each row's key range in
// kmin / kmax (atomics), and per row and 128 columns the kProbePool smallest
// entries (key rounded up to a multiple of 128 | column index in the 128,
// ascending) in pool. CTA b takes the items [b items / G, (b + 1) items / G).
// Stage it of the CTA's sequence lives in ring slot it % kPdStages; tile j of
// the CTA accumulates in TMEM columns (j & 1) * kPdN and is drained by
// epilogue group j & 1. Barriers: full (copies landed), empty (the MMAs
// reading the slot are done), tfull (a tile's accumulator is complete),
// tempty (its epilogue group has read it). A wait that expires sets
// *err = 2; the roles then stop, wait (bounded) for their own copies or
// MMAs in flight, and the CTA frees its TMEM.
__global__ void __launch_bounds__(kPdThreads, 1) probe_dot_kernel(
    const float* __restrict__ qt, const float* __restrict__ ct, int64_t M, int N, int nks,
    int ntn, int64_t items, int d, int metric, const float* __restrict__ nq2,
    const float* __restrict__ cn2, const float* __restrict__ cnorm, uint32_t* __restrict__ keys,
    uint32_t* __restrict__ kmin, uint32_t* __restrict__ kmax, uint32_t* __restrict__ pool,
    int* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint32_t s_taddr;
  __shared__ __align__(8) uint64_t s_full[kPdStages], s_empty[kPdStages], s_tfull[2], s_tempty[2];
  __shared__ volatile int s_fail;
  __shared__ __align__(16) float s_cn2[2][kPdN];  // each group's tile's centroid norms
  __shared__ __align__(16) float s_cnorm[2][kPdN];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t G = gridDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * items / G, i1 = ((int64_t)blockIdx.x + 1) * items / G;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_taddr)),
                 "r"(2 * kPdN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < kPdStages; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&s_full[i])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&s_empty[i])), "r"(1));
    }
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&s_tfull[i])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&s_tempty[i])),
                   "r"(kPdEpiG * 32));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = s_taddr;
  const uint32_t sbase = smem_u32(smem);
  auto slot_a = [&](uint32_t slot) { return sbase + slot * (uint32_t)(kPdA + kPdB); };
  auto slot_b = [&](uint32_t slot) { return sbase + slot * (uint32_t)(kPdA + kPdB) + (uint32_t)kPdA; };

  if (warp == kPdEpi) {  // producer: one lane issues every stage's two bulk copies
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t i = i0; i < i1 && ok; ++i) {
        const int64_t mt = i / ntn;
        const int nt = (int)(i % ntn);
        const uint8_t* a_src = reinterpret_cast<const uint8_t*>(qt) + mt * nks * (int64_t)kPdA;
        const uint8_t* b_src = reinterpret_cast<const uint8_t*>(ct) + (int64_t)nt * nks * kPdB;
        for (int ks = 0; ks < nks; ++ks, ++it) {
          const uint32_t slot = it % kPdStages;
          if (it >= (uint32_t)kPdStages &&
              !pd_wait(smem_u32(&s_empty[slot]), ((it / kPdStages) - 1) & 1u, &s_fail)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&s_full[slot]);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                       "r"((uint32_t)(kPdA + kPdB))
                       : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
              ::"r"(slot_a(slot)), "l"(a_src + (int64_t)ks * kPdA), "r"((uint32_t)kPdA), "r"(fb)
              : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
              ::"r"(slot_b(slot)), "l"(b_src + (int64_t)ks * kPdB), "r"((uint32_t)kPdB), "r"(fb)
              : "memory");
        }
      }
      if (!ok) {
        s_fail = 1;
        // the copies already issued land before the CTA exits: stages
        // it - kPdStages .. it - 1 may be in flight
        for (uint32_t j = it > (uint32_t)kPdStages ? it - kPdStages : 0; j < it; ++j)
          mbar_wait(smem_u32(&s_full[j % kPdStages]), (j / kPdStages) & 1u);
      }
    }
  } else if (warp == kPdEpi + 1) {  // MMA issue
    if (lane == 0) {
      const uint32_t idesc = make_idesc(2u, kPdM, kPdN);
      constexpr uint32_t lboA = (kPdM / 8) * 128, lboB = (kPdN / 8) * 128;
      uint32_t it = 0, tc = 0;
      bool ok = true, issued = false;
      for (int64_t i = i0; i < i1 && ok; ++i, ++tc) {
        const uint32_t buf = tc & 1u;
        if (tc >= 2 && !pd_wait(smem_u32(&s_tempty[buf]), ((tc / 2) - 1) & 1u, &s_fail)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t dt = taddr + buf * (uint32_t)kPdN;
        for (int ks = 0; ks < nks; ++ks, ++it) {
          const uint32_t slot = it % kPdStages;
          if (!pd_wait(smem_u32(&s_full[slot]), (it / kPdStages) & 1u, &s_fail)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t a0 = slot_a(slot), b0 = slot_b(slot);
#pragma unroll
          for (int sI = 0; sI < kPdEl / 8; ++sI) {
            const uint64_t da = make_desc(a0 + (uint32_t)(2 * sI) * lboA, lboA, 128);
            const uint64_t db = make_desc(b0 + (uint32_t)(2 * sI) * lboB, lboB, 128);
            const uint32_t acc = (ks > 0 || sI > 0) ? 1u : 0u;
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dt),
                "l"(da), "l"(db), "r"(idesc), "r"(acc));
          }
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  smem_u32(&s_empty[slot]))
              : "memory");
          issued = true;
        }
        if (!ok) break;
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&s_tfull[buf]))
            : "memory");
      }
      if (!ok) {
        s_fail = 1;
        if (issued) {  // the last MMAs issued complete before the CTA exits
          const uint32_t j = it - 1;
          mbar_wait(smem_u32(&s_empty[j % kPdStages]), (j / kPdStages) & 1u);
        }
      }
    }
  } else {
    // epilogue: group g (warps 8g .. 8g + 7) takes the CTA's tiles g, g + 2,
    // ..., which accumulate in TMEM buffer g. Its warp w reads TMEM lanes
    // 32 (w % 4) .. + 31 (tile rows) and the columns [kPdCols ((w / 4) % 2),
    // + kPdCols); the two halves keep their own pool entries. Each half
    // stages its columns' ||c||^2 and ||c|| in shared memory (loaded before
    // the tile's MMAs are waited for).
    const int group = warp / kPdEpiG, quarter = warp & 3, half = (warp >> 2) & 1;
    const int ht = tid & 127;
    const uint32_t bar_id = 1u + 2u * (uint32_t)group + (uint32_t)half;
    float* g_cn2 = s_cn2[group];
    float* g_cnorm = s_cnorm[group];
    for (int64_t i = i0 + group; i < i1; i += 2) {
      const uint32_t tc = (uint32_t)(i - i0);
      const uint32_t buf = tc & 1u;
      const int64_t mt = i / ntn;
      const int nt = (int)(i % ntn);
      const int h0 = nt * kPdN + half * kPdCols;  // first column of this half
      const int cl = min(h0 + ht, N - 1);
      const float ncn2 = __ldg(cn2 + cl), ncnorm = __ldg(cnorm + cl);
      const bool ok = pd_wait(smem_u32(&s_tfull[buf]), (tc / 2) & 1u, &s_fail);
      // one decision for the whole half (a thread that gave up stops all of
      // them); the same barrier finds the half's previous tile read
      uint32_t gave_up;
      asm volatile(
          "{\n.reg .pred p, q;\nsetp.eq.u32 q, %1, 0;\nbar.red.or.pred p, %2, 128, q;\n"
          "selp.u32 %0, 1, 0, p;\n}"
          : "=r"(gave_up)
          : "r"((uint32_t)ok), "r"(bar_id)
          : "memory");
      if (gave_up) {
        s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      g_cn2[half * kPdCols + ht] = ncn2;
      g_cnorm[half * kPdCols + ht] = ncnorm;
      asm volatile("bar.sync %0, 128;" ::"r"(bar_id));
      const int64_t row = mt * kPdM + quarter * 32 + lane;
      const bool live = row < M;
      const float q2 = live ? __ldg(nq2 + row) : 0.0f;
      const ProbeEps eps(metric, __fsqrt_rn(q2), d);
      uint32_t tmin = 0xffffffffu, tmax = 0u;
      // the smallest pool entries of this row and half, ascending: the key
      // rounded up to a multiple of 128, then the centroid's index in the
      // half (7 bits)
      uint32_t top[kProbePool];
#pragma unroll
      for (int j = 0; j < kProbePool; ++j) top[j] = 0xffffffffu;
      const uint32_t src = taddr + ((uint32_t)(quarter * 32) << 16) + buf * (uint32_t)kPdN +
                           (uint32_t)(half * kPdCols);
      for (int c0 = 0; c0 < kPdCols; c0 += 16) {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
              "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(src + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        const int gb = h0 + c0;
        // U_c = approximate score + eps_c as an order-preserving key (the
        // same FP32 operations as the filter's definition)
        uint32_t u[16];
        uint32_t below = 0;  // the chunk's entries under the pool's largest
        const uint32_t thr = top[kProbePool - 1];
        // the chunk's 16 norms as four 16-byte broadcast reads each
        float n2v[16], nnv[16];
#pragma unroll
        for (int v4 = 0; v4 < 4; ++v4) {
          const float4 a = reinterpret_cast<const float4*>(g_cn2 + half * kPdCols + c0)[v4];
          const float4 b = reinterpret_cast<const float4*>(g_cnorm + half * kPdCols + c0)[v4];
          n2v[4 * v4] = a.x; n2v[4 * v4 + 1] = a.y; n2v[4 * v4 + 2] = a.z; n2v[4 * v4 + 3] = a.w;
          nnv[4 * v4] = b.x; nnv[4 * v4 + 1] = b.y; nnv[4 * v4 + 2] = b.z; nnv[4 * v4 + 3] = b.w;
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const float v = __uint_as_float(r[e]);
          const float sc = metric ? -v : __fsub_rn(__fadd_rn(q2, n2v[e]), __fmul_rn(2.0f, v));
          u[e] = float_key(__fadd_rn(sc, eps(nnv[e])));
          if (gb + e < N) {
            tmin = u[e] < tmin ? u[e] : tmin;
            tmax = u[e] > tmax ? u[e] : tmax;
            if ((((u[e] + 127u) & ~127u) | (uint32_t)(c0 + e)) < thr) below |= 1u << e;
          }
        }
        // insert them, keeping the order (only entries under the largest
        // before the chunk can enter it)
        if (below) {
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            if ((below >> e) & 1u) {
              uint32_t x = ((u[e] + 127u) & ~127u) | (uint32_t)(c0 + e);
#pragma unroll
              for (int jj = 0; jj < kProbePool; ++jj) {
                const uint32_t lo = min(top[jj], x);
                x = max(top[jj], x);
                top[jj] = lo;
              }
            }
          }
        }
        if (live) {
          if (gb + 16 <= N && (N & 3) == 0) {  // whole chunk: four 16-byte stores
            uint4* dst = reinterpret_cast<uint4*>(keys + row * N + gb);
#pragma unroll
            for (int v = 0; v < 4; ++v) dst[v] = make_uint4(u[4 * v], u[4 * v + 1], u[4 * v + 2], u[4 * v + 3]);
          } else {
#pragma unroll
            for (int e = 0; e < 16; ++e)
              if (gb + e < N) keys[row * N + gb + e] = u[e];
          }
        }
      }
      if (live) {
        atomicMin(kmin + row, tmin);
        atomicMax(kmax + row, tmax);
        // unused slots (past the last centroid) hold 0xffffffff, which no
        // real entry equals (finite keys are at most 0xff800000)
        uint4* dst = reinterpret_cast<uint4*>(pool + row * (int64_t)(2 * ntn * kProbePool) +
                                              (int64_t)(2 * nt + half) * kProbePool);
        dst[0] = make_uint4(top[0], top[1], top[2], top[3]);
        dst[1] = make_uint4(top[4], top[5], top[6], top[7]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&s_tempty[buf]))
                   : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0 && s_fail) atomicExch(err, 2);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                 "r"(2 * kPdN));
}

// Self-test of the bounded waits (two warps, nothing ever completes the
// barrier): warp 0 waits `polls` times on an mbarrier that no one arrives on
// and must give up (bit 0 of *status); then it waits again with no poll
// limit that matters while warp 1 raises the CTA's failure flag, and must
// give up on the flag (bit 1). The kernel then returns normally.
__global__ void wait_selftest_kernel(uint32_t polls, int* status) {
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ volatile int s_fail;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&s_bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  __syncthreads();
  int st = 0;
  if (threadIdx.x == 0) {
    if (!mbar_wait(smem_u32(&s_bar), 0u, polls)) st |= 1;
    if (!pd_wait(smem_u32(&s_bar), 0u, &s_fail)) st |= 2;  // ends once warp 1 sets the flag
    *status = st;
  } else if (threadIdx.x == 32) {
    const long long t0 = clock64();
    while (clock64() - t0 < 100000) {
    }
    s_fail = 1;
  }
  __syncthreads();
}

}  // namespace

int wait_selftest(uint32_t polls, int* status_host) {
  DevBuf st;
  RBQ_CHECK(st.alloc(sizeof(int), nullptr));
  RBQ_CUDA(cudaMemset(st.p, 0, sizeof(int)));
  wait_selftest_kernel<<<1, 64>>>(polls, st.as<int>());
  RBQ_CUDA(cudaGetLastError());
  RBQ_CUDA(cudaMemcpy(status_host, st.p, sizeof(int), cudaMemcpyDeviceToHost));
  return RABITQ_OK;
}

int64_t centroid_tile_rows(int K) { return ((int64_t)K + kPdN - 1) / kPdN * kPdN; }

ProbeScratch probe_scratch(const rabitq_index* X, int64_t nq, float* base) {
  const int64_t rows = (nq + kPdM - 1) / kPdM * kPdM;
  ProbeScratch v;
  size_t o = align_up((size_t)nq * X->K, 256);
  v.keys = reinterpret_cast<uint32_t*>(base);
  v.qt = base + o;
  o = align_up(o + (size_t)rows * X->kp, 64);
  v.nq2 = base + o;
  o = align_up(o + (size_t)nq, 64);
  v.kmin = reinterpret_cast<uint32_t*>(base + o);
  o = align_up(o + (size_t)nq, 64);
  v.kmax = reinterpret_cast<uint32_t*>(base + o);
  o = align_up(o + (size_t)nq, 64);
  v.pool_n = 2 * kProbePool * (int)((X->K + kPdN - 1) / kPdN);
  v.pool = reinterpret_cast<uint32_t*>(base + o);
  o = align_up(o + (size_t)nq * v.pool_n, 64);
  v.floats = o;
  return v;
}

size_t probe_scratch_floats(const rabitq_index* X, int64_t nq) {
  return probe_scratch(X, nq, nullptr).floats;
}

int pack_centroids(rabitq_index* X, cudaStream_t s) {
  const int64_t rows = centroid_tile_rows(X->K);
  const int64_t total = rows * X->kp;
  pack_centroids_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
      X->centroids, X->K, X->d, X->kp, rows, X->ctf, X->cn2, X->cnorm);
  RBQ_CUDA(cudaGetLastError());
  max_norm_kernel<<<1, 1024, 0, s>>>(X->cnorm, X->K, X->cnorm_max);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

int probe_keys_tc(const rabitq_index* X, const float* Q, int64_t M, float* scratch, int* err,
                  cudaStream_t s) {
  if (M <= 0) return RABITQ_OK;
  const int N = X->K, Kp = X->kp, nks = Kp / kPdEl;
  const int64_t rows = (M + kPdM - 1) / kPdM * kPdM;
  const ProbeScratch v = probe_scratch(X, M, scratch);
  query_prep_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(Q, M, X->d, Kp, rows, v.qt,
                                                                        v.nq2, v.kmin, v.kmax);
  RBQ_CUDA(cudaGetLastError());
  const int ntn = (N + kPdN - 1) / kPdN;
  const int64_t items = (rows / kPdM) * ntn;
  int dev = 0, sms = 0;
  RBQ_CUDA(cudaGetDevice(&dev));
  RBQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t grid = std::min<int64_t>(items, sms);
  RBQ_CUDA(cudaFuncSetAttribute(probe_dot_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kPdSmem));
  probe_dot_kernel<<<(unsigned)grid, kPdThreads, kPdSmem, s>>>(
      v.qt, X->ctf, M, N, nks, ntn, items, X->d, X->metric != RABITQ_METRIC_L2 ? 1 : 0, v.nq2,
      X->cn2, X->cnorm, v.keys, v.kmin, v.kmax, v.pool, err);
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
