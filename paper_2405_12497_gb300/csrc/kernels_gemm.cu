// kernels_gemm.cu -- canonical-order SIMT contractions.
//
// Every output element is one thread's accumulator, folded over the
// reduction index in ascending order (canonical dot: fma(a, b, s); canonical
// squared distance: t = a - b, fma(t, t, s)), so the result is bit-identical
// to a plain sequential loop whatever the tile shape. Used for the residual
// rotation P^{-1}(o_r - c) of the index phase (§3.1.3), the query rotation
// (§3.3, FP32 mode), P^T c per centroid and the k-means assignment.
//
// Register-tiled: 128 x 128 block tile, 8-deep k slices staged in shared
// memory, an 8 x 8 micro-tile per thread (256 threads).
#include "common.cuh"
#include "internal.h"

namespace rbq {
namespace {

constexpr int BM = 128, BN = 128, BK = 8, NT = 256;

template <int OP>
__device__ __forceinline__ float accum(float acc, float a, float b) {
  if (OP == kDot) return __fmaf_rn(a, b, acc);
  const float t = __fsub_rn(a, b);
  return __fmaf_rn(t, t, acc);
}

// Stage one BK-deep slice of A' (transposed) and B into shared memory.
template <bool HAS_SUB>
__device__ __forceinline__ void load_slice(float (*As)[BM], float (*Bs)[BN],
                                           const float* const* arow, const float* const* srow,
                                           const bool* aval, const float* __restrict__ B,
                                           int64_t ldb, int k0, int n0, int N, int K) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const int idx = tid + NT * l;
    const int mm = idx >> 3, kk = idx & 7;
    const int gk = k0 + kk;
    float v = 0.0f;
    if (aval[l] && gk < K) {
      v = arow[l][gk];
      if (HAS_SUB) v = __fsub_rn(v, srow[l][gk]);
    }
    As[kk][mm] = v;
  }
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const int idx = tid + NT * l;
    const int kk = idx >> 7, nn = idx & 127;
    const int gk = k0 + kk, gn = n0 + nn;
    Bs[kk][nn] = (gk < K && gn < N) ? B[(int64_t)gk * ldb + gn] : 0.0f;
  }
}

template <int OP, bool HAS_SUB>
__device__ __forceinline__ void tile_product(float (&acc)[8][8], float (*As)[BM], float (*Bs)[BN],
                                             const float* const* arow, const float* const* srow,
                                             const bool* aval, const float* __restrict__ B,
                                             int64_t ldb, int n0, int N, int K) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  for (int k0 = 0; k0 < K; k0 += BK) {
    load_slice<HAS_SUB>(As, Bs, arow, srow, aval, B, ldb, k0, n0, N, K);
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[8], b[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 8; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = accum<OP>(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
}

template <bool HAS_SUB>
__device__ __forceinline__ void row_pointers(const float* A, int64_t lda, const int32_t* a_rows,
                                             const float* sub, int64_t ld_sub,
                                             const int32_t* sub_rows, int64_t m0, int64_t M,
                                             const float** arow, const float** srow, bool* aval) {
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const int mm = (threadIdx.x + NT * l) >> 3;
    const int64_t gm = m0 + mm;
    aval[l] = gm < M;
    const int64_t gmc = aval[l] ? gm : 0;
    const int64_t r = a_rows ? (int64_t)a_rows[gmc] : gmc;
    arow[l] = A + r * lda;
    srow[l] = HAS_SUB ? sub + (int64_t)sub_rows[gmc] * ld_sub : nullptr;
  }
}

template <int OP, bool HAS_SUB>
__global__ void __launch_bounds__(NT) gemm_canon_kernel(
    const float* __restrict__ A, int64_t lda, const int32_t* __restrict__ a_rows,
    const float* __restrict__ sub, int64_t ld_sub, const int32_t* __restrict__ sub_rows,
    const float* __restrict__ B, int64_t ldb, float* __restrict__ C, int64_t ldc, int64_t M,
    int N, int K) {
  __shared__ float As[BK][BM];
  __shared__ float Bs[BK][BN];
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;
  const float* arow[4];
  const float* srow[4];
  bool aval[4];
  row_pointers<HAS_SUB>(A, lda, a_rows, sub, ld_sub, sub_rows, m0, M, arow, srow, aval);
  float acc[8][8];
  tile_product<OP, HAS_SUB>(acc, As, Bs, arow, srow, aval, B, ldb, n0, N, K);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn < N) C[gm * ldc + gn] = acc[i][j];
    }
  }
}

// Row-wise argmin of canonical squared distances, ties to the lower column.
__global__ void __launch_bounds__(NT) argmin_sqdist_kernel(const float* __restrict__ A,
                                                           int64_t lda,
                                                           const float* __restrict__ Bt,
                                                           int64_t ldb, int64_t M, int N, int K,
                                                           int32_t* __restrict__ assign,
                                                           float* __restrict__ dist) {
  __shared__ float As[BK][BM];
  __shared__ float Bs[BK][BN];
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const float* arow[4];
  const float* srow[4];
  bool aval[4];
  row_pointers<false>(A, lda, nullptr, nullptr, 0, nullptr, m0, M, arow, srow, aval);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float best[8];
  int bidx[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    best[i] = __int_as_float(0x7f800000);
    bidx[i] = 0x7fffffff;
  }
  float acc[8][8];
  for (int n0 = 0; n0 < N; n0 += BN) {
    tile_product<kSqDist, false>(acc, As, Bs, arow, srow, aval, Bt, ldb, n0, N, K);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float v = __int_as_float(0x7f800000);
      int id = 0x7fffffff;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int gn = n0 + tx + 16 * j;
        if (gn < N && acc[i][j] < v) {  // ascending j = ascending column
          v = acc[i][j];
          id = gn;
        }
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        const float v2 = __shfl_xor_sync(kFull, v, o);
        const int i2 = __shfl_xor_sync(kFull, id, o);
        if (v2 < v || (v2 == v && i2 < id)) {
          v = v2;
          id = i2;
        }
      }
      if (v < best[i] || (v == best[i] && id < bidx[i])) {
        best[i] = v;
        bidx[i] = id;
      }
    }
  }
  if (tx == 0) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t gm = m0 + ty + 16 * i;
      if (gm < M) {
        assign[gm] = (bidx[i] == 0x7fffffff) ? 0 : bidx[i];  // all-infinite row
        if (dist) dist[gm] = best[i];
      }
    }
  }
}

}  // namespace

int gemm_canon(GemmOp op, const float* A, int64_t lda, const int32_t* a_rows, const float* sub,
               int64_t ld_sub, const int32_t* sub_rows, const float* B, int64_t ldb, float* C,
               int64_t ldc, int64_t M, int N, int K, cudaStream_t s) {
  if (M <= 0 || N <= 0) return RABITQ_OK;
  dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN));
  if (op == kDot) {
    if (sub)
      gemm_canon_kernel<kDot, true><<<grid, NT, 0, s>>>(A, lda, a_rows, sub, ld_sub, sub_rows, B,
                                                         ldb, C, ldc, M, N, K);
    else
      gemm_canon_kernel<kDot, false><<<grid, NT, 0, s>>>(A, lda, a_rows, nullptr, 0, nullptr, B,
                                                          ldb, C, ldc, M, N, K);
  } else {
    gemm_canon_kernel<kSqDist, false><<<grid, NT, 0, s>>>(A, lda, a_rows, nullptr, 0, nullptr,
                                                           B, ldb, C, ldc, M, N, K);
  }
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

int argmin_sqdist(const float* A, int64_t lda, const float* Bt, int64_t ldb, int64_t M, int N,
                  int K, int32_t* assign, float* dist, cudaStream_t s) {
  if (M <= 0) return RABITQ_OK;
  dim3 grid((unsigned)((M + BM - 1) / BM));
  argmin_sqdist_kernel<<<grid, NT, 0, s>>>(A, lda, Bt, ldb, M, N, K, assign, dist);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

}  // namespace rbq
