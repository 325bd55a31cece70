// kernels_mlp.cu -- learned probe count (an extension: §4 of the paper
// probes a fixed number of buckets). An MLP 64 -> 256 -> 256 -> 1 reads
// features of a query's 64 smallest centroid distances and predicts log2 of
// the number of buckets to probe. Trained on the GPU by the kernels below:
// the canonical-order contractions of kernels_gemm.cu for the forward and
// backward products (FP32, ascending reduction index, so every pass is
// deterministic), element-wise bias/ReLU/mask kernels, ordered column sums,
// and Adam on an FP32 master copy whose BF16 rounding is the working weight.
//
// Layers (row-major, batch B): Z1 = X W1 + b1, H1 = relu(Z1);
// Z2 = H1 W2 + b2, H2 = relu(Z2); y = H2 w3 + b3. Loss = mean (y - t)^2.
// Inference is one fused kernel (features + three layers + probe count)
// reading the BF16 weights; its arithmetic is the training forward's, term
// for term, so both give the same y bit for bit.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace rbq {
namespace {

constexpr int kF = kMlpIn, kH = kMlpHidden;

// parameter offsets in the packed vector
constexpr int oW1 = 0, ob1 = oW1 + kF * kH, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, ow3 = ob2 + kH,
              ob3 = ow3 + kH, kParams = ob3 + 1;
static_assert(kParams == kMlpParams, "parameter count");

constexpr int kGrid = 512;  // calibration grid: mult_i = 2^((i - 128) / 32)

inline unsigned nb(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__global__ void bias_act_kernel(float* __restrict__ Z, int64_t B, int N,
                                const float* __restrict__ b, float* __restrict__ H) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= B * N) return;
  const float z = __fadd_rn(Z[i], b[i % N]);
  Z[i] = z;
  if (H) H[i] = z > 0.0f ? z : 0.0f;
}

// dy = 2 (y - t) / B
__global__ void loss_grad_kernel(const float* __restrict__ y, const float* __restrict__ t,
                                 int64_t B, float* __restrict__ dy) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= B) return;
  const float e = __fsub_rn(y[i], t[i]);
  dy[i] = __fdiv_rn(__fmul_rn(2.0f, e), (float)B);
}

// dZ2[b][n] = dy[b] w3[n] [Z2[b][n] > 0]
__global__ void outer_mask_kernel(const float* __restrict__ dy, const float* __restrict__ w,
                                  const float* __restrict__ Z, int64_t B, int N,
                                  float* __restrict__ dZ) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= B * N) return;
  dZ[i] = Z[i] > 0.0f ? __fmul_rn(dy[i / N], w[i % N]) : 0.0f;
}

__global__ void mask_kernel(float* __restrict__ dH, const float* __restrict__ Z, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && !(Z[i] > 0.0f)) dH[i] = 0.0f;
}

// column sums over the batch in ascending row order (bias gradients)
__global__ void colsum_kernel(const float* __restrict__ A, int64_t B, int N,
                              float* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.0f;
  for (int64_t b = 0; b < B; ++b) s = __fadd_rn(s, A[b * N + n]);
  out[n] = s;
}

// Adam on the FP32 master parameters; the working copy is its BF16 rounding.
__global__ void adam_kernel(float* __restrict__ master, float* __restrict__ work,
                            const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, int n, float lr, float b1, float b2,
                            float c1, float c2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = __fadd_rn(__fmul_rn(b1, m1[i]), __fmul_rn(__fsub_rn(1.0f, b1), gi));
  const float v =
      __fadd_rn(__fmul_rn(b2, m2[i]), __fmul_rn(__fsub_rn(1.0f, b2), __fmul_rn(gi, gi)));
  m1[i] = a;
  m2[i] = v;
  const float mh = __fdiv_rn(a, c1), vh = __fdiv_rn(v, c2);
  const float step = __fdiv_rn(__fmul_rn(lr, mh), __fadd_rn(__fsqrt_rn(vh), eps));
  const float w = __fsub_rn(master[i], step);
  master[i] = w;
  work[i] = __bfloat162float(__float2bfloat16_rn(w));
}

__global__ void round_bf16_kernel(const float* __restrict__ in, float* __restrict__ out,
                                  __nv_bfloat16* __restrict__ packed, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const __nv_bfloat16 h = __float2bfloat16_rn(in[i]);
  if (out) out[i] = __bfloat162float(h);
  if (packed) packed[i] = h;
}

// Feature j of a query from its ascending centroid distances d (navail valid
// entries; the last repeats beyond them).
__device__ __forceinline__ float feature(const float* d, int navail, int j, float s0) {
  const float d0 = d[0];
  if (j == 0) return __fdiv_rn(d0, __fadd_rn(d0, s0));
  const float dj = d[min(j, navail - 1)];
  return dj > 0.0f ? __fdiv_rn(d0, dj) : 1.0f;
}

__global__ void features_kernel(const float* __restrict__ sel_dist, int64_t ld, int64_t nq,
                                int navail, float s0, float* __restrict__ X) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nq * kF) return;
  X[i] = feature(sel_dist + (i / kF) * ld, navail, (int)(i % kF), s0);
}

// probe count from the network output: clamp(ceil(mult 2^y), 1, nmax)
__device__ __forceinline__ int probe_count(float y, float mult, int nmax) {
  const float v = __fmul_rn(mult, exp2f(fminf(y, 30.0f)));
  if (!(v < (float)nmax)) return nmax;  // also NaN
  const int n = (int)ceilf(v);
  return n < 1 ? 1 : n;
}

// Fused inference: kQB queries per block, one hidden unit per thread. The
// activations are stored transposed ([unit][query]) so that each step of a
// dot product reads the kQB values of one unit with 16-byte broadcast loads.
constexpr int kQB = 32, kInferThreads = kH;
constexpr size_t kInferSmem = sizeof(float) * (kQB * kF + 2 * kQB * kH);

__global__ void __launch_bounds__(kInferThreads) mlp_infer_kernel(
    const float* __restrict__ sel_dist, int64_t ld, int64_t nq, int navail, float s0,
    const __nv_bfloat16* __restrict__ P, float mult, int nmax, float* __restrict__ feat_out,
    float* __restrict__ y_out, int32_t* __restrict__ np_out) {
  extern __shared__ __align__(1024) float sm[];
  float* xT = sm;               // kF x kQB
  float* h1T = xT + kQB * kF;   // kH x kQB
  float* h2T = h1T + kQB * kH;  // kH x kQB
  const int tid = threadIdx.x;
  const int64_t q0 = (int64_t)blockIdx.x * kQB;
  const int nqb = (int)(nq - q0 < kQB ? nq - q0 : kQB);
  for (int i = tid; i < kQB * kF; i += blockDim.x) {
    const int q = i / kF, j = i % kF;
    float v = 0.0f;
    if (q < nqb) {
      v = feature(sel_dist + (q0 + q) * ld, navail, j, s0);
      if (feat_out) feat_out[(q0 + q) * kF + j] = v;
    }
    xT[j * kQB + q] = v;
  }
  __syncthreads();
  const int n = tid;
  float acc[kQB];
  // one dense layer: acc[q] = fold_j fma(in[j][q], W[j][n], acc[q]), ascending j
  auto layer = [&](const float* inT, int nin, int woff) {
#pragma unroll
    for (int q = 0; q < kQB; ++q) acc[q] = 0.0f;
    for (int j = 0; j < nin; ++j) {
      const float w = __bfloat162float(P[woff + j * kH + n]);
      const float4* a4 = reinterpret_cast<const float4*>(inT + j * kQB);
#pragma unroll
      for (int c = 0; c < kQB / 4; ++c) {
        const float4 a = a4[c];
        acc[4 * c] = __fmaf_rn(a.x, w, acc[4 * c]);
        acc[4 * c + 1] = __fmaf_rn(a.y, w, acc[4 * c + 1]);
        acc[4 * c + 2] = __fmaf_rn(a.z, w, acc[4 * c + 2]);
        acc[4 * c + 3] = __fmaf_rn(a.w, w, acc[4 * c + 3]);
      }
    }
  };
  auto bias_relu_store = [&](int boff, float* outT) {
    const float bb = __bfloat162float(P[boff + n]);
    float4* o4 = reinterpret_cast<float4*>(outT + n * kQB);
#pragma unroll
    for (int c = 0; c < kQB / 4; ++c) {
      float4 v;
      float z = __fadd_rn(acc[4 * c], bb);
      v.x = z > 0.0f ? z : 0.0f;
      z = __fadd_rn(acc[4 * c + 1], bb);
      v.y = z > 0.0f ? z : 0.0f;
      z = __fadd_rn(acc[4 * c + 2], bb);
      v.z = z > 0.0f ? z : 0.0f;
      z = __fadd_rn(acc[4 * c + 3], bb);
      v.w = z > 0.0f ? z : 0.0f;
      o4[c] = v;
    }
  };
  layer(xT, kF, oW1);
  bias_relu_store(ob1, h1T);
  __syncthreads();
  layer(h1T, kH, oW2);
  bias_relu_store(ob2, h2T);
  __syncthreads();
  // output layer: one lane per query, ascending hidden index
  if (tid < nqb) {
    float s = 0.0f;
    for (int j = 0; j < kH; ++j)
      s = __fmaf_rn(h2T[j * kQB + tid], __bfloat162float(P[ow3 + j]), s);
    const float y = __fadd_rn(s, __bfloat162float(P[ob3]));
    if (y_out) y_out[q0 + tid] = y;
    if (np_out) np_out[q0 + tid] = probe_count(y, mult, nmax);
  }
}

// Labels: ranks of the buckets of a query's true neighbours among its nmax
// nearest buckets (ids in ascending (distance, id) order), censored at nmax;
// label_r = min(1 + the need-th smallest rank, nmax).
__global__ void __launch_bounds__(256) label_kernel(
    const int32_t* __restrict__ sel_ids, int64_t ld, int nmax, int K,
    const int64_t* __restrict__ gt, int k, int need, const int32_t* __restrict__ assign,
    int64_t n_points, int sort_n, int32_t* __restrict__ ranks, int32_t* __restrict__ label_r) {
  extern __shared__ __align__(1024) unsigned char lsm[];
  uint16_t* table = reinterpret_cast<uint16_t*>(lsm);  // K entries: rank or nmax
  uint32_t* srt = reinterpret_cast<uint32_t*>(lsm + ((sizeof(uint16_t) * K + 15) / 16) * 16);
  const int64_t q = blockIdx.x;
  for (int c = threadIdx.x; c < K; c += blockDim.x) table[c] = (uint16_t)nmax;
  __syncthreads();
  for (int j = threadIdx.x; j < nmax; j += blockDim.x) {
    const int c = sel_ids[q * ld + j];
    if (c >= 0 && c < K) table[c] = (uint16_t)j;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < sort_n; j += blockDim.x) {
    uint32_t r = 0xffffffffu;
    if (j < k) {
      const int64_t id = gt[q * k + j];
      r = (uint32_t)nmax;
      if (id >= 0 && id < n_points) r = table[assign[id]];
      ranks[q * k + j] = (int32_t)r;
    }
    srt[j] = r;
  }
  __syncthreads();
  block_bitonic_sort_u32(srt, sort_n);
  if (threadIdx.x == 0) label_r[q] = (int32_t)min(srt[need - 1] + 1u, (uint32_t)nmax);
}

__global__ void log2_label_kernel(const int32_t* __restrict__ r, int64_t n, float* __restrict__ t) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) t[i] = log2f((float)r[i]);
}

// One block, fixed order: mean over rows of d[row * ld] in FP64.
__global__ void mean_first_kernel(const float* __restrict__ d, int64_t ld, int64_t n,
                                  double* __restrict__ out) {
  __shared__ double part[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)d[i * ld];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = part[0] / (double)n;
}

// One block, fixed order: sum of (y - t)^2 in FP64.
__global__ void sq_err_kernel(const float* __restrict__ y, const float* __restrict__ t, int64_t n,
                              double* __restrict__ out) {
  __shared__ double part[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double e = (double)y[i] - (double)t[i];
    s += e * e;
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = part[0];
}

// Calibration: block i tries mult_i; counts (exactly, in integers) the
// validation neighbours inside the predicted buckets and the probe counts.
__global__ void __launch_bounds__(256) coverage_kernel(
    const float* __restrict__ y, const int32_t* __restrict__ ranks, int64_t nv, int k, int nmax,
    float* __restrict__ mults, unsigned long long* __restrict__ covered,
    unsigned long long* __restrict__ probes) {
  const int i = blockIdx.x;
  const float mult = exp2f((float)(i - 128) / 32.0f);
  unsigned long long cov = 0, np_sum = 0;
  for (int64_t q = threadIdx.x; q < nv; q += blockDim.x) {
    const int np = probe_count(y[q], mult, nmax);
    np_sum += (unsigned long long)np;
    for (int j = 0; j < k; ++j) cov += ranks[q * k + j] < np ? 1ull : 0ull;
  }
  __shared__ unsigned long long s_cov, s_np;
  if (threadIdx.x == 0) {
    s_cov = 0;
    s_np = 0;
  }
  __syncthreads();
  atomicAdd(&s_cov, cov);
  atomicAdd(&s_np, np_sum);
  __syncthreads();
  if (threadIdx.x == 0) {
    mults[i] = mult;
    covered[i] = s_cov;
    probes[i] = s_np;
  }
}

// Initial parameters: He-uniform weights from a seeded host generator, zero
// biases (rounded to BF16 values on the device).
void mlp_init(std::vector<float>& p, uint64_t seed) {
  p.assign(kParams, 0.0f);
  std::mt19937_64 g(seed);
  auto fill = [&](int off, int fan_in, int n) {
    const float a = std::sqrt(6.0f / (float)fan_in);
    std::uniform_real_distribution<float> u(-a, a);
    for (int i = 0; i < n; ++i) p[off + i] = u(g);
  };
  fill(oW1, kF, kF * kH);
  fill(oW2, kH, kH * kH);
  fill(ow3, kH, kH);
}

}  // namespace

int MlpWork::alloc(int64_t B, cudaStream_t s) {
  const int64_t nT = std::max<int64_t>(B, kH) * kH;
  RBQ_CHECK(buf.alloc(sizeof(float) * (size_t)(B * kH * 6 + B * 3 + nT + kH * kH), s));
  float* p = buf.as<float>();
  Z1 = p; p += B * kH;
  H1 = p; p += B * kH;
  Z2 = p; p += B * kH;
  H2 = p; p += B * kH;
  dH2 = p; p += B * kH;
  dH1 = p; p += B * kH;
  y = p; p += B;
  dy = p; p += B;
  se = p; p += B;
  T = p; p += nT;
  W2T = p;
  return RABITQ_OK;
}

int mlp_forward(const float* params, const float* X, int64_t B, float* Z1, float* H1, float* Z2,
                float* H2, float* y, cudaStream_t s) {
  if (B <= 0) return RABITQ_OK;
  RBQ_CHECK(gemm_canon(kDot, X, kF, nullptr, nullptr, 0, nullptr, params + oW1, kH, Z1, kH, B, kH,
                       kF, s));
  bias_act_kernel<<<nb(B * kH, 256), 256, 0, s>>>(Z1, B, kH, params + ob1, H1);
  RBQ_CHECK(gemm_canon(kDot, H1, kH, nullptr, nullptr, 0, nullptr, params + oW2, kH, Z2, kH, B, kH,
                       kH, s));
  bias_act_kernel<<<nb(B * kH, 256), 256, 0, s>>>(Z2, B, kH, params + ob2, H2);
  RBQ_CHECK(gemm_canon(kDot, H2, kH, nullptr, nullptr, 0, nullptr, params + ow3, 1, y, 1, B, 1, kH,
                       s));
  bias_act_kernel<<<nb(B, 256), 256, 0, s>>>(y, B, 1, params + ob3, nullptr);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

int mlp_backward(const float* params, const float* X, const float* t, int64_t B, float* grads,
                 MlpWork& w, cudaStream_t s) {
  RBQ_CHECK(mlp_forward(params, X, B, w.Z1, w.H1, w.Z2, w.H2, w.y, s));
  loss_grad_kernel<<<nb(B, 256), 256, 0, s>>>(w.y, t, B, w.dy);
  // output layer: dw3 = H2^T dy, db3 = sum dy
  RBQ_CHECK(transpose_f32(w.H2, B, kH, w.T, s));
  RBQ_CHECK(gemm_canon(kDot, w.T, B, nullptr, nullptr, 0, nullptr, w.dy, 1, grads + ow3, 1, kH, 1,
                       (int)B, s));
  colsum_kernel<<<1, 32, 0, s>>>(w.dy, B, 1, grads + ob3);
  // second layer: dZ2 = dy w3^T [Z2 > 0]; dW2 = H1^T dZ2; db2 = colsum dZ2
  outer_mask_kernel<<<nb(B * kH, 256), 256, 0, s>>>(w.dy, params + ow3, w.Z2, B, kH, w.dH2);
  RBQ_CHECK(transpose_f32(w.H1, B, kH, w.T, s));
  RBQ_CHECK(gemm_canon(kDot, w.T, B, nullptr, nullptr, 0, nullptr, w.dH2, kH, grads + oW2, kH, kH,
                       kH, (int)B, s));
  colsum_kernel<<<nb(kH, 128), 128, 0, s>>>(w.dH2, B, kH, grads + ob2);
  // first layer: dZ1 = dZ2 W2^T [Z1 > 0]; dW1 = X^T dZ1; db1 = colsum dZ1
  RBQ_CHECK(transpose_f32(params + oW2, kH, kH, w.W2T, s));
  RBQ_CHECK(gemm_canon(kDot, w.dH2, kH, nullptr, nullptr, 0, nullptr, w.W2T, kH, w.dH1, kH, B, kH,
                       kH, s));
  mask_kernel<<<nb(B * kH, 256), 256, 0, s>>>(w.dH1, w.Z1, B * kH);
  RBQ_CHECK(transpose_f32(X, B, kF, w.T, s));
  RBQ_CHECK(gemm_canon(kDot, w.T, B, nullptr, nullptr, 0, nullptr, w.dH1, kH, grads + oW1, kH, kF,
                       kH, (int)B, s));
  colsum_kernel<<<nb(kH, 128), 128, 0, s>>>(w.dH1, B, kH, grads + ob1);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

int mlp_adam(float* master, float* work, const float* g, float* m1, float* m2, float lr, int step,
             cudaStream_t s) {
  // beta1, beta2 are the FP32 values 0.9f, 0.999f everywhere (also in the
  // bias corrections 1 - beta^step, evaluated in FP64 and rounded once)
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = (float)(1.0 - std::pow((double)b1, step));
  const float c2 = (float)(1.0 - std::pow((double)b2, step));
  adam_kernel<<<nb(kParams, 256), 256, 0, s>>>(master, work, g, m1, m2, kParams, lr, b1, b2, c1,
                                               c2, 1e-8f);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

int mlp_features(const float* sel_dist, int64_t ld, int64_t nq, int navail, float s0, float* X,
                 cudaStream_t s) {
  if (nq <= 0) return RABITQ_OK;
  features_kernel<<<nb(nq * kF, 256), 256, 0, s>>>(sel_dist, ld, nq, navail, s0, X);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

int mlp_infer(const rabitq_predictor* pr, const float* sel_dist, int64_t ld, int64_t nq,
              int navail, int32_t* nprobe_out, float* feat, float* y, cudaStream_t s) {
  if (nq <= 0) return RABITQ_OK;
  RBQ_CUDA(cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kInferSmem));
  mlp_infer_kernel<<<nb(nq, kQB), kInferThreads, kInferSmem, s>>>(
      sel_dist, ld, nq, navail, pr->s0, static_cast<const __nv_bfloat16*>(pr->params_bf16),
      pr->mult, pr->nprobe_max, feat, y, nprobe_out);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

int mlp_round(const float* in, float* out, void* packed, int n, cudaStream_t s) {
  round_bf16_kernel<<<nb(n, 256), 256, 0, s>>>(in, out, static_cast<__nv_bfloat16*>(packed), n);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

int mlp_pack_bf16(rabitq_predictor* pr, cudaStream_t s) {
  return mlp_round(pr->params, pr->params, pr->params_bf16, kParams, s);
}

int mlp_sum_sq_err(const float* y, const float* t, int64_t n, double* out, cudaStream_t s) {
  sq_err_kernel<<<1, 256, 0, s>>>(y, t, n, out);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

// Ranks and label probe counts of nq queries with true neighbours gt (device).
int mlp_labels_dev(const rabitq_index* X, const float* Q, int64_t nq, const int64_t* gt, int k,
                   int need, int nmax, int32_t* ranks, int32_t* label_r, cudaStream_t s) {
  if (nq <= 0) return RABITQ_OK;
  const int K = X->K;
  int sort_n = 1;
  while (sort_n < k) sort_n <<= 1;
  const size_t smem = ((sizeof(uint16_t) * K + 15) / 16) * 16 + sizeof(uint32_t) * sort_n;
  // one fixed limit (K <= 65536, k <= 1024), so concurrent callers agree
  RBQ_CUDA(cudaFuncSetAttribute(label_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(uint16_t) * 65536 + sizeof(uint32_t) * 1024)));
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(nq, (int64_t(1) << 26) / nmax));
  DevBuf ids, dist;
  RBQ_CHECK(ids.alloc(sizeof(int32_t) * chunk * nmax, s));
  RBQ_CHECK(dist.alloc(sizeof(float) * chunk * nmax, s));
  for (int64_t q0 = 0; q0 < nq; q0 += chunk) {
    const int64_t m = std::min(chunk, nq - q0);
    RBQ_CHECK(select_buckets(X, Q + q0 * X->d, m, nmax, ids.as<int32_t>(), dist.as<float>(), s));
    label_kernel<<<(unsigned)m, 256, smem, s>>>(ids.as<int32_t>(), nmax, nmax, K, gt + q0 * k, k,
                                               need, X->assign, X->n, sort_n, ranks + q0 * k,
                                               label_r + q0);
    RBQ_CUDA(cudaGetLastError());
  }
  return RABITQ_OK;
}

// Labels, features, training and calibration (rabitq_predictor_train).
int predictor_train_dev(const rabitq_index* X, const float* Q, int64_t nt, const int64_t* gt_in,
                        const rabitq_predictor_opts& o, rabitq_predictor* pr, cudaStream_t s) {
  const int K = X->K, k = o.k;
  const int nmax = pr->nprobe_max;
  const int need = mlp_need(o.target_recall, k);
  // 1. true neighbours: the re-ranked search over the nmax nearest buckets
  DevBuf gtb, gdist;
  const int64_t* gt = gt_in;
  if (!gt) {
    RBQ_CHECK(gtb.alloc(sizeof(int64_t) * nt * k, s));
    RBQ_CHECK(gdist.alloc(sizeof(float) * nt * k, s));
    SearchArgs a;
    a.X = X;
    a.queries = Q;
    a.nq = nt;
    a.k = k;
    a.nprobe = nmax;
    a.bq = 4;
    a.eps0 = 1.9f;
    a.seed = 3;
    a.per_query_nprobe = nullptr;
    a.cand_cap = 1 << 18;
    a.out_ids = gtb.as<int64_t>();
    a.out_dist = gdist.as<float>();
    a.trace = nullptr;
    a.rot_precision = RABITQ_ROT_FP32;
    a.scan_path = RABITQ_SCAN_POPC;
    a.stage_ms = nullptr;
    RBQ_CHECK(search_dev(a, s));
    gt = gtb.as<int64_t>();
  }
  // 2. labels
  DevBuf ranks, label_r, tl;
  RBQ_CHECK(ranks.alloc(sizeof(int32_t) * nt * k, s));
  RBQ_CHECK(label_r.alloc(sizeof(int32_t) * nt, s));
  RBQ_CHECK(tl.alloc(sizeof(float) * nt, s));
  RBQ_CHECK(mlp_labels_dev(X, Q, nt, gt, k, need, nmax, ranks.as<int32_t>(), label_r.as<int32_t>(),
                           s));
  log2_label_kernel<<<nb(nt, 256), 256, 0, s>>>(label_r.as<int32_t>(), nt, tl.as<float>());
  RBQ_CUDA(cudaGetLastError());
  // 3. features: the 64 smallest centroid distances, s0 = mean d_0
  const int navail = std::min(kF, K);
  DevBuf dsel_ids, dsel, feat, s0buf;
  RBQ_CHECK(dsel_ids.alloc(sizeof(int32_t) * nt * navail, s));
  RBQ_CHECK(dsel.alloc(sizeof(float) * nt * navail, s));
  RBQ_CHECK(feat.alloc(sizeof(float) * nt * kF, s));
  RBQ_CHECK(s0buf.alloc(sizeof(double), s));
  RBQ_CHECK(select_buckets(X, Q, nt, navail, dsel_ids.as<int32_t>(), dsel.as<float>(), s));
  mean_first_kernel<<<1, 256, 0, s>>>(dsel.as<float>(), navail, nt, s0buf.as<double>());
  RBQ_CUDA(cudaGetLastError());
  double s0 = 0.0;
  RBQ_CUDA(cudaMemcpyAsync(&s0, s0buf.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaStreamSynchronize(s));
  pr->s0 = (s0 > 0.0 && std::isfinite(s0)) ? (float)s0 : 1.0f;
  RBQ_CHECK(mlp_features(dsel.as<float>(), navail, nt, navail, pr->s0, feat.as<float>(), s));

  // 4. training on the first ntr queries
  const int64_t nval = std::max<int64_t>(
      1, std::min<int64_t>(nt - 1, (int64_t)std::floor((double)nt * o.val_fraction)));
  const int64_t ntr = nt - nval;
  const int64_t B = std::min<int64_t>(o.batch, ntr);
  std::vector<float> init;
  mlp_init(init, o.seed);
  DevBuf master, m1, m2, grads, perm, xb, tb;
  RBQ_CHECK(master.alloc(sizeof(float) * kParams, s));
  RBQ_CHECK(m1.alloc(sizeof(float) * kParams, s));
  RBQ_CHECK(m2.alloc(sizeof(float) * kParams, s));
  RBQ_CHECK(grads.alloc(sizeof(float) * kParams, s));
  RBQ_CHECK(perm.alloc(sizeof(int32_t) * ntr, s));
  RBQ_CHECK(xb.alloc(sizeof(float) * B * kF, s));
  RBQ_CHECK(tb.alloc(sizeof(float) * B, s));
  RBQ_CUDA(cudaMemcpyAsync(master.p, init.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice,
                           s));
  RBQ_CHECK(mlp_round(master.as<float>(), master.as<float>(), nullptr, kParams, s));
  RBQ_CUDA(cudaMemcpyAsync(pr->params, master.p, sizeof(float) * kParams,
                           cudaMemcpyDeviceToDevice, s));
  RBQ_CUDA(cudaMemsetAsync(m1.p, 0, sizeof(float) * kParams, s));
  RBQ_CUDA(cudaMemsetAsync(m2.p, 0, sizeof(float) * kParams, s));
  MlpWork w;
  RBQ_CHECK(w.alloc(B, s));
  std::vector<int32_t> order(ntr);
  std::mt19937_64 g(o.seed ^ 0x9e3779b97f4a7c15ull);
  int step = 0;
  for (int e = 0; e < o.epochs; ++e) {
    std::iota(order.begin(), order.end(), 0);
    std::shuffle(order.begin(), order.end(), g);
    RBQ_CUDA(cudaMemcpyAsync(perm.p, order.data(), sizeof(int32_t) * ntr, cudaMemcpyHostToDevice,
                             s));
    RBQ_CUDA(cudaStreamSynchronize(s));  // `order` is rewritten next epoch
    for (int64_t b0 = 0; b0 < ntr; b0 += B) {
      const int64_t bc = std::min(B, ntr - b0);
      RBQ_CHECK(gather_rows_f32(feat.as<float>(), kF, perm.as<int32_t>() + b0, bc, kF,
                                xb.as<float>(), s));
      RBQ_CHECK(gather_rows_f32(tl.as<float>(), 1, perm.as<int32_t>() + b0, bc, 1, tb.as<float>(),
                                s));
      RBQ_CHECK(mlp_backward(pr->params, xb.as<float>(), tb.as<float>(), bc, grads.as<float>(), w,
                             s));
      RBQ_CHECK(mlp_adam(master.as<float>(), pr->params, grads.as<float>(), m1.as<float>(),
                         m2.as<float>(), o.lr, ++step, s));
    }
  }
  // 5. losses and validation outputs (forward in batches of B)
  DevBuf yall, acc;
  RBQ_CHECK(yall.alloc(sizeof(float) * nt, s));
  RBQ_CHECK(acc.alloc(sizeof(double) * 2, s));
  for (int64_t b0 = 0; b0 < nt; b0 += B) {
    const int64_t bc = std::min(B, nt - b0);
    RBQ_CHECK(mlp_forward(pr->params, feat.as<float>() + b0 * kF, bc, w.Z1, w.H1, w.Z2, w.H2,
                          yall.as<float>() + b0, s));
  }
  sq_err_kernel<<<1, 256, 0, s>>>(yall.as<float>(), tl.as<float>(), ntr, acc.as<double>());
  sq_err_kernel<<<1, 256, 0, s>>>(yall.as<float>() + ntr, tl.as<float>() + ntr, nval,
                                  acc.as<double>() + 1);
  // 6. calibration of the multiplier on the validation split
  DevBuf mults, cov, nps;
  RBQ_CHECK(mults.alloc(sizeof(float) * kGrid, s));
  RBQ_CHECK(cov.alloc(sizeof(unsigned long long) * kGrid, s));
  RBQ_CHECK(nps.alloc(sizeof(unsigned long long) * kGrid, s));
  coverage_kernel<<<kGrid, 256, 0, s>>>(yall.as<float>() + ntr, ranks.as<int32_t>() + ntr * k,
                                        nval, k, nmax, mults.as<float>(),
                                        cov.as<unsigned long long>(), nps.as<unsigned long long>());
  RBQ_CUDA(cudaGetLastError());
  std::vector<float> h_mult(kGrid);
  std::vector<unsigned long long> h_cov(kGrid), h_np(kGrid);
  double h_acc[2];
  RBQ_CUDA(cudaMemcpyAsync(h_mult.data(), mults.p, sizeof(float) * kGrid, cudaMemcpyDeviceToHost,
                           s));
  RBQ_CUDA(cudaMemcpyAsync(h_cov.data(), cov.p, sizeof(unsigned long long) * kGrid,
                           cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaMemcpyAsync(h_np.data(), nps.p, sizeof(unsigned long long) * kGrid,
                           cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaMemcpyAsync(h_acc, acc.p, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaStreamSynchronize(s));
  const double total = (double)nval * k;
  int pick = kGrid - 1;
  for (int i = 0; i < kGrid; ++i)
    if ((double)h_cov[i] >= ((double)o.target_recall - 1e-6) * total) {
      pick = i;
      break;
    }
  pr->mult = h_mult[pick];
  pr->val_recall = (float)(h_cov[pick] / total);
  pr->val_mean_nprobe = (float)((double)h_np[pick] / (double)nval);
  pr->train_loss = (float)(h_acc[0] / (double)ntr);
  pr->val_loss = (float)(h_acc[1] / (double)nval);
  pr->n_train = ntr;
  pr->n_val = nval;
  return mlp_pack_bf16(pr, s);
}

}  // namespace rbq
