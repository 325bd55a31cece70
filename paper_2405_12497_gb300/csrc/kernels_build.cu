// kernels_build.cu -- index phase (Alg. 1 of the paper, with the IVF of §4):
// k-means buckets, the random orthogonal matrix P, sign codes and factors.
#include <atomic>
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace rbq {
namespace {

// ------------------------------------------------------------------ scan
constexpr int kScanThreads = 1024, kScanPer = 4, kScanTile = kScanThreads * kScanPer;

// Block-wide exclusive scan of one int per thread; returns the block total.
__device__ int block_exclusive_scan(int v, int* total) {
  __shared__ int warp_tot[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    int t = (lane < nw) ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;  // inclusive over warps
  }
  __syncthreads();
  const int before = (wid > 0) ? warp_tot[wid - 1] : 0;
  *total = warp_tot[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) scan_tile_sums(const int32_t* __restrict__ in,
                                                               int64_t n,
                                                               int32_t* __restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  int s = 0;
#pragma unroll
  for (int i = 0; i < kScanPer; ++i)
    if (base + i < n) s += in[base + i];
  int tot;
  block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) scan_sums_inplace(int32_t* __restrict__ sums,
                                                                  int nb) {
  int carry = 0;
  for (int b0 = 0; b0 < nb; b0 += kScanThreads) {
    const int i = b0 + threadIdx.x;
    const int v = (i < nb) ? sums[i] : 0;
    int tot;
    const int ex = block_exclusive_scan(v, &tot);
    if (i < nb) sums[i] = carry + ex;
    carry += tot;
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_tile_apply(const int32_t* __restrict__ in,
                                                                int32_t* __restrict__ out,
                                                                int64_t n,
                                                                const int32_t* __restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  int v[kScanPer];
  int s = 0;
#pragma unroll
  for (int i = 0; i < kScanPer; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0;
    s += v[i];
  }
  int tot;
  int run = block_exclusive_scan(s, &tot) + sums[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanPer; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
}

// ------------------------------------------------------- counting sort
// Stable counting sort of ids [0, n) by key. Warp w owns the id range
// [w*L, (w+1)*L); counts live in hist[c*nw + w] so that one exclusive scan
// in (key, warp) order yields every warp's output offset for every key.
__global__ void sort_hist_kernel(const int32_t* __restrict__ key, int64_t n, int nw, int64_t L,
                                 int32_t* __restrict__ hist) {
  const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= nw) return;
  const int64_t beg = (int64_t)w * L, end = min(n, beg + L);
  for (int64_t b = beg; b < end; b += 32) {
    const int64_t id = b + lane;
    const int c = (id < end) ? key[id] : -1;
    const unsigned mask = __match_any_sync(kFull, c);
    if (c >= 0 && lane == __ffs(mask) - 1) hist[(int64_t)c * nw + w] += __popc(mask);
    __syncwarp();
  }
}

__global__ void sort_scatter_kernel(const int32_t* __restrict__ key, int64_t n, int nw, int64_t L,
                                    int32_t* __restrict__ off, int32_t* __restrict__ perm) {
  const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= nw) return;
  const int64_t beg = (int64_t)w * L, end = min(n, beg + L);
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t b = beg; b < end; b += 32) {
    const int64_t id = b + lane;
    const int c = (id < end) ? key[id] : -1;
    const unsigned mask = __match_any_sync(kFull, c);
    int pos = 0;
    if (c >= 0) pos = off[(int64_t)c * nw + w] + __popc(mask & lt);
    __syncwarp();
    if (c >= 0 && lane == __ffs(mask) - 1) off[(int64_t)c * nw + w] += __popc(mask);
    __syncwarp();
    if (c >= 0) perm[pos] = (int32_t)id;
  }
}

// Counting sort of ids [0, n) by key in one block (small n and K): counts
// in shared memory, one scan, then each id takes the next slot of its key
// (the order within a key is unspecified).
constexpr int kOrderThreads = 1024;
__global__ void __launch_bounds__(kOrderThreads) order_sort_kernel(const int32_t* __restrict__ key,
                                                                   int n, int K,
                                                                   int32_t* __restrict__ perm,
                                                                   int32_t* __restrict__ offsets) {
  extern __shared__ int ocnt[];  // K
  for (int i = threadIdx.x; i < K; i += blockDim.x) ocnt[i] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&ocnt[key[i]], 1);
  __syncthreads();
  const int per = (K + (int)blockDim.x - 1) / (int)blockDim.x;
  const int b0 = min(K, (int)threadIdx.x * per), b1 = min(K, b0 + per);
  int sum = 0;
  for (int b = b0; b < b1; ++b) sum += ocnt[b];
  int tot;
  int run = block_exclusive_scan(sum, &tot);
  for (int b = b0; b < b1; ++b) {
    const int c = ocnt[b];
    ocnt[b] = run;
    offsets[b] = run;
    run += c;
  }
  if (threadIdx.x == 0) offsets[K] = n;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) perm[atomicAdd(&ocnt[key[i]], 1)] = i;
}

__global__ void bucket_offsets_kernel(const int32_t* __restrict__ off, int K, int nw, int64_t n,
                                      int32_t* __restrict__ offsets) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < K) offsets[c] = off[(int64_t)c * nw];
  if (c == K) offsets[K] = (int32_t)n;
}

// ------------------------------------------------------- small helpers
__global__ void gather_rows_kernel(const float* __restrict__ in, int64_t ld,
                                   const int32_t* __restrict__ rows, int64_t m, int d,
                                   float* __restrict__ out) {
  const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= m) return;
  const float* src = in + (int64_t)rows[r] * ld;
  float* dst = out + r * d;
  for (int i = lane; i < d; i += 32) dst[i] = src[i];
}

__global__ void invert_perm_kernel(const int32_t* __restrict__ perm, int64_t n,
                                   int32_t* __restrict__ inv) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < n) inv[perm[p]] = (int32_t)p;
}

__global__ void transpose_kernel(const float* __restrict__ in, int64_t rows, int64_t cols,
                                 float* __restrict__ out) {
  __shared__ float t[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[i][threadIdx.x] = in[r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[c * rows + r] = t[threadIdx.x][i];
  }
}

__global__ void finite_kernel(const float* __restrict__ x, int64_t count, int* __restrict__ bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) *bad = 1;
}

// ------------------------------------------------------------ rotation P
// Natural logarithm from the mathematics with basic IEEE operations only
// (bit-reproducible): x = m 2^e, m in [sqrt(1/2), sqrt(2)), log m =
// 2 atanh((m-1)/(m+1)) by its odd power series (12 terms).
__device__ double own_log(double x) {
  const long long bits = __double_as_longlong(x);
  long long e = ((bits >> 52) & 0x7ff) - 1023;
  double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
  if (m > 1.4142135623730951) {
    m = __dmul_rn(m, 0.5);
    e += 1;
  }
  const double y = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double z = __dmul_rn(y, y);
  double p = __ddiv_rn(1.0, 23.0);
  for (int j = 10; j >= 0; --j) {
    const double coef = __ddiv_rn(1.0, (double)(2 * j + 1));
    p = __dmul_rn(p, z);
    p = __dadd_rn(p, coef);
  }
  const double t1 = __dmul_rn((double)e, 0.6931471805599453);
  const double t2 = __dmul_rn(__dmul_rn(2.0, y), p);
  return __dadd_rn(t1, t2);
}

// Standard Gaussians by the Marsaglia polar method; pair m, attempt t draws
// Philox(seed; m, t, 0, tag) (53-bit uniforms from two words each).
__global__ void gaussian_kernel(uint64_t seed, int64_t pairs, double* __restrict__ G) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= pairs) return;
  double g0 = 0.0, g1 = 0.0;
  for (uint32_t t = 0; t < 64; ++t) {
    const U4 w = philox4x32_10(seed, (uint32_t)m, t, 0u, kTagGauss);
    const unsigned long long a = ((unsigned long long)w.x << 21) | (w.y >> 11);
    const unsigned long long b = ((unsigned long long)w.z << 21) | (w.w >> 11);
    const double u1 = __dmul_rn(__ull2double_rn(a), 0x1.0p-53);
    const double u2 = __dmul_rn(__ull2double_rn(b), 0x1.0p-53);
    const double v1 = __dsub_rn(__dmul_rn(2.0, u1), 1.0);
    const double v2 = __dsub_rn(__dmul_rn(2.0, u2), 1.0);
    const double s = __dadd_rn(__dmul_rn(v1, v1), __dmul_rn(v2, v2));
    if (s > 0.0 && s < 1.0) {
      const double q = __ddiv_rn(__dmul_rn(-2.0, own_log(s)), s);
      const double f = __dsqrt_rn(q);
      g0 = __dmul_rn(v1, f);
      g1 = __dmul_rn(v2, f);
      break;
    }
  }
  G[2 * m] = g0;
  G[2 * m + 1] = g1;
}

// Gram-Schmidt, one projection pass of row i: c_j = <v, p_j> for j < i
// (PT is P transposed so that threads j read consecutive addresses).
__global__ void gs_dot_kernel(const double* __restrict__ v, const double* __restrict__ PT, int i,
                              int dpad, double* __restrict__ c) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= i) return;
  double s = 0.0;
  for (int k = 0; k < dpad; ++k) s = __fma_rn(v[k], PT[(int64_t)k * dpad + j], s);
  c[j] = s;
}

// v_k -= sum_{j<i} c_j p_j[k]
__global__ void gs_update_kernel(double* __restrict__ v, const double* __restrict__ P,
                                 const double* __restrict__ c, int i, int dpad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= dpad) return;
  double t = 0.0;
  for (int j = 0; j < i; ++j) t = __fma_rn(c[j], P[(int64_t)j * dpad + k], t);
  v[k] = __dsub_rn(v[k], t);
}

// p_i = v / ||v||; also writes the transposed copy. One block of dpad threads
// (dpad <= 1024 is enforced by the caller via the grid-stride loop).
__global__ void gs_normalize_kernel(const double* __restrict__ v, int i, int dpad,
                                    double* __restrict__ P, double* __restrict__ PT) {
  __shared__ double nrm;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < dpad; ++k) s = __fma_rn(v[k], v[k], s);
    nrm = __dsqrt_rn(s);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < dpad; k += blockDim.x) {
    const double p = __ddiv_rn(v[k], nrm);
    P[(int64_t)i * dpad + k] = p;
    PT[(int64_t)k * dpad + i] = p;
  }
}

__global__ void to_f32_kernel(const double* __restrict__ in, int64_t count,
                              float* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < count) out[i] = __double2float_rn(in[i]);
}

// ------------------------------------------------------------------ k-means
__global__ void sample_flags_kernel(int64_t n, uint32_t thr, uint64_t seed,
                                    int32_t* __restrict__ flags) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const U4 w = philox4x32_10(seed, (uint32_t)i, 0u, 0u, kTagSample);
  flags[i] = (w.x < thr) ? 1 : 0;
}

__global__ void compact_kernel(const int32_t* __restrict__ flags, const int32_t* __restrict__ pos,
                               int64_t n, int32_t* __restrict__ ids) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && flags[i]) ids[pos[i]] = (int32_t)i;
}

// Floyd's sampling of K distinct indices of [0, m), in the order chosen.
// Sequential by nature (each pick depends on the set so far); K <= 65536.
__global__ void floyd_kernel(int64_t m, int K, uint64_t seed, uint8_t* __restrict__ taken,
                             int32_t* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int t = 0; t < K; ++t) {
    const unsigned long long j = (unsigned long long)(m - K + t);
    const U4 w = philox4x32_10(seed, (uint32_t)t, 0u, 0u, kTagKmeansInit);
    const unsigned long long r = ((unsigned long long)w.x * (j + 1)) >> 32;
    const unsigned long long pick = taken[r] ? j : r;
    taken[pick] = 1;
    out[t] = (int32_t)pick;
  }
}

// Mean update: centroid c = (sum of its members in ascending id order) /
// count; an empty cluster keeps its centroid.
__global__ void kmeans_update_kernel(const float* __restrict__ x, int d,
                                     const int32_t* __restrict__ perm,
                                     const int32_t* __restrict__ off,
                                     float* __restrict__ centroids) {
  const int c = blockIdx.x;
  const int beg = off[c], end = off[c + 1];
  if (end == beg) return;
  const float cnt = __int2float_rn(end - beg);
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    float s = 0.0f;
    int p = beg;
    for (; p + 4 <= end; p += 4) {  // loads issued ahead; adds stay in order
      const float a0 = x[(int64_t)perm[p] * d + i], a1 = x[(int64_t)perm[p + 1] * d + i];
      const float a2 = x[(int64_t)perm[p + 2] * d + i], a3 = x[(int64_t)perm[p + 3] * d + i];
      s = __fadd_rn(s, a0);
      s = __fadd_rn(s, a1);
      s = __fadd_rn(s, a2);
      s = __fadd_rn(s, a3);
    }
    for (; p < end; ++p) s = __fadd_rn(s, x[(int64_t)perm[p] * d + i]);
    centroids[(int64_t)c * d + i] = __fdiv_rn(s, cnt);
  }
}

// ------------------------------------------------------------ encoding
__global__ void position_cluster_kernel(const int32_t* __restrict__ off,
                                        int32_t* __restrict__ cl) {
  const int c = blockIdx.x;
  for (int p = off[c] + threadIdx.x; p < off[c + 1]; p += blockDim.x) cl[p] = c;
}

// One warp per row of R = P^{-1}(o_r - c): sign code, popcount, ||r||_1 and
// the per-vector factors of the estimator (Alg. 1 line 4, App. B.1).
// Inner-product metric (closing footnote of §6: <o_r, q_r> = ||o_r - c||
// ||q_r - c|| <o, q> + <o_r - c, c> + <q_r, c>): the score -<o_r, q_r> takes
// the estimator's form (F1 + add) - F2 xq with F1 = -<o_r - c, c> (canonical
// dot of the FP32 residual and c), F2 and F3 halved (exact scaling).
__global__ void encode_epilogue_kernel(const float* __restrict__ R, int64_t rows, int dpad,
                                       const float* __restrict__ adist,
                                       uint64_t* __restrict__ codes, float4* __restrict__ fac,
                                       int ip, const float* __restrict__ data_b,
                                       const float* __restrict__ centroids,
                                       const int32_t* __restrict__ cl, int d) {
  const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  const float* row = R + r * dpad;
  const int W = dpad >> 6;
  int pc = 0;
  for (int w = 0; w < W; ++w) {
    const unsigned lo = __ballot_sync(kFull, row[64 * w + lane] >= 0.0f);
    const unsigned hi = __ballot_sync(kFull, row[64 * w + 32 + lane] >= 0.0f);
    pc += __popc(lo) + __popc(hi);
    if (lane == 0) codes[r * W + w] = ((uint64_t)hi << 32) | lo;
  }
  if (lane != 0) return;
  float l1 = 0.0f;
  for (int k = 0; k < dpad; ++k) l1 = __fadd_rn(l1, fabsf(row[k]));
  const float F1 = adist[r];
  const float n_o = __fsqrt_rn(F1);
  float a_o = 1.0f;
  if (n_o > 0.0f) {
    const float den = __fmul_rn(__fsqrt_rn((float)dpad), n_o);
    a_o = __fdiv_rn(l1, den);
    if (a_o > 1.0f) a_o = 1.0f;
  }
  float F2 = __fdiv_rn(__fmul_rn(2.0f, n_o), a_o);
  const float om = __fsub_rn(1.0f, __fmul_rn(a_o, a_o));
  float F3 = __fdiv_rn(__fmul_rn(n_o, __fsqrt_rn(om)), a_o);
  float f1 = F1;
  if (ip) {  // RABITQ_METRIC_IP and RABITQ_METRIC_COSINE (unit rows)
    const float* o = data_b + r * d;
    const float* c = centroids + (int64_t)cl[r] * d;
    float oc = 0.0f;
    for (int i = 0; i < d; ++i) oc = __fmaf_rn(__fsub_rn(o[i], c[i]), c[i], oc);
    f1 = -oc;
    F2 = __fmul_rn(0.5f, F2);
    F3 = __fmul_rn(0.5f, F3);
  }
  fac[r] = make_float4(f1, F2, F3, (float)(2 * pc - dpad));
}

// Unit rows: one warp per row; lane 0 folds the canonical sum of squares,
// every lane divides its elements by the root (zero rows unchanged).
__global__ void normalize_rows_kernel(const float* __restrict__ in, int64_t n, int d,
                                      float* __restrict__ out) {
  const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= n) return;
  const float* x = in + r * d;
  float ss = 0.0f;
  if (lane == 0)
    for (int i = 0; i < d; ++i) ss = __fmaf_rn(x[i], x[i], ss);
  const float nrm = __fsqrt_rn(__shfl_sync(kFull, ss, 0));
  for (int i = lane; i < d; i += 32) {
    const float v = x[i];
    out[r * d + i] = nrm > 0.0f ? __fdiv_rn(v, nrm) : v;
  }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------- launchers
// The stream-ordered scratch comes from the device's default memory pool,
// which by default returns its memory to the system at every
// synchronization, so each search would map its scratch again (a gigabyte
// takes milliseconds). The pool is told once per device to keep what it
// holds; it then grows to the largest scratch in use and is reused.
static void keep_pool_memory() {
  static std::atomic<uint64_t> done{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  const uint64_t bit = uint64_t(1) << dev;
  if (done.load() & bit) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~uint64_t(0);
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done.fetch_or(bit);
}

int DevBuf::alloc(size_t bytes, cudaStream_t st) {
  s = st;
  if (bytes == 0) bytes = 16;
  keep_pool_memory();
  cudaError_t e = cudaMallocAsync(&p, bytes, st);
  if (e != cudaSuccess) {
    p = nullptr;
    return fail(RABITQ_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  return RABITQ_OK;
}

namespace {
int scan_ws(const int32_t* in, int32_t* out, int64_t n, int32_t* sums, cudaStream_t s) {
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  scan_tile_sums<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
  scan_sums_inplace<<<1, kScanThreads, 0, s>>>(sums, (int)nb);
  scan_tile_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}
}  // namespace

int exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return RABITQ_OK;
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  DevBuf sums;
  RBQ_CHECK(sums.alloc(sizeof(int32_t) * nb, s));
  return scan_ws(in, out, n, sums.as<int32_t>(), s);
}

namespace {
int64_t sort_windows(int64_t n, int32_t K) {
  int64_t nw = (n + 2047) / 2048;
  const int64_t cap = (int64_t(1) << 25) / K;
  if (nw > cap) nw = cap;
  if (nw < 1) nw = 1;
  return nw;
}
}  // namespace

int64_t counting_sort_ws_ints(int64_t n, int32_t K) {
  const int64_t cells = (int64_t)K * sort_windows(n, K);
  return 2 * cells + (cells + kScanTile - 1) / kScanTile;
}

int counting_sort_ws(const int32_t* key, int64_t n, int32_t K, int32_t* perm, int32_t* offsets,
                     int32_t* ws, cudaStream_t s) {
  const int64_t nw = sort_windows(n, K);
  const int64_t L = (n + nw - 1) / nw;
  const int64_t cells = (int64_t)K * nw;
  int32_t* hist = ws;
  int32_t* off = ws + cells;
  int32_t* sums = ws + 2 * cells;
  RBQ_CUDA(cudaMemsetAsync(hist, 0, sizeof(int32_t) * cells, s));
  const unsigned blocks = blocks_for(nw * 32, 256);
  sort_hist_kernel<<<blocks, 256, 0, s>>>(key, n, (int)nw, L, hist);
  RBQ_CUDA(cudaGetLastError());
  RBQ_CHECK(scan_ws(hist, off, cells, sums, s));
  bucket_offsets_kernel<<<blocks_for(K + 1, 256), 256, 0, s>>>(off, K, (int)nw, n, offsets);
  sort_scatter_kernel<<<blocks, 256, 0, s>>>(key, n, (int)nw, L, off, perm);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

bool order_sort_fits(int64_t n, int32_t K) { return n <= (int64_t(1) << 16) && K <= 8192; }

int order_sort(const int32_t* key, int64_t n, int32_t K, int32_t* perm, int32_t* offsets,
               int32_t* ws, cudaStream_t s) {
  if (n <= 0) return RABITQ_OK;
  if (!order_sort_fits(n, K)) return counting_sort_ws(key, n, K, perm, offsets, ws, s);
  order_sort_kernel<<<1, kOrderThreads, sizeof(int) * (size_t)K, s>>>(key, (int)n, K, perm, offsets);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

int counting_sort(const int32_t* key, int64_t n, int32_t K, int32_t* perm, int32_t* offsets,
                  cudaStream_t s) {
  DevBuf ws;
  RBQ_CHECK(ws.alloc(sizeof(int32_t) * counting_sort_ws_ints(n, K), s));
  return counting_sort_ws(key, n, K, perm, offsets, ws.as<int32_t>(), s);
}

int gather_rows_f32(const float* in, int64_t ld, const int32_t* rows, int64_t m, int32_t d,
                    float* out, cudaStream_t s) {
  if (m <= 0) return RABITQ_OK;
  gather_rows_kernel<<<blocks_for(m * 32, 256), 256, 0, s>>>(in, ld, rows, m, d, out);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

int invert_perm(const int32_t* perm, int64_t n, int32_t* inv, cudaStream_t s) {
  if (n <= 0) return RABITQ_OK;
  invert_perm_kernel<<<blocks_for(n, 256), 256, 0, s>>>(perm, n, inv);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

int transpose_f32(const float* in, int64_t rows, int64_t cols, float* out, cudaStream_t s) {
  dim3 grid(blocks_for(cols, 32), blocks_for(rows, 32));
  transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(in, rows, cols, out);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

int finite_flag(const float* x, int64_t count, int* flag, cudaStream_t s) {
  if (count <= 0) return RABITQ_OK;
  finite_kernel<<<(unsigned)std::min<int64_t>(blocks_for(count, 256), 4096), 256, 0, s>>>(
      x, count, flag);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

int check_finite(const float* x, int64_t count, cudaStream_t s, bool* finite) {
  DevBuf bad;
  RBQ_CHECK(bad.alloc(sizeof(int), s));
  RBQ_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
  if (count > 0) {
    finite_kernel<<<(unsigned)std::min<int64_t>(blocks_for(count, 256), 4096), 256, 0, s>>>(
        x, count, bad.as<int>());
    RBQ_CUDA(cudaGetLastError());
  }
  int h = 0;
  RBQ_CUDA(cudaMemcpyAsync(&h, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaStreamSynchronize(s));
  *finite = (h == 0);
  return RABITQ_OK;
}

int sample_rotation_dev(uint64_t seed, int32_t dpad, double* P64, float* P32, cudaStream_t s) {
  const int64_t total = (int64_t)dpad * dpad;
  DevBuf G, PT, v, c;
  RBQ_CHECK(G.alloc(sizeof(double) * total, s));
  RBQ_CHECK(PT.alloc(sizeof(double) * total, s));
  RBQ_CHECK(v.alloc(sizeof(double) * dpad, s));
  RBQ_CHECK(c.alloc(sizeof(double) * dpad, s));
  gaussian_kernel<<<blocks_for(total / 2, 128), 128, 0, s>>>(seed, total / 2, G.as<double>());
  RBQ_CUDA(cudaGetLastError());
  for (int i = 0; i < dpad; ++i) {
    RBQ_CUDA(cudaMemcpyAsync(v.p, G.as<double>() + (int64_t)i * dpad, sizeof(double) * dpad,
                             cudaMemcpyDeviceToDevice, s));
    if (i > 0) {
      for (int pass = 0; pass < 2; ++pass) {
        gs_dot_kernel<<<blocks_for(i, 64), 64, 0, s>>>(v.as<double>(), PT.as<double>(), i, dpad,
                                                      c.as<double>());
        gs_update_kernel<<<blocks_for(dpad, 64), 64, 0, s>>>(v.as<double>(), P64, c.as<double>(),
                                                            i, dpad);
      }
    }
    gs_normalize_kernel<<<1, 256, 0, s>>>(v.as<double>(), i, dpad, P64, PT.as<double>());
  }
  RBQ_CUDA(cudaGetLastError());
  to_f32_kernel<<<blocks_for(total, 256), 256, 0, s>>>(P64, total, P32);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

int kmeans_dev(const float* data, int64_t n, int32_t d, int32_t K, int32_t iters, int64_t sample,
               uint64_t seed, float* centroids, cudaStream_t s) {
  // training set: every point, or the Philox-sampled subset (ascending id)
  DevBuf train_buf, ids;
  const float* train = data;
  int64_t m = n;
  if (sample > 0 && sample < n) {
    DevBuf flags, pos;
    RBQ_CHECK(flags.alloc(sizeof(int32_t) * n, s));
    RBQ_CHECK(pos.alloc(sizeof(int32_t) * n, s));
    const uint32_t thr = (uint32_t)(((uint64_t)sample << 32) / (uint64_t)n);
    sample_flags_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, thr, seed, flags.as<int32_t>());
    RBQ_CHECK(exclusive_scan_i32(flags.as<int32_t>(), pos.as<int32_t>(), n, s));
    int32_t last[2];
    RBQ_CUDA(cudaMemcpyAsync(&last[0], pos.as<int32_t>() + n - 1, 4, cudaMemcpyDeviceToHost, s));
    RBQ_CUDA(cudaMemcpyAsync(&last[1], flags.as<int32_t>() + n - 1, 4, cudaMemcpyDeviceToHost, s));
    RBQ_CUDA(cudaStreamSynchronize(s));
    const int64_t ms = (int64_t)last[0] + last[1];
    if (ms >= K) {
      m = ms;
      RBQ_CHECK(ids.alloc(sizeof(int32_t) * m, s));
      compact_kernel<<<blocks_for(n, 256), 256, 0, s>>>(flags.as<int32_t>(), pos.as<int32_t>(), n,
                                                       ids.as<int32_t>());
      RBQ_CHECK(train_buf.alloc(sizeof(float) * m * d, s));
      RBQ_CHECK(gather_rows_f32(data, d, ids.as<int32_t>(), m, d, train_buf.as<float>(), s));
      train = train_buf.as<float>();
    }
  }
  DevBuf taken, init, ct, a, perm, off;
  RBQ_CHECK(taken.alloc(m, s));
  RBQ_CHECK(init.alloc(sizeof(int32_t) * K, s));
  RBQ_CUDA(cudaMemsetAsync(taken.p, 0, m, s));
  floyd_kernel<<<1, 32, 0, s>>>(m, K, seed, taken.as<uint8_t>(), init.as<int32_t>());
  RBQ_CUDA(cudaGetLastError());
  RBQ_CHECK(gather_rows_f32(train, d, init.as<int32_t>(), K, d, centroids, s));
  RBQ_CHECK(ct.alloc(sizeof(float) * K * d, s));
  RBQ_CHECK(a.alloc(sizeof(int32_t) * m, s));
  RBQ_CHECK(perm.alloc(sizeof(int32_t) * m, s));
  RBQ_CHECK(off.alloc(sizeof(int32_t) * (K + 1), s));
  for (int it = 0; it < iters; ++it) {
    RBQ_CHECK(transpose_f32(centroids, K, d, ct.as<float>(), s));
    RBQ_CHECK(argmin_sqdist(train, d, ct.as<float>(), K, m, K, d, a.as<int32_t>(), nullptr, s));
    RBQ_CHECK(counting_sort(a.as<int32_t>(), m, K, perm.as<int32_t>(), off.as<int32_t>(), s));
    kmeans_update_kernel<<<K, 128, 0, s>>>(train, d, perm.as<int32_t>(), off.as<int32_t>(),
                                          centroids);
    RBQ_CUDA(cudaGetLastError());
  }
  return RABITQ_OK;
}

int encode_dev(rabitq_index* X, const float* adist_b, cudaStream_t s) {
  const int64_t n = X->n;
  const int dpad = X->dpad, d = X->d;
  DevBuf cl, R;
  RBQ_CHECK(cl.alloc(sizeof(int32_t) * n, s));
  position_cluster_kernel<<<X->K, 128, 0, s>>>(X->bucket_off, cl.as<int32_t>());
  RBQ_CUDA(cudaGetLastError());
  int64_t chunk = (int64_t(1) << 28) / dpad;  // 1 GiB of FP32 R per chunk
  if (chunk > n) chunk = n;
  RBQ_CHECK(R.alloc(sizeof(float) * chunk * dpad, s));
  for (int64_t p0 = 0; p0 < n; p0 += chunk) {
    const int64_t m = std::min<int64_t>(chunk, n - p0);
    RBQ_CHECK(gemm_canon(kDot, X->data_b + p0 * d, d, nullptr, X->centroids, d,
                         cl.as<int32_t>() + p0, X->P32, dpad, R.as<float>(), dpad, m, dpad, d, s));
    encode_epilogue_kernel<<<blocks_for(m * 32, 256), 256, 0, s>>>(
        R.as<float>(), m, dpad, adist_b + p0, X->codes + p0 * X->W, X->factors + p0,
        X->metric != RABITQ_METRIC_L2 ? 1 : 0,
        X->data_b + p0 * d, X->centroids, cl.as<int32_t>() + p0, d);
    RBQ_CUDA(cudaGetLastError());
  }
  return RABITQ_OK;
}

int normalize_rows(const float* in, int64_t n, int32_t d, float* out, cudaStream_t s) {
  if (n <= 0) return RABITQ_OK;
  normalize_rows_kernel<<<blocks_for(n * 32, 256), 256, 0, s>>>(in, n, d, out);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

}  // namespace rbq
