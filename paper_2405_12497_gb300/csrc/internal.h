// internal.h -- host-side declarations shared by the library's translation
// units (index object, kernel launchers, error plumbing). Not installed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/rabitq.h"

struct rabitq_index {
  int64_t n = 0;
  int32_t d = 0, dpad = 0, K = 0, W = 0;  // W = dpad / 64 code words
  int device = 0;
  int32_t max_bucket = 0;
  // device arrays; "bucket order" = sorted by (cluster, id)
  float* data_b = nullptr;        // n x d raw vectors, bucket order
  uint64_t* codes = nullptr;      // n x W, bucket order
  float4* factors = nullptr;      // n: {F1, F2, F3, G}, bucket order
  int32_t* perm = nullptr;        // n: bucket position -> id
  int32_t* inv_perm = nullptr;    // n: id -> bucket position
  int32_t* bucket_off = nullptr;  // K + 1
  int32_t* assign = nullptr;      // n: cluster of id
  float* centroids = nullptr;     // K x d
  float* centroids_t = nullptr;   // d x K
  float* ptc = nullptr;           // K x dpad: P^T [c; 0]
  double* P64 = nullptr;          // dpad x dpad
  float* P32 = nullptr;           // dpad x dpad
  // P^T rows (one per code coordinate), K = d padded to kp, rounded to the
  // tensor-core operand types of the BF16 / TF32 query rotation
  int32_t kp = 0;
  int32_t tuned_path = 0;         // scan path AUTO uses (rabitq_autotune)
  void* ptb = nullptr;            // dpad x kp BF16
  float* ptf = nullptr;           // dpad x kp TF32-rounded FP32
};

namespace rbq {

// error plumbing (thread-local message)
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

#define RBQ_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return ::rbq::fail(RABITQ_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define RBQ_CHECK(status)     \
  do {                        \
    int s_ = (status);        \
    if (s_ != RABITQ_OK) return s_; \
  } while (0)

// Stream-ordered device scratch that frees itself.
struct DevBuf {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFreeAsync(p, s);
  }
  int alloc(size_t bytes, cudaStream_t st);
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

// ---- canonical SIMT "GEMM" (kernels_gemm.cu) ----------------------------
// C[m][n] = fold_k op(A'[m][k], B[k][n]) in ascending k, where
// A'[m][k] = A[arow(m)][k] - (sub ? sub[srow(m)][k] : 0); arow(m) = a_rows ? a_rows[m] : m.
enum GemmOp { kDot = 0, kSqDist = 1 };
int gemm_canon(GemmOp op, const float* A, int64_t lda, const int32_t* a_rows, const float* sub,
               int64_t ld_sub, const int32_t* sub_rows, const float* B, int64_t ldb, float* C,
               int64_t ldc, int64_t M, int N, int K, cudaStream_t s);
// argmin_n of squared distance rows (ties to the lower n): assign[m], dist[m]
int argmin_sqdist(const float* A, int64_t lda, const float* Bt, int64_t ldb, int64_t M, int N,
                  int K, int32_t* assign, float* dist, cudaStream_t s);

// ---- build (kernels_build.cu) -------------------------------------------
int exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s);
// stable counting sort of ids [0, n) by key (cluster); perm: position -> id
int counting_sort(const int32_t* key, int64_t n, int32_t K, int32_t* perm, int32_t* offsets,
                  cudaStream_t s);
int sample_rotation_dev(uint64_t seed, int32_t dpad, double* P64, float* P32, cudaStream_t s);
int kmeans_dev(const float* data, int64_t n, int32_t d, int32_t K, int32_t iters, int64_t sample,
               uint64_t seed, float* centroids, cudaStream_t s);
int encode_dev(rabitq_index* X, const float* adist_b, cudaStream_t s);
int gather_rows_f32(const float* in, int64_t ld, const int32_t* rows, int64_t m, int32_t d,
                    float* out, cudaStream_t s);
int invert_perm(const int32_t* perm, int64_t n, int32_t* inv, cudaStream_t s);
int transpose_f32(const float* in, int64_t rows, int64_t cols, float* out, cudaStream_t s);
int check_finite(const float* x, int64_t count, cudaStream_t s, bool* finite);

// ---- tensor-core query rotation (kernels_tc.cu) --------------------------
int pack_pt(rabitq_index* X, cudaStream_t s);
// out[M x dpad] = Q[M x d] P (mode RABITQ_ROT_BF16 or RABITQ_ROT_TF32);
// a bounded wait that expires sets *err = 2
int rotate_tc(const rabitq_index* X, const float* Q, int64_t M, int mode, float* out, int* err,
              cudaStream_t s);

// ---- search (kernels_search.cu) -----------------------------------------
struct SearchArgs {
  const rabitq_index* X;
  const float* queries;  // device, nq x d
  int64_t nq;
  int32_t k, nprobe, bq;
  float eps0;
  uint64_t seed;
  const int32_t* per_query_nprobe;  // device or null
  int32_t cand_cap;
  int64_t* out_ids;   // device
  float* out_dist;    // device
  const rabitq_trace* trace;  // device pointers or null
  int32_t rot_precision;
  int32_t scan_path;
  float* stage_ms;    // host, 5 entries or null
};
int search_dev(const SearchArgs& a, cudaStream_t s);
int search_dev_prealloc(const SearchArgs& a, unsigned char* scratch, size_t scratch_bytes,
                        cudaStream_t s);

}  // namespace rbq
