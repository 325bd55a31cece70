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
  int32_t metric = 0;                     // RABITQ_METRIC_*
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
  int32_t tuned_layout = 0;       // scan layout AUTO uses (rabitq_autotune), 0 = default
  // tiles chosen by rabitq_autotune_tiles per (k class, nprobe class)
  // (path: the fastest overall; layout, ppl: the fastest popcount tile,
  // which plans run)
  struct Tile {
    int32_t valid, path, layout, ppl, stage;
  } tune[4][4] = {};
  void* ptb = nullptr;            // dpad x kp BF16
  float* ptf = nullptr;           // dpad x kp TF32-rounded FP32
  // centroids for the tensor-core probe scores: TF32-rounded, stored in
  // tiles of 256 rows (centroid_tile_rows(K) x kp, zero padding), each a run
  // of 32-column stages in the core-matrix layout; and the FP32 norms
  // ||c||^2 (canonical fold) and ||c||
  float* ctf = nullptr;
  float* cn2 = nullptr;
  float* cnorm = nullptr;
  float* cnorm_max = nullptr;  // max ||c|| (one value)
};

// Learned probe-count predictor (kernels_mlp.cu): MLP weights with BF16
// values, the feature scale s0 and the calibrated multiplier.
struct rabitq_predictor {
  int device = 0;
  int32_t K = 0;           // bucket count of the index it was trained on
  int32_t k = 0;           // neighbours per query its labels cover
  int32_t nprobe_max = 0;  // largest probe count it predicts
  float target_recall = 0, s0 = 0, mult = 1;
  float train_loss = 0, val_loss = 0, val_recall = 0, val_mean_nprobe = 0;
  int64_t n_train = 0, n_val = 0;
  float* params = nullptr;  // RABITQ_MLP_PARAMS, BF16 values stored as FP32
  void* params_bf16 = nullptr;  // the same values packed as BF16 (inference)
};

namespace rbq {

// error plumbing (thread-local message)
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
// EINVAL (message names `who`) unless the calling thread's current device is
// `device`, the device an index, predictor or plan lives on: its arrays are
// device pointers of that GPU only.
int check_device(int device, const char* who);

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

// N timing events, destroyed on every return path (create() may be skipped
// when no timing is asked for).
template <int N>
struct EventSet {
  cudaEvent_t e[N] = {};
  EventSet() = default;
  EventSet(const EventSet&) = delete;
  EventSet& operator=(const EventSet&) = delete;
  ~EventSet() {
    for (auto& x : e)
      if (x) cudaEventDestroy(x);
  }
  int create() {
    for (auto& x : e) RBQ_CUDA(cudaEventCreate(&x));
    return RABITQ_OK;
  }
  cudaEvent_t& operator[](int i) { return e[i]; }
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
// the same with caller-provided scratch of counting_sort_ws_ints(n, K) ints
// (no allocation, so it can be captured in a CUDA graph)
int64_t counting_sort_ws_ints(int64_t n, int32_t K);
// Ids [0, n) grouped by key, the order within a key unspecified (a work
// order): one block when n <= 65536 and K <= 8192, else counting_sort_ws
// with the caller's scratch ws (counting_sort_ws_ints(n, K) ints, unused by
// the one-block sort).
int order_sort(const int32_t* key, int64_t n, int32_t K, int32_t* perm, int32_t* offsets,
               int32_t* ws, cudaStream_t s);
bool order_sort_fits(int64_t n, int32_t K);
int counting_sort_ws(const int32_t* key, int64_t n, int32_t K, int32_t* perm, int32_t* offsets,
                     int32_t* ws, cudaStream_t s);
int sample_rotation_dev(uint64_t seed, int32_t dpad, double* P64, float* P32, cudaStream_t s);
int kmeans_dev(const float* data, int64_t n, int32_t d, int32_t K, int32_t iters, int64_t sample,
               uint64_t seed, float* centroids, cudaStream_t s);
int encode_dev(rabitq_index* X, const float* adist_b, cudaStream_t s);
// unit rows (canonical FP32 norm, zero rows unchanged); in and out distinct
int normalize_rows(const float* in, int64_t n, int32_t d, float* out, cudaStream_t s);
int gather_rows_f32(const float* in, int64_t ld, const int32_t* rows, int64_t m, int32_t d,
                    float* out, cudaStream_t s);
int invert_perm(const int32_t* perm, int64_t n, int32_t* inv, cudaStream_t s);
int transpose_f32(const float* in, int64_t rows, int64_t cols, float* out, cudaStream_t s);
int check_finite(const float* x, int64_t count, cudaStream_t s, bool* finite);
// sets *flag (device, zeroed by the caller) to 1 if x has a non-finite value;
// no synchronization
int finite_flag(const float* x, int64_t count, int* flag, cudaStream_t s);

// ---- tensor-core query rotation (kernels_tc.cu) --------------------------
int pack_pt(rabitq_index* X, cudaStream_t s);
// TF32 centroid rows and their norms (after the centroids are final)
int pack_centroids(rabitq_index* X, cudaStream_t s);
// Probe filter keys of M queries against all K centroids (tensor cores,
// TF32 operands, FP32 accumulation): keys[m][c] = the order-preserving key
// of U_c = approximate score + eps_c, with each query's key range and
// FP32 ||q||^2; *err = 2 when a bounded wait expired. The scratch holds
// probe_scratch_floats(X, M) floats, viewed by probe_scratch().
constexpr int kProbePool = 8;  // smallest keys pooled per query and 128 centroids
struct ProbeScratch {
  uint32_t* keys;   // M x K
  float* qt;        // the queries' TF32 tiles
  float* nq2;       // M
  uint32_t* kmin;   // M: smallest key
  uint32_t* kmax;   // M: largest key
  // M x pool_n: the kProbePool smallest entries of each 128 centroids,
  // ascending: the key rounded up to a multiple of 128 | the centroid's index
  // among the 128 (0xffffffff past the last centroid)
  uint32_t* pool;
  int pool_n;       // kProbePool x (K / 128, rounded up to whole tiles of 256)
  size_t floats;    // total size
};
ProbeScratch probe_scratch(const rabitq_index* X, int64_t nq, float* base);
size_t probe_scratch_floats(const rabitq_index* X, int64_t nq);
// runs the bounded-wait self-test kernel; *status_host gets its result bits
int wait_selftest(uint32_t polls, int* status_host);
int probe_keys_tc(const rabitq_index* X, const float* Q, int64_t M, float* scratch, int* err,
                  cudaStream_t s);
// rows of the index's tiled TF32 centroid array (K padded to whole tiles)
int64_t centroid_tile_rows(int K);
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
  // learned probe counts: the predictor sets each query's probe count (at
  // most nprobe) from its centroid distances; pred_nprobe (device, nq) keeps
  // them. Null for a fixed or caller-given probe count.
  const rabitq_predictor* pred = nullptr;
  int32_t* pred_nprobe = nullptr;
  // carved path only: 5 events recorded (as external graph nodes when
  // captured) around the stages: distances | selection (+ MLP) | rotation |
  // fused scan, prune and re-rank. Single-chunk searches only.
  cudaEvent_t* stage_ev = nullptr;
  // a batch too small to fill the GPU may split each query's probes over
  // several CTAs and merge them (identical results); off where scratch is fixed
  int allow_split = 1;
  // work layout of the popcount scan (RABITQ_LAYOUT_*); the warp-per-query
  // kernel also needs allow_warp (off where the scratch is fixed)
  int32_t layout = 0;
  int allow_warp = 1;
  int32_t ppl = 0;  // codes per lane per step in the warp layout (0 = default)
  // the layout AUTO resolves to (resolve_tile; set by search_dev and plans):
  // taken for batches that fill the GPU, while an explicit RABITQ_LAYOUT_WARP
  // request is taken for every batch
  int32_t tile_layout = 0;
  // bulk-copy staging of the CTA layout's scan rounds (RABITQ_STAGING_*;
  // AUTO resolves to the tuned or default choice)
  int32_t stage = 0;
};
// Resolve the AUTO choices of a search (scan path, layout, codes per lane)
// from the index's tuned tiles for the shape's class, else the defaults.
void resolve_tile(const rabitq_index* X, int k, int nprobe, int32_t* path, int32_t* layout,
                  int32_t* ppl, int32_t* stage);
int tile_class_k(int k);
int tile_class_np(int nprobe);
int search_dev(const SearchArgs& a, cudaStream_t s);
// Probe counts of nq queries from a predictor: query-centroid distances, the
// 64 smallest, features, MLP, multiplier. feat (nq x 64) and y (nq) optional.
int predict_dev(const rabitq_index* X, const rabitq_predictor* pr, const float* Q, int64_t nq,
                int32_t* nprobe_out, float* feat, float* y, cudaStream_t s);
// Top-nsel buckets of each query (ascending (distance, id)), for nq queries.
int select_buckets(const rabitq_index* X, const float* Q, int64_t nq, int nsel, int32_t* ids,
                   float* dist, cudaStream_t s);
int search_dev_prealloc(const SearchArgs& a, unsigned char* scratch, size_t scratch_bytes,
                        cudaStream_t s);
// Single-code estimates (§3.3.2, first case): out nq x m x 3; *err (device,
// zeroed by the caller) is set for an id outside [-1, n).
int estimate_dev(const rabitq_index* X, const float* Q, int64_t nq, const int64_t* ids, int m,
                 int bq, float eps0, uint64_t seed, int rot_precision, float* out, int* err,
                 cudaStream_t s);
// The allocation-free, synchronization-free launch sequence of the popcount
// search (capturable in a CUDA graph). The scratch's first int is the error
// flag (1 = candidate overflow, 2 = tensor-core wait expired), which this call
// sets but never clears.
int search_enqueue_carved(const SearchArgs& a, unsigned char* scratch, size_t scratch_bytes,
                          int64_t grid, int64_t cap, cudaStream_t s);
// scratch bytes for nq_max queries in one chunk with a.cand_cap candidates per CTA
size_t carved_bytes(const SearchArgs& a, int64_t grid, int64_t nq_max);
// CTAs of the fused kernel at full residency for these search parameters
int fused_grid(const SearchArgs& a, int* grid_out);

// ---- learned probe count (kernels_mlp.cu) ---------------------------------
constexpr int kMlpIn = RABITQ_MLP_IN, kMlpHidden = RABITQ_MLP_HIDDEN;
constexpr int kMlpParams = RABITQ_MLP_PARAMS;
struct MlpWork {  // activations and gradients of one batch
  DevBuf buf;
  float *Z1, *H1, *Z2, *H2, *dH2, *dH1, *y, *dy, *se, *T, *W2T;
  int alloc(int64_t B, cudaStream_t s);
};
int mlp_forward(const float* params, const float* X, int64_t B, float* Z1, float* H1, float* Z2,
                float* H2, float* y, cudaStream_t s);
int mlp_backward(const float* params, const float* X, const float* t, int64_t B, float* grads,
                 MlpWork& w, cudaStream_t s);
int mlp_adam(float* master, float* work, const float* g, float* m1, float* m2, float lr, int step,
             cudaStream_t s);
// features from each query's ascending centroid distances (row stride ld,
// navail = min(64, K) valid entries)
int mlp_features(const float* sel_dist, int64_t ld, int64_t nq, int navail, float s0, float* X,
                 cudaStream_t s);
// fused inference: features, MLP and probe counts in one kernel
int mlp_infer(const rabitq_predictor* pr, const float* sel_dist, int64_t ld, int64_t nq,
              int navail, int32_t* nprobe_out, float* feat, float* y, cudaStream_t s);
// in = out allowed; packed (BF16) may be null
int mlp_round(const float* in, float* out, void* packed, int n, cudaStream_t s);
// neighbours a label must cover: ceil(target k), with a tolerance of 1e-6 k
// for the float target (0.95f * 100 is 94.9999988...)
inline int mlp_need(float target, int k) {
  const double v = (double)target * k - 1e-6 * k;
  int need = (int)v;
  if ((double)need < v) ++need;
  return need < 1 ? 1 : (need > k ? k : need);
}
int predictor_train_dev(const rabitq_index* X, const float* Q, int64_t nt,
                        const int64_t* gt, const rabitq_predictor_opts& o, rabitq_predictor* pr,
                        cudaStream_t s);
int mlp_labels_dev(const rabitq_index* X, const float* Q, int64_t nq, const int64_t* gt, int k,
                   int need, int nmax, int32_t* ranks, int32_t* label_r, cudaStream_t s);
int mlp_pack_bf16(rabitq_predictor* pr, cudaStream_t s);
// sum of (y - t)^2 over n rows in FP64, fixed order (one value at out, device)
int mlp_sum_sq_err(const float* y, const float* t, int64_t n, double* out, cudaStream_t s);

}  // namespace rbq
