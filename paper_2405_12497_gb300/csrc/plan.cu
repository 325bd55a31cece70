// plan.cu -- search plans: a search of up to nq_max queries at fixed
// parameters whose device memory is allocated once and whose whole launch
// sequence (centroid distances, probe selection [, learned probe counts],
// rotation, longest-first order, fused scan/prune/re-rank) is replayed as
// one CUDA graph per batch size. No allocation, no host synchronization and
// no per-launch host work on the replay path: the graph launch is the only
// host call. Errors (candidate overflow, an expired tensor-core wait) are
// recorded in a device flag that rabitq_plan_sync reads and clears.
#include <map>
#include <mutex>
#include <string>

#include "internal.h"

using namespace rbq;

struct rabitq_plan {
  int device = 0;
  SearchArgs a{};             // parameters (queries/outputs point at the plan's buffers)
  int64_t nq_max = 0, grid = 0;
  size_t bytes = 0;
  unsigned char* scratch = nullptr;
  float* queries = nullptr;   // nq_max x d
  int64_t* ids = nullptr;     // nq_max x k
  float* dist = nullptr;      // nq_max x k
  int32_t* nprobe = nullptr;  // nq_max (learned probe counts) or null
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev[5] = {};     // stage events (collect_stats)
  bool stats = false;
  std::mutex mu;
  std::map<int64_t, cudaGraphExec_t> graphs;
};

namespace {

void destroy(rabitq_plan* P) {
  for (auto& kv : P->graphs) cudaGraphExecDestroy(kv.second);
  P->graphs.clear();
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
  for (auto& e : P->ev)
    if (e) cudaEventDestroy(e);
  cudaFree(P->scratch);
  cudaFree(P->queries);
  cudaFree(P->ids);
  cudaFree(P->dist);
  cudaFree(P->nprobe);
  delete P;
}

// The graph of a batch of nq queries (captured on first use).
int graph_for(rabitq_plan* P, int64_t nq, cudaGraphExec_t* out) {
  std::lock_guard<std::mutex> lock(P->mu);
  auto it = P->graphs.find(nq);
  if (it != P->graphs.end()) {
    *out = it->second;
    return RABITQ_OK;
  }
  SearchArgs a = P->a;
  a.nq = nq;
  RBQ_CUDA(cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal));
  const int st = search_enqueue_carved(a, P->scratch, P->bytes, P->grid, a.cand_cap,
                                       P->cap_stream);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(P->cap_stream, &g);
  if (st != RABITQ_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (ce != cudaSuccess)
    return fail(RABITQ_ECUDA, std::string("graph capture failed: ") + cudaGetErrorString(ce));
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess)
    return fail(RABITQ_ECUDA, std::string("graph instantiation failed: ") + cudaGetErrorString(ie));
  P->graphs[nq] = ex;
  *out = ex;
  return RABITQ_OK;
}

}  // namespace

extern "C" {

int rabitq_plan_create(const rabitq_index* X, const rabitq_predictor* pr, int64_t nq_max,
                       int32_t k, int32_t nprobe, int32_t bq, float eps0,
                       const rabitq_search_opts* opts_in, rabitq_plan** out) {
  set_error("");
  if (!out) return fail(RABITQ_EINVAL, "rabitq_plan_create: out is null");
  *out = nullptr;
  if (!X) return fail(RABITQ_EINVAL, "rabitq_plan_create: index is null");
  RBQ_CHECK(check_device(X->device, "rabitq_plan_create"));
  if (pr) RBQ_CHECK(check_device(pr->device, "rabitq_plan_create (predictor)"));
  rabitq_search_opts opts;
  rabitq_search_opts_default(&opts);
  if (opts_in) opts = *opts_in;
  if (opts.max_candidates == 0) opts.max_candidates = 65536;
  if (pr) {
    if (pr->K != X->K)
      return fail(RABITQ_EINVAL, "rabitq_plan_create: predictor made for another bucket count");
    if (X->metric != RABITQ_METRIC_L2)
      return fail(RABITQ_EUNSUPPORTED, "rabitq_plan_create: learned probe counts need a squared-distance (L2) index");
    nprobe = pr->nprobe_max;
  }
  if (nq_max < 1 || nq_max > (int64_t(1) << 24))
    return fail(RABITQ_EINVAL, "rabitq_plan_create: need 1 <= nq_max <= 2^24");
  if (k < 1 || k > 1024) return fail(RABITQ_EINVAL, "rabitq_plan_create: need 1 <= k <= 1024");
  if (nprobe < 1 || nprobe > X->K || nprobe > 16384)
    return fail(RABITQ_EINVAL, "rabitq_plan_create: need 1 <= nprobe <= min(K, 16384)");
  if (bq < 1 || bq > 8) return fail(RABITQ_EINVAL, "rabitq_plan_create: need 1 <= bq <= 8");
  if (!(eps0 >= 0.0f) || !(eps0 < __builtin_inff()))
    return fail(RABITQ_EINVAL, "rabitq_plan_create: eps0 must be finite and >= 0");
  if (opts.max_candidates < 4096 || opts.max_candidates > (1 << 26))
    return fail(RABITQ_EINVAL, "rabitq_plan_create: max_candidates must be in [4096, 2^26]");
  if (opts.rot_precision != RABITQ_ROT_FP32 && opts.rot_precision != RABITQ_ROT_TF32 &&
      opts.rot_precision != RABITQ_ROT_BF16)
    return fail(RABITQ_EINVAL, "rabitq_plan_create: unknown rot_precision");
  if (opts.per_query_nprobe)
    return fail(RABITQ_EUNSUPPORTED, "rabitq_plan_create: per_query_nprobe is not supported "
                                     "(use a predictor)");
  if (opts.scan_layout < RABITQ_LAYOUT_AUTO || opts.scan_layout > RABITQ_LAYOUT_WARP)
    return fail(RABITQ_EINVAL, "rabitq_plan_create: unknown scan_layout");
  if (opts.lane_pairs < 0 || opts.lane_pairs > 2)
    return fail(RABITQ_EINVAL, "rabitq_plan_create: lane_pairs must be 0, 1 or 2");
  if (opts.scan_staging < RABITQ_STAGING_AUTO || opts.scan_staging > RABITQ_STAGING_BULK)
    return fail(RABITQ_EINVAL, "rabitq_plan_create: unknown scan_staging");
  int dev = 0;
  RBQ_CUDA(cudaGetDevice(&dev));
  auto* P = new rabitq_plan();
  P->device = dev;
  SearchArgs& a = P->a;
  a.X = X;
  a.nq = nq_max;
  a.k = k;
  a.nprobe = nprobe;
  a.bq = bq;
  a.eps0 = eps0;
  a.seed = opts.quant_seed;
  a.per_query_nprobe = nullptr;
  a.cand_cap = opts.max_candidates;
  a.trace = nullptr;
  a.rot_precision = opts.rot_precision;
  a.scan_path = RABITQ_SCAN_POPC;
  a.layout = opts.scan_layout;
  a.ppl = opts.lane_pairs;
  a.stage = opts.scan_staging;
  // the plan keeps the tile resolved now (later tuning does not change it)
  a.tile_layout = a.layout;
  resolve_tile(X, k, nprobe, &a.scan_path, &a.tile_layout, &a.ppl, &a.stage);
  a.scan_path = RABITQ_SCAN_POPC;  // plans run the popcount scan
  a.stage_ms = nullptr;
  a.pred = pr;
  P->nq_max = nq_max;
  int grid = 0;
  int st = fused_grid(a, &grid);
  P->grid = grid;
  cudaError_t e = cudaSuccess;
  if (st == RABITQ_OK) {
    P->bytes = carved_bytes(a, P->grid, nq_max);
    e = cudaMalloc(reinterpret_cast<void**>(&P->scratch), P->bytes);
    if (e == cudaSuccess)
      e = cudaMalloc(reinterpret_cast<void**>(&P->queries), sizeof(float) * nq_max * X->d);
    if (e == cudaSuccess)
      e = cudaMalloc(reinterpret_cast<void**>(&P->ids), sizeof(int64_t) * nq_max * k);
    if (e == cudaSuccess)
      e = cudaMalloc(reinterpret_cast<void**>(&P->dist), sizeof(float) * nq_max * k);
    if (e == cudaSuccess && pr)
      e = cudaMalloc(reinterpret_cast<void**>(&P->nprobe), sizeof(int32_t) * nq_max);
    if (e == cudaSuccess) e = cudaMemset(P->scratch, 0, 256);  // the error flag
    if (e == cudaSuccess) e = cudaMemset(P->queries, 0, sizeof(float) * nq_max * X->d);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking);
    if (opts.collect_stats)
      for (auto& ev : P->ev)
        if (e == cudaSuccess) e = cudaEventCreate(&ev);
    if (e != cudaSuccess)
      st = fail(RABITQ_ENOMEM, std::string("rabitq_plan_create: ") + cudaGetErrorString(e));
  }
  if (st != RABITQ_OK) {
    destroy(P);
    return st;
  }
  a.queries = P->queries;
  a.out_ids = P->ids;
  a.out_dist = P->dist;
  a.pred_nprobe = P->nprobe;
  P->stats = opts.collect_stats != 0;
  a.stage_ev = P->stats ? P->ev : nullptr;
  *out = P;
  return RABITQ_OK;
}

int rabitq_plan_buffers(const rabitq_plan* P, float** queries, int64_t** ids, float** dist,
                        int32_t** nprobe) {
  if (!P) return fail(RABITQ_EINVAL, "rabitq_plan_buffers: plan is null");
  if (queries) *queries = P->queries;
  if (ids) *ids = P->ids;
  if (dist) *dist = P->dist;
  if (nprobe) *nprobe = P->nprobe;
  return RABITQ_OK;
}

int rabitq_plan_run(rabitq_plan* P, int64_t nq, void* stream) {
  set_error("");
  if (!P) return fail(RABITQ_EINVAL, "rabitq_plan_run: plan is null");
  if (nq < 0 || nq > P->nq_max) return fail(RABITQ_EINVAL, "rabitq_plan_run: need 0 <= nq <= nq_max");
  RBQ_CHECK(check_device(P->device, "rabitq_plan_run"));
  if (nq == 0) return RABITQ_OK;
  cudaGraphExec_t ex = nullptr;
  RBQ_CHECK(graph_for(P, nq, &ex));
  RBQ_CUDA(cudaGraphLaunch(ex, static_cast<cudaStream_t>(stream)));
  return RABITQ_OK;
}

int rabitq_plan_sync(rabitq_plan* P, void* stream) {
  if (!P) return fail(RABITQ_EINVAL, "rabitq_plan_sync: plan is null");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int h_err = 0;
  RBQ_CUDA(cudaMemcpyAsync(&h_err, P->scratch, sizeof(int), cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaMemsetAsync(P->scratch, 0, sizeof(int), s));
  RBQ_CUDA(cudaStreamSynchronize(s));
  if (h_err == 2) return fail(RABITQ_ETIMEOUT, "a tensor-core wait expired (probe scores or query rotation)");
  if (h_err)
    return fail(RABITQ_EOVERFLOW,
                "a query's candidate list exceeded max_candidates; raise max_candidates");
  return RABITQ_OK;
}

int rabitq_plan_search(rabitq_plan* P, const float* queries, int64_t nq, int64_t* out_ids,
                       float* out_dist, void* stream) {
  set_error("");
  if (!P) return fail(RABITQ_EINVAL, "rabitq_plan_search: plan is null");
  if (nq < 0 || nq > P->nq_max)
    return fail(RABITQ_EINVAL, "rabitq_plan_search: need 0 <= nq <= nq_max");
  if (nq == 0) return RABITQ_OK;
  if (!queries || !out_ids || !out_dist) return fail(RABITQ_EINVAL, "rabitq_plan_search: null pointer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int d = P->a.X->d, k = P->a.k;
  if (queries != P->queries)
    RBQ_CUDA(cudaMemcpyAsync(P->queries, queries, sizeof(float) * nq * d, cudaMemcpyDefault, s));
  RBQ_CHECK(rabitq_plan_run(P, nq, stream));
  if (out_ids != P->ids)
    RBQ_CUDA(cudaMemcpyAsync(out_ids, P->ids, sizeof(int64_t) * nq * k, cudaMemcpyDefault, s));
  if (out_dist != P->dist)
    RBQ_CUDA(cudaMemcpyAsync(out_dist, P->dist, sizeof(float) * nq * k, cudaMemcpyDefault, s));
  return rabitq_plan_sync(P, stream);
}

int rabitq_plan_tile(const rabitq_plan* P, rabitq_tile* out) {
  if (!P || !out) return fail(RABITQ_EINVAL, "rabitq_plan_tile: null argument");
  out->scan_path = RABITQ_SCAN_POPC;
  const rabitq_index* X = P->a.X;
  const bool warp = P->a.tile_layout == RABITQ_LAYOUT_WARP && P->a.bq == 4 && P->a.k <= 128 &&
                    X->d <= 256 && (X->W == 2 || X->W == 4);
  out->scan_layout = warp ? RABITQ_LAYOUT_WARP : RABITQ_LAYOUT_CTA;
  out->lane_pairs = warp ? (P->a.ppl ? P->a.ppl : (X->W == 2 ? 2 : 1)) : 0;
  out->staging = !warp && P->a.stage == RABITQ_STAGING_BULK && P->a.bq == 4 &&
                         (X->W == 2 || X->W == 4)
                     ? RABITQ_STAGING_BULK
                     : RABITQ_STAGING_OFF;
  out->time_ms = 0.0f;
  return RABITQ_OK;
}

int rabitq_plan_stats(rabitq_plan* P, float* ms, int32_t cap) {
  if (!P || !ms || cap < 0) return fail(RABITQ_EINVAL, "rabitq_plan_stats: null argument");
  if (!P->stats) return 0;
  RBQ_CUDA(cudaEventSynchronize(P->ev[4]));
  const int m = cap < 4 ? cap : 4;
  for (int i = 0; i < m; ++i) RBQ_CUDA(cudaEventElapsedTime(&ms[i], P->ev[i], P->ev[i + 1]));
  return m;
}

void rabitq_plan_free(rabitq_plan* P) {
  if (!P) return;
  cudaDeviceSynchronize();
  destroy(P);
}

}  // extern "C"
