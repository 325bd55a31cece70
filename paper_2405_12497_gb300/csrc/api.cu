// api.cu -- the C-ABI entry points of include/rabitq.h: argument checks,
// device memory of the index, host<->device copies, stream handling, stats,
// accessors and the index file format.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace rbq {

namespace {
thread_local std::string g_err;
thread_local float g_stats[5] = {0, 0, 0, 0, 0};
thread_local int g_nstats = 0;
}  // namespace

void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int check_device(int device, const char* who) {
  int cur = 0;
  RBQ_CUDA(cudaGetDevice(&cur));
  if (cur != device)
    return fail(RABITQ_EINVAL, std::string(who) + ": the current device (" + std::to_string(cur) +
                                   ") is not the device the index lives on (" +
                                   std::to_string(device) + ")");
  return RABITQ_OK;
}

namespace {

template <class T>
int dev_alloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(RABITQ_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  return RABITQ_OK;
}

void free_index_arrays(rabitq_index* X) {
  cudaFree(X->data_b);
  cudaFree(X->codes);
  cudaFree(X->factors);
  cudaFree(X->perm);
  cudaFree(X->inv_perm);
  cudaFree(X->bucket_off);
  cudaFree(X->assign);
  cudaFree(X->centroids);
  cudaFree(X->centroids_t);
  cudaFree(X->ptc);
  cudaFree(X->P64);
  cudaFree(X->P32);
  cudaFree(X->ptb);
  cudaFree(X->ptf);
  cudaFree(X->ctf);
  cudaFree(X->cn2);
  cudaFree(X->cnorm);
  cudaFree(X->cnorm_max);
}

int alloc_index_arrays(rabitq_index* X) {
  const int64_t n = X->n;
  RBQ_CHECK(dev_alloc(&X->data_b, (size_t)n * X->d));
  RBQ_CHECK(dev_alloc(&X->codes, (size_t)n * X->W));
  RBQ_CHECK(dev_alloc(&X->factors, (size_t)n));
  RBQ_CHECK(dev_alloc(&X->perm, (size_t)n));
  RBQ_CHECK(dev_alloc(&X->inv_perm, (size_t)n));
  RBQ_CHECK(dev_alloc(&X->bucket_off, (size_t)X->K + 1));
  RBQ_CHECK(dev_alloc(&X->assign, (size_t)n));
  RBQ_CHECK(dev_alloc(&X->centroids, (size_t)X->K * X->d));
  RBQ_CHECK(dev_alloc(&X->centroids_t, (size_t)X->K * X->d));
  RBQ_CHECK(dev_alloc(&X->ptc, (size_t)X->K * X->dpad));
  RBQ_CHECK(dev_alloc(&X->P64, (size_t)X->dpad * X->dpad));
  RBQ_CHECK(dev_alloc(&X->P32, (size_t)X->dpad * X->dpad));
  X->kp = (X->d + 63) / 64 * 64;
  RBQ_CHECK(dev_alloc(reinterpret_cast<uint16_t**>(&X->ptb), (size_t)X->dpad * X->kp));
  RBQ_CHECK(dev_alloc(&X->ptf, (size_t)X->dpad * X->kp));
  RBQ_CHECK(dev_alloc(&X->ctf, (size_t)centroid_tile_rows(X->K) * X->kp));
  RBQ_CHECK(dev_alloc(&X->cn2, (size_t)X->K));
  RBQ_CHECK(dev_alloc(&X->cnorm, (size_t)X->K));
  RBQ_CHECK(dev_alloc(&X->cnorm_max, 1));
  return RABITQ_OK;
}

int max_bucket_size(rabitq_index* X, cudaStream_t s) {
  std::vector<int32_t> off(X->K + 1);
  RBQ_CUDA(cudaMemcpyAsync(off.data(), X->bucket_off, sizeof(int32_t) * (X->K + 1),
                           cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaStreamSynchronize(s));
  int mx = 0;
  for (int c = 0; c < X->K; ++c) mx = std::max(mx, off[c + 1] - off[c]);
  X->max_bucket = mx;
  return RABITQ_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---- CRC-32 (IEEE 802.3, reflected polynomial 0xEDB88320) for index files
uint32_t crc32_update(uint32_t crc, const void* data, size_t len) {
  static uint32_t table[256];
  static bool init = false;
  if (!init) {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t c = i;
      for (int k = 0; k < 8; ++k) c = (c & 1) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
      table[i] = c;
    }
    init = true;
  }
  const uint8_t* p = static_cast<const uint8_t*>(data);
  crc = ~crc;
  for (size_t i = 0; i < len; ++i) crc = table[(crc ^ p[i]) & 0xff] ^ (crc >> 8);
  return ~crc;
}

struct FileHeader {
  char magic[8];  // "RABITQ\0\1"
  uint32_t version;
  uint32_t metric;  // RABITQ_METRIC_* (0, the squared distance, in older files)
  int64_t n;
  int32_t d, dpad, K, W;
  uint64_t payload_bytes;
  uint32_t payload_crc;
  uint32_t header_crc;
};

}  // namespace
}  // namespace rbq

using namespace rbq;

extern "C" {

void rabitq_build_opts_default(rabitq_build_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->kmeans_iters = 10;
}

void rabitq_search_opts_default(rabitq_search_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->quant_seed = 3;
  o->max_candidates = 65536;
}

const char* rabitq_last_error(void) { return g_err.c_str(); }

int rabitq_selftest_wait(uint32_t polls) {
  g_err.clear();
  if (polls == 0) return fail(RABITQ_EINVAL, "rabitq_selftest_wait: polls must be positive");
  int status = 0;
  RBQ_CHECK(wait_selftest(polls, &status));
  if (status != 3)
    return fail(RABITQ_EIO, "rabitq_selftest_wait: a bounded wait did not give up (status " +
                                std::to_string(status) + ")");
  return RABITQ_OK;
}

int rabitq_last_stats(float* ms, int32_t cap) {
  if (!ms || cap < 0) return fail(RABITQ_EINVAL, "rabitq_last_stats: null output");
  const int m = std::min<int>(cap, g_nstats);
  for (int i = 0; i < m; ++i) ms[i] = g_stats[i];
  return m;
}

int rabitq_build(const float* data, int64_t n, int32_t d, int32_t n_clusters, uint64_t seed,
                 const rabitq_build_opts* opts_in, rabitq_index** out) {
  g_err.clear();
  if (!out) return fail(RABITQ_EINVAL, "rabitq_build: out is null");
  *out = nullptr;
  rabitq_build_opts opts;
  rabitq_build_opts_default(&opts);
  if (opts_in) opts = *opts_in;
  if (!data) return fail(RABITQ_EINVAL, "rabitq_build: data is null");
  if (n < 1 || n > 0x7fffffffLL) return fail(RABITQ_EINVAL, "rabitq_build: need 1 <= n < 2^31");
  if (d < 1 || d > 4096) return fail(RABITQ_EINVAL, "rabitq_build: need 1 <= d <= 4096");
  if (n_clusters < 1 || n_clusters > n || n_clusters > 65536)
    return fail(RABITQ_EINVAL, "rabitq_build: need 1 <= n_clusters <= min(n, 65536)");
  if (opts.kmeans_iters < 0) return fail(RABITQ_EINVAL, "rabitq_build: kmeans_iters < 0");
  if (opts.metric != RABITQ_METRIC_L2 && opts.metric != RABITQ_METRIC_IP &&
      opts.metric != RABITQ_METRIC_COSINE)
    return fail(RABITQ_EINVAL, "rabitq_build: unknown metric");
  int32_t dpad = opts.code_bits ? opts.code_bits : (d + 63) / 64 * 64;
  if (dpad % 64 != 0 || dpad < d || dpad > 4096)
    return fail(RABITQ_EINVAL, "rabitq_build: code_bits must be a multiple of 64, >= d, <= 4096");
  if (int64_t(n_clusters) * (n + 2047) / 2048 > (int64_t(1) << 31))
    return fail(RABITQ_EINVAL, "rabitq_build: n_clusters too large for n");
  cudaStream_t s = static_cast<cudaStream_t>(opts.stream);

  int dev = 0;
  RBQ_CUDA(cudaGetDevice(&dev));
  auto* X = new rabitq_index();
  X->device = dev;
  X->n = n;
  X->d = d;
  X->dpad = dpad;
  X->K = n_clusters;
  X->W = dpad / 64;
  X->metric = opts.metric;
  int st = alloc_index_arrays(X);
  if (st != RABITQ_OK) {
    free_index_arrays(X);
    delete X;
    return st;
  }
  auto body = [&]() -> int {
    DevBuf dbuf, adist, adist_b, unit;
    const float* ddata = data;
    if (!opts.data_on_device) {
      RBQ_CHECK(dbuf.alloc(sizeof(float) * n * d, s));
      RBQ_CUDA(cudaMemcpyAsync(dbuf.p, data, sizeof(float) * n * d, cudaMemcpyHostToDevice, s));
      ddata = dbuf.as<float>();
    }
    bool finite = true;
    RBQ_CHECK(check_finite(ddata, n * d, s, &finite));
    if (!finite) return fail(RABITQ_EINVAL, "rabitq_build: data has a non-finite value");
    if (opts.metric == RABITQ_METRIC_COSINE) {  // the index holds unit vectors
      RBQ_CHECK(unit.alloc(sizeof(float) * n * d, s));
      RBQ_CHECK(normalize_rows(ddata, n, d, unit.as<float>(), s));
      ddata = unit.as<float>();
    }
    if (opts.centroids) {
      RBQ_CUDA(cudaMemcpyAsync(X->centroids, opts.centroids, sizeof(float) * n_clusters * d,
                               opts.data_on_device ? cudaMemcpyDeviceToDevice
                                                   : cudaMemcpyHostToDevice,
                               s));
      RBQ_CHECK(check_finite(X->centroids, (int64_t)n_clusters * d, s, &finite));
      if (!finite) return fail(RABITQ_EINVAL, "rabitq_build: centroids have a non-finite value");
    } else {
      RBQ_CHECK(kmeans_dev(ddata, n, d, n_clusters, opts.kmeans_iters, opts.kmeans_sample, seed,
                           X->centroids, s));
    }
    RBQ_CHECK(transpose_f32(X->centroids, n_clusters, d, X->centroids_t, s));
    RBQ_CHECK(pack_centroids(X, s));
    RBQ_CHECK(adist.alloc(sizeof(float) * n, s));
    RBQ_CHECK(argmin_sqdist(ddata, d, X->centroids_t, n_clusters, n, n_clusters, d, X->assign,
                            adist.as<float>(), s));
    RBQ_CHECK(counting_sort(X->assign, n, n_clusters, X->perm, X->bucket_off, s));
    RBQ_CHECK(invert_perm(X->perm, n, X->inv_perm, s));
    RBQ_CHECK(gather_rows_f32(ddata, d, X->perm, n, d, X->data_b, s));
    RBQ_CHECK(adist_b.alloc(sizeof(float) * n, s));
    RBQ_CHECK(gather_rows_f32(adist.as<float>(), 1, X->perm, n, 1, adist_b.as<float>(), s));
    RBQ_CHECK(sample_rotation_dev(seed, dpad, X->P64, X->P32, s));
    RBQ_CHECK(pack_pt(X, s));
    RBQ_CHECK(gemm_canon(kDot, X->centroids, d, nullptr, nullptr, 0, nullptr, X->P32, dpad,
                         X->ptc, dpad, n_clusters, dpad, d, s));
    RBQ_CHECK(encode_dev(X, adist_b.as<float>(), s));
    RBQ_CHECK(max_bucket_size(X, s));
    RBQ_CUDA(cudaStreamSynchronize(s));
    return RABITQ_OK;
  };
  st = body();
  if (st != RABITQ_OK) {
    cudaStreamSynchronize(s);
    free_index_arrays(X);
    delete X;
    return st;
  }
  *out = X;
  return RABITQ_OK;
}

static int search_common(const rabitq_index* X, const float* queries, int64_t nq, int32_t k,
                         int32_t nprobe, int32_t bq, float eps0, int64_t* out_ids,
                         float* out_dist, const rabitq_search_opts* opts_in,
                         const rabitq_trace* trace, const rabitq_predictor* pr = nullptr) {
  g_err.clear();
  g_nstats = 0;
  if (!X) return fail(RABITQ_EINVAL, "rabitq_search: index is null");
  RBQ_CHECK(check_device(X->device, "rabitq_search"));
  rabitq_search_opts opts;
  rabitq_search_opts_default(&opts);
  if (opts_in) opts = *opts_in;
  if (opts.max_candidates == 0) opts.max_candidates = 65536;
  if (nq < 0) return fail(RABITQ_EINVAL, "rabitq_search: nq < 0");
  if (nq == 0) return RABITQ_OK;
  if (!queries || !out_ids || !out_dist) return fail(RABITQ_EINVAL, "rabitq_search: null pointer");
  if (k < 1 || k > 1024) return fail(RABITQ_EINVAL, "rabitq_search: need 1 <= k <= 1024");
  if (nprobe < 1 || nprobe > X->K || nprobe > 16384)
    return fail(RABITQ_EINVAL, "rabitq_search: need 1 <= nprobe <= min(K, 16384)");
  if (bq < 1 || bq > 8) return fail(RABITQ_EINVAL, "rabitq_search: need 1 <= bq <= 8");
  if (!(eps0 >= 0.0f) || !std::isfinite(eps0))
    return fail(RABITQ_EINVAL, "rabitq_search: eps0 must be finite and >= 0");
  if (opts.max_candidates < 4096 || opts.max_candidates > (1 << 26))
    return fail(RABITQ_EINVAL, "rabitq_search: max_candidates must be in [4096, 2^26]");
  if (opts.rot_precision != RABITQ_ROT_FP32 && opts.rot_precision != RABITQ_ROT_TF32 &&
      opts.rot_precision != RABITQ_ROT_BF16)
    return fail(RABITQ_EINVAL, "rabitq_search: unknown rot_precision");
  if (opts.scan_path != RABITQ_SCAN_AUTO && opts.scan_path != RABITQ_SCAN_POPC &&
      opts.scan_path != RABITQ_SCAN_TC)
    return fail(RABITQ_EINVAL, "rabitq_search: unknown scan_path");
  if (opts.scan_layout < RABITQ_LAYOUT_AUTO || opts.scan_layout > RABITQ_LAYOUT_WARP)
    return fail(RABITQ_EINVAL, "rabitq_search: unknown scan_layout");
  if (opts.lane_pairs < 0 || opts.lane_pairs > 2)
    return fail(RABITQ_EINVAL, "rabitq_search: lane_pairs must be 0, 1 or 2");
  if (opts.scan_staging < RABITQ_STAGING_AUTO || opts.scan_staging > RABITQ_STAGING_BULK)
    return fail(RABITQ_EINVAL, "rabitq_search: unknown scan_staging");
  if (trace && opts.scan_path != RABITQ_SCAN_POPC &&
      (trace->planes || trace->sum_qu || trace->meta || trace->pair_id))
    opts.scan_path = RABITQ_SCAN_POPC;  // bit-planes and per-pair values come from that path
  if (trace && (trace->pair_id || trace->pair_ip || trace->pair_est) &&
      (!trace->pair_id || !trace->pair_ip || !trace->pair_est || trace->pair_cap < 0))
    return fail(RABITQ_EINVAL, "rabitq_search_trace: pair arrays must be given together");
  if (trace && trace->surv_ids && trace->surv_cap < 0)
    return fail(RABITQ_EINVAL, "rabitq_search_trace: surv_cap < 0");
  cudaStream_t s = static_cast<cudaStream_t>(opts.stream);
  const bool on_dev = trace ? true : opts.io_on_device != 0;

  EventSet<2> ev;  // t0, t1 of the whole search (stats)
  if (opts.collect_stats) {
    RBQ_CHECK(ev.create());
    RBQ_CUDA(cudaEventRecord(ev[0], s));
  }
  DevBuf qb, ib, db, nb, pb;
  const float* dq = queries;
  int64_t* dids = out_ids;
  float* ddist = out_dist;
  const int32_t* dnp = opts.per_query_nprobe;
  if (!on_dev) {
    RBQ_CHECK(qb.alloc(sizeof(float) * nq * X->d, s));
    RBQ_CHECK(ib.alloc(sizeof(int64_t) * nq * k, s));
    RBQ_CHECK(db.alloc(sizeof(float) * nq * k, s));
    RBQ_CUDA(cudaMemcpyAsync(qb.p, queries, sizeof(float) * nq * X->d, cudaMemcpyHostToDevice, s));
    if (dnp) {
      RBQ_CHECK(nb.alloc(sizeof(int32_t) * nq, s));
      RBQ_CUDA(cudaMemcpyAsync(nb.p, dnp, sizeof(int32_t) * nq, cudaMemcpyHostToDevice, s));
      dnp = nb.as<int32_t>();
    }
    dq = qb.as<float>();
    dids = ib.as<int64_t>();
    ddist = db.as<float>();
  } else if (!is_device_ptr(queries) || !is_device_ptr(out_ids) || !is_device_ptr(out_dist)) {
    return fail(RABITQ_EINVAL, "rabitq_search: io_on_device set but a pointer is not device memory");
  }
  SearchArgs a;
  a.X = X;
  a.queries = dq;
  a.nq = nq;
  a.k = k;
  a.nprobe = nprobe;
  a.bq = bq;
  a.eps0 = eps0;
  a.seed = opts.quant_seed;
  a.per_query_nprobe = dnp;
  a.cand_cap = opts.max_candidates;
  a.out_ids = dids;
  a.out_dist = ddist;
  a.trace = trace;
  a.rot_precision = opts.rot_precision;
  a.scan_path = opts.scan_path;
  a.layout = opts.scan_layout;
  a.ppl = opts.lane_pairs;
  a.stage = opts.scan_staging;
  if (pr) {
    RBQ_CHECK(pb.alloc(sizeof(int32_t) * nq, s));
    a.pred = pr;
    a.pred_nprobe = pb.as<int32_t>();
  }
  float stage[5] = {0, 0, 0, 0, 0};
  a.stage_ms = opts.collect_stats ? stage : nullptr;
  // non-finite query values are reported after the search (no extra wait)
  DevBuf fin;
  RBQ_CHECK(fin.alloc(sizeof(int), s));
  RBQ_CUDA(cudaMemsetAsync(fin.p, 0, sizeof(int), s));
  RBQ_CHECK(finite_flag(dq, nq * X->d, fin.as<int>(), s));
  RBQ_CHECK(search_dev(a, s));
  if (!on_dev) {
    RBQ_CUDA(cudaMemcpyAsync(out_ids, dids, sizeof(int64_t) * nq * k, cudaMemcpyDeviceToHost, s));
    RBQ_CUDA(cudaMemcpyAsync(out_dist, ddist, sizeof(float) * nq * k, cudaMemcpyDeviceToHost, s));
  }
  // the total ends with the search and its output copies (before the flag read)
  if (opts.collect_stats) RBQ_CUDA(cudaEventRecord(ev[1], s));
  int h_fin = 0;
  RBQ_CUDA(cudaMemcpyAsync(&h_fin, fin.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaStreamSynchronize(s));
  if (h_fin)
    return fail(RABITQ_EINVAL, "rabitq_search: a query has a non-finite value (outputs undefined)");
  if (opts.collect_stats) {
    RBQ_CUDA(cudaEventElapsedTime(&stage[4], ev[0], ev[1]));
    for (int i = 0; i < 5; ++i) g_stats[i] = stage[i];
    g_nstats = 5;
  }
  if (!on_dev) RBQ_CUDA(cudaStreamSynchronize(s));
  return RABITQ_OK;
}

int rabitq_search(const rabitq_index* idx, const float* queries, int64_t nq, int32_t k,
                  int32_t nprobe, int32_t bq, float eps0, int64_t* out_ids, float* out_dist,
                  const rabitq_search_opts* opts) {
  return search_common(idx, queries, nq, k, nprobe, bq, eps0, out_ids, out_dist, opts, nullptr);
}

int rabitq_search_trace(const rabitq_index* idx, const float* queries, int64_t nq, int32_t k,
                        int32_t nprobe, int32_t bq, float eps0, int64_t* out_ids,
                        float* out_dist, const rabitq_search_opts* opts,
                        const rabitq_trace* trace) {
  if (!trace) return fail(RABITQ_EINVAL, "rabitq_search_trace: trace is null");
  return search_common(idx, queries, nq, k, nprobe, bq, eps0, out_ids, out_dist, opts, trace);
}

int rabitq_search_learned(const rabitq_index* idx, const rabitq_predictor* pr,
                          const float* queries, int64_t nq, int32_t k, int32_t bq, float eps0,
                          int64_t* out_ids, float* out_dist, const rabitq_search_opts* opts) {
  if (!idx || !pr) return fail(RABITQ_EINVAL, "rabitq_search_learned: null index or predictor");
  RBQ_CHECK(check_device(pr->device, "rabitq_search_learned (predictor)"));
  if (pr->K != idx->K)
    return fail(RABITQ_EINVAL, "rabitq_search_learned: predictor made for another bucket count");
  if (idx->metric != RABITQ_METRIC_L2)
    return fail(RABITQ_EUNSUPPORTED, "rabitq_search_learned: learned probe counts need a squared-distance (L2) index");
  if (opts && opts->per_query_nprobe)
    return fail(RABITQ_EINVAL, "rabitq_search_learned: per_query_nprobe must be NULL");
  return search_common(idx, queries, nq, k, pr->nprobe_max, bq, eps0, out_ids, out_dist, opts,
                       nullptr, pr);
}

int rabitq_autotune(rabitq_index* X, const float* queries, int64_t nq, int32_t k,
                    int32_t nprobe, int32_t bq, float eps0, int32_t reps,
                    const rabitq_search_opts* opts_in, int32_t* chosen, float* times_ms) {
  g_err.clear();
  if (!X) return fail(RABITQ_EINVAL, "rabitq_autotune: index is null");
  RBQ_CHECK(check_device(X->device, "rabitq_autotune"));
  if (nq < 1 || !queries) return fail(RABITQ_EINVAL, "rabitq_autotune: need queries (nq >= 1)");
  if (reps < 1 || reps > 1000) return fail(RABITQ_EINVAL, "rabitq_autotune: need 1 <= reps <= 1000");
  rabitq_search_opts opts;
  rabitq_search_opts_default(&opts);
  if (opts_in) opts = *opts_in;
  opts.collect_stats = 0;
  cudaStream_t s = static_cast<cudaStream_t>(opts.stream);
  // device copies of the inputs and outputs, so that every timed run is the
  // same device-resident search
  DevBuf qb, ib, db, nb;
  const float* dq = queries;
  const int32_t* dnp = opts.per_query_nprobe;
  if (!opts.io_on_device) {
    RBQ_CHECK(qb.alloc(sizeof(float) * nq * X->d, s));
    RBQ_CUDA(cudaMemcpyAsync(qb.p, queries, sizeof(float) * nq * X->d, cudaMemcpyHostToDevice, s));
    dq = qb.as<float>();
    if (dnp) {
      RBQ_CHECK(nb.alloc(sizeof(int32_t) * nq, s));
      RBQ_CUDA(cudaMemcpyAsync(nb.p, dnp, sizeof(int32_t) * nq, cudaMemcpyHostToDevice, s));
      dnp = nb.as<int32_t>();
    }
  }
  RBQ_CHECK(ib.alloc(sizeof(int64_t) * nq * k, s));
  RBQ_CHECK(db.alloc(sizeof(float) * nq * k, s));
  opts.io_on_device = 1;
  opts.per_query_nprobe = dnp;
  EventSet<2> ev;
  RBQ_CHECK(ev.create());
  float best[2] = {-1.0f, -1.0f};
  const int paths[2] = {RABITQ_SCAN_POPC, RABITQ_SCAN_TC};
  int st_all = RABITQ_OK;
  for (int p = 0; p < 2 && st_all == RABITQ_OK; ++p) {
    opts.scan_path = paths[p];
    for (int r = 0; r <= reps; ++r) {  // run 0 warms up
      RBQ_CUDA(cudaEventRecord(ev[0], s));
      const int st = search_common(X, dq, nq, k, nprobe, bq, eps0, ib.as<int64_t>(),
                                   db.as<float>(), &opts, nullptr);
      if (st == RABITQ_EOVERFLOW && paths[p] == RABITQ_SCAN_TC) {
        best[p] = -1.0f;
        break;
      }
      if (st != RABITQ_OK) {
        st_all = st;
        break;
      }
      RBQ_CUDA(cudaEventRecord(ev[1], s));
      RBQ_CUDA(cudaEventSynchronize(ev[1]));
      float ms = 0.0f;
      RBQ_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
      if (r > 0 && (best[p] < 0.0f || ms < best[p])) best[p] = ms;
    }
  }
  if (st_all != RABITQ_OK) return st_all;
  const int pick = (best[1] >= 0.0f && best[1] < best[0]) ? RABITQ_SCAN_TC : RABITQ_SCAN_POPC;
  X->tuned_path = pick;
  if (chosen) *chosen = pick;
  if (times_ms) {
    times_ms[0] = best[0];
    times_ms[1] = best[1];
  }
  g_err.clear();
  return RABITQ_OK;
}

int rabitq_autotune_tiles(rabitq_index* X, const float* queries, int64_t nq, int32_t k,
                          int32_t nprobe, int32_t bq, float eps0, int32_t reps,
                          const rabitq_search_opts* opts_in, rabitq_tile* best, rabitq_tile* all,
                          int32_t cap, int32_t* n_all) {
  g_err.clear();
  if (!X) return fail(RABITQ_EINVAL, "rabitq_autotune_tiles: index is null");
  RBQ_CHECK(check_device(X->device, "rabitq_autotune_tiles"));
  if (nq < 1 || !queries) return fail(RABITQ_EINVAL, "rabitq_autotune_tiles: need queries (nq >= 1)");
  if (reps < 1 || reps > 1000)
    return fail(RABITQ_EINVAL, "rabitq_autotune_tiles: need 1 <= reps <= 1000");
  if (!best || cap < 0 || (cap > 0 && !all))
    return fail(RABITQ_EINVAL, "rabitq_autotune_tiles: null output");
  rabitq_search_opts opts;
  rabitq_search_opts_default(&opts);
  if (opts_in) opts = *opts_in;
  opts.collect_stats = 0;
  cudaStream_t s = static_cast<cudaStream_t>(opts.stream);
  DevBuf qb, ib, db, nb;
  const float* dq = queries;
  const int32_t* dnp = opts.per_query_nprobe;
  if (!opts.io_on_device) {
    RBQ_CHECK(qb.alloc(sizeof(float) * nq * X->d, s));
    RBQ_CUDA(cudaMemcpyAsync(qb.p, queries, sizeof(float) * nq * X->d, cudaMemcpyHostToDevice, s));
    dq = qb.as<float>();
    if (dnp) {
      RBQ_CHECK(nb.alloc(sizeof(int32_t) * nq, s));
      RBQ_CUDA(cudaMemcpyAsync(nb.p, dnp, sizeof(int32_t) * nq, cudaMemcpyHostToDevice, s));
      dnp = nb.as<int32_t>();
    }
  }
  RBQ_CHECK(ib.alloc(sizeof(int64_t) * nq * k, s));
  RBQ_CHECK(db.alloc(sizeof(float) * nq * k, s));
  opts.io_on_device = 1;
  opts.per_query_nprobe = dnp;
  // the candidates: the warp layout only where it applies
  const bool warp_ok = bq == 4 && k <= 128 && X->d <= 256 && (X->W == 2 || X->W == 4);
  const bool stage_ok = bq == 4 && (X->W == 2 || X->W == 4);
  rabitq_tile cand[6];
  int nc = 0;
  cand[nc++] = rabitq_tile{RABITQ_SCAN_POPC, RABITQ_LAYOUT_CTA, 0, RABITQ_STAGING_OFF, -1.0f};
  if (stage_ok)
    cand[nc++] = rabitq_tile{RABITQ_SCAN_POPC, RABITQ_LAYOUT_CTA, 0, RABITQ_STAGING_BULK, -1.0f};
  if (warp_ok) {
    cand[nc++] = rabitq_tile{RABITQ_SCAN_POPC, RABITQ_LAYOUT_WARP, 1, RABITQ_STAGING_OFF, -1.0f};
    cand[nc++] = rabitq_tile{RABITQ_SCAN_POPC, RABITQ_LAYOUT_WARP, 2, RABITQ_STAGING_OFF, -1.0f};
  }
  cand[nc++] = rabitq_tile{RABITQ_SCAN_TC, 0, 0, 0, -1.0f};
  EventSet<2> ev;
  RBQ_CHECK(ev.create());
  // time with the warp-layout batch rule waived (the tuned tile is then
  // taken for every batch of the class)
  for (int c = 0; c < nc; ++c) {
    opts.scan_path = cand[c].scan_path;
    opts.scan_layout = cand[c].scan_layout;
    opts.lane_pairs = cand[c].lane_pairs;
    opts.scan_staging = cand[c].staging;
    for (int r = 0; r <= reps; ++r) {  // run 0 warms up
      RBQ_CUDA(cudaEventRecord(ev[0], s));
      const int st = search_common(X, dq, nq, k, nprobe, bq, eps0, ib.as<int64_t>(),
                                   db.as<float>(), &opts, nullptr);
      // the tensor-core path is ruled out by an overflow of its lists or a
      // shape it does not take
      if ((st == RABITQ_EOVERFLOW || st == RABITQ_EUNSUPPORTED) &&
          cand[c].scan_path == RABITQ_SCAN_TC) {
        cand[c].time_ms = -1.0f;
        break;
      }
      if (st != RABITQ_OK) return st;
      RBQ_CUDA(cudaEventRecord(ev[1], s));
      RBQ_CUDA(cudaEventSynchronize(ev[1]));
      float ms = 0.0f;
      RBQ_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
      if (r > 0 && (cand[c].time_ms < 0.0f || ms < cand[c].time_ms)) cand[c].time_ms = ms;
    }
  }
  int pick = 0, pick_popc = 0;  // candidate 0 is the popcount CTA tile, always timed
  for (int c = 1; c < nc; ++c) {
    if (cand[c].time_ms < 0.0f) continue;
    if (cand[c].time_ms < cand[pick].time_ms) pick = c;
    if (cand[c].scan_path == RABITQ_SCAN_POPC && cand[c].time_ms < cand[pick_popc].time_ms)
      pick_popc = c;
  }
  rabitq_index::Tile& t = X->tune[tile_class_k(k)][tile_class_np(std::min(nprobe, X->K))];
  t.valid = 1;
  t.path = cand[pick].scan_path;
  t.layout = cand[pick_popc].scan_layout;
  t.ppl = cand[pick_popc].lane_pairs;
  t.stage = cand[pick_popc].staging ? cand[pick_popc].staging : RABITQ_STAGING_OFF;
  *best = cand[pick];
  for (int c = 0; c < nc && c < cap; ++c) all[c] = cand[c];
  if (n_all) *n_all = nc;
  g_err.clear();
  return RABITQ_OK;
}

int rabitq_index_metric(const rabitq_index* X, int32_t* metric) {
  if (!X || !metric) return fail(RABITQ_EINVAL, "rabitq_index_metric: null pointer");
  *metric = X->metric;
  return RABITQ_OK;
}

int rabitq_estimate(const rabitq_index* X, const float* queries, int64_t nq, const int64_t* ids,
                    int32_t m, int32_t bq, float eps0, float* out,
                    const rabitq_search_opts* opts_in) {
  g_err.clear();
  if (!X) return fail(RABITQ_EINVAL, "rabitq_estimate: index is null");
  RBQ_CHECK(check_device(X->device, "rabitq_estimate"));
  rabitq_search_opts opts;
  rabitq_search_opts_default(&opts);
  if (opts_in) opts = *opts_in;
  if (nq < 0 || m < 0) return fail(RABITQ_EINVAL, "rabitq_estimate: nq < 0 or m < 0");
  if (nq == 0 || m == 0) return RABITQ_OK;
  if (!queries || !ids || !out) return fail(RABITQ_EINVAL, "rabitq_estimate: null pointer");
  if (m > (1 << 20) || nq > (int64_t(1) << 40) / m)
    return fail(RABITQ_EINVAL, "rabitq_estimate: nq x m too large");
  if (bq < 1 || bq > 8) return fail(RABITQ_EINVAL, "rabitq_estimate: need 1 <= bq <= 8");
  if (!(eps0 >= 0.0f) || !std::isfinite(eps0))
    return fail(RABITQ_EINVAL, "rabitq_estimate: eps0 must be finite and >= 0");
  if (opts.rot_precision != RABITQ_ROT_FP32 && opts.rot_precision != RABITQ_ROT_TF32 &&
      opts.rot_precision != RABITQ_ROT_BF16)
    return fail(RABITQ_EINVAL, "rabitq_estimate: unknown rot_precision");
  cudaStream_t s = static_cast<cudaStream_t>(opts.stream);
  DevBuf qb, ib, ob, eb;
  const float* dq = queries;
  const int64_t* dids = ids;
  float* dout = out;
  if (!opts.io_on_device) {
    RBQ_CHECK(qb.alloc(sizeof(float) * nq * X->d, s));
    RBQ_CHECK(ib.alloc(sizeof(int64_t) * nq * m, s));
    RBQ_CHECK(ob.alloc(sizeof(float) * nq * m * 3, s));
    RBQ_CUDA(cudaMemcpyAsync(qb.p, queries, sizeof(float) * nq * X->d, cudaMemcpyHostToDevice, s));
    RBQ_CUDA(cudaMemcpyAsync(ib.p, ids, sizeof(int64_t) * nq * m, cudaMemcpyHostToDevice, s));
    dq = qb.as<float>();
    dids = ib.as<int64_t>();
    dout = ob.as<float>();
  } else if (!is_device_ptr(queries) || !is_device_ptr(ids) || !is_device_ptr(out)) {
    return fail(RABITQ_EINVAL,
                "rabitq_estimate: io_on_device set but a pointer is not device memory");
  }
  RBQ_CHECK(eb.alloc(sizeof(int), s));
  RBQ_CUDA(cudaMemsetAsync(eb.p, 0, sizeof(int), s));
  RBQ_CHECK(estimate_dev(X, dq, nq, dids, m, bq, eps0, opts.quant_seed, opts.rot_precision, dout,
                         eb.as<int>(), s));
  if (!opts.io_on_device)
    RBQ_CUDA(cudaMemcpyAsync(out, dout, sizeof(float) * nq * m * 3, cudaMemcpyDeviceToHost, s));
  int h_err = 0;
  RBQ_CUDA(cudaMemcpyAsync(&h_err, eb.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaStreamSynchronize(s));
  if (h_err == 2) return fail(RABITQ_ETIMEOUT, "a tensor-core wait expired (probe scores or query rotation)");
  if (h_err) return fail(RABITQ_EINVAL, "rabitq_estimate: an id is outside [-1, n)");
  return RABITQ_OK;
}

int rabitq_index_info(const rabitq_index* X, int64_t* n, int32_t* d, int32_t* d_pad,
                      int32_t* n_clusters) {
  if (!X) return fail(RABITQ_EINVAL, "rabitq_index_info: index is null");
  if (n) *n = X->n;
  if (d) *d = X->d;
  if (d_pad) *d_pad = X->dpad;
  if (n_clusters) *n_clusters = X->K;
  return RABITQ_OK;
}

int rabitq_get_centroids(const rabitq_index* X, float* out) {
  if (!X || !out) return fail(RABITQ_EINVAL, "rabitq_get_centroids: null pointer");
  RBQ_CUDA(cudaMemcpy(out, X->centroids, sizeof(float) * X->K * X->d, cudaMemcpyDeviceToHost));
  return RABITQ_OK;
}

int rabitq_get_rotation(const rabitq_index* X, double* out) {
  if (!X || !out) return fail(RABITQ_EINVAL, "rabitq_get_rotation: null pointer");
  RBQ_CUDA(cudaMemcpy(out, X->P64, sizeof(double) * X->dpad * X->dpad, cudaMemcpyDeviceToHost));
  return RABITQ_OK;
}

int rabitq_get_assign(const rabitq_index* X, int32_t* cluster) {
  if (!X || !cluster) return fail(RABITQ_EINVAL, "rabitq_get_assign: null pointer");
  RBQ_CUDA(cudaMemcpy(cluster, X->assign, sizeof(int32_t) * X->n, cudaMemcpyDeviceToHost));
  return RABITQ_OK;
}

int rabitq_get_buckets(const rabitq_index* X, int32_t* offsets, int32_t* ids) {
  if (!X) return fail(RABITQ_EINVAL, "rabitq_get_buckets: index is null");
  if (offsets)
    RBQ_CUDA(cudaMemcpy(offsets, X->bucket_off, sizeof(int32_t) * (X->K + 1),
                        cudaMemcpyDeviceToHost));
  if (ids) RBQ_CUDA(cudaMemcpy(ids, X->perm, sizeof(int32_t) * X->n, cudaMemcpyDeviceToHost));
  return RABITQ_OK;
}

int rabitq_get_codes(const rabitq_index* X, uint64_t* out) {
  if (!X || !out) return fail(RABITQ_EINVAL, "rabitq_get_codes: null pointer");
  std::vector<uint64_t> b((size_t)X->n * X->W);
  std::vector<int32_t> perm(X->n);
  RBQ_CUDA(cudaMemcpy(b.data(), X->codes, sizeof(uint64_t) * b.size(), cudaMemcpyDeviceToHost));
  RBQ_CUDA(cudaMemcpy(perm.data(), X->perm, sizeof(int32_t) * X->n, cudaMemcpyDeviceToHost));
  for (int64_t p = 0; p < X->n; ++p)
    std::memcpy(out + (size_t)perm[p] * X->W, b.data() + (size_t)p * X->W, sizeof(uint64_t) * X->W);
  return RABITQ_OK;
}

int rabitq_get_factors(const rabitq_index* X, float* out) {
  if (!X || !out) return fail(RABITQ_EINVAL, "rabitq_get_factors: null pointer");
  std::vector<float4> b(X->n);
  std::vector<int32_t> perm(X->n);
  RBQ_CUDA(cudaMemcpy(b.data(), X->factors, sizeof(float4) * X->n, cudaMemcpyDeviceToHost));
  RBQ_CUDA(cudaMemcpy(perm.data(), X->perm, sizeof(int32_t) * X->n, cudaMemcpyDeviceToHost));
  for (int64_t p = 0; p < X->n; ++p) {
    float* o = out + (size_t)perm[p] * 4;
    o[0] = b[p].x;
    o[1] = b[p].y;
    o[2] = b[p].z;
    o[3] = b[p].w;
  }
  return RABITQ_OK;
}

int rabitq_sample_rotation(uint64_t seed, int32_t d_pad, double* out) {
  g_err.clear();
  if (!out) return fail(RABITQ_EINVAL, "rabitq_sample_rotation: out is null");
  if (d_pad < 2 || d_pad > 4096 || d_pad % 2)
    return fail(RABITQ_EINVAL, "rabitq_sample_rotation: need even 2 <= d_pad <= 4096");
  double* P = nullptr;
  float* P32 = nullptr;
  RBQ_CHECK(dev_alloc(&P, (size_t)d_pad * d_pad));
  int st = dev_alloc(&P32, (size_t)d_pad * d_pad);
  if (st == RABITQ_OK) st = sample_rotation_dev(seed, d_pad, P, P32, nullptr);
  if (st == RABITQ_OK) {
    cudaError_t e = cudaMemcpy(out, P, sizeof(double) * d_pad * d_pad, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) st = fail(RABITQ_ECUDA, cudaGetErrorString(e));
  }
  cudaFree(P);
  cudaFree(P32);
  return st;
}

int rabitq_index_save(const rabitq_index* X, const char* path) {
  g_err.clear();
  if (!X || !path) return fail(RABITQ_EINVAL, "rabitq_index_save: null pointer");
  struct Part {
    const void* dev;
    size_t bytes;
  };
  const Part parts[] = {
      {X->data_b, sizeof(float) * X->n * X->d},     {X->codes, sizeof(uint64_t) * X->n * X->W},
      {X->factors, sizeof(float4) * X->n},          {X->perm, sizeof(int32_t) * X->n},
      {X->bucket_off, sizeof(int32_t) * (X->K + 1)}, {X->assign, sizeof(int32_t) * X->n},
      {X->centroids, sizeof(float) * X->K * X->d},  {X->ptc, sizeof(float) * X->K * X->dpad},
      {X->P64, sizeof(double) * X->dpad * X->dpad}};
  std::vector<std::vector<uint8_t>> host;
  FileHeader h;
  std::memset(&h, 0, sizeof h);
  std::memcpy(h.magic, "RABITQ\0\1", 8);
  h.version = 1;
  h.metric = (uint32_t)X->metric;
  h.n = X->n;
  h.d = X->d;
  h.dpad = X->dpad;
  h.K = X->K;
  h.W = X->W;
  uint32_t crc = 0;
  for (const Part& p : parts) {
    host.emplace_back(p.bytes);
    RBQ_CUDA(cudaMemcpy(host.back().data(), p.dev, p.bytes, cudaMemcpyDeviceToHost));
    crc = crc32_update(crc, host.back().data(), p.bytes);
    h.payload_bytes += p.bytes;
  }
  h.payload_crc = crc;
  h.header_crc = crc32_update(0, &h, offsetof(FileHeader, header_crc));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(RABITQ_EIO, std::string("cannot open for writing: ") + path);
  bool ok = std::fwrite(&h, sizeof h, 1, f) == 1;
  for (auto& b : host) ok = ok && std::fwrite(b.data(), 1, b.size(), f) == b.size();
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(RABITQ_EIO, std::string("write failed: ") + path);
  return RABITQ_OK;
}

int rabitq_index_load(const char* path, const rabitq_build_opts* opts, rabitq_index** out) {
  g_err.clear();
  (void)opts;
  if (!path || !out) return fail(RABITQ_EINVAL, "rabitq_index_load: null pointer");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(RABITQ_EIO, std::string("cannot open: ") + path);
  FileHeader h;
  if (std::fread(&h, sizeof h, 1, f) != 1 || std::memcmp(h.magic, "RABITQ\0\1", 8) != 0 ||
      h.header_crc != crc32_update(0, &h, offsetof(FileHeader, header_crc)) || h.version != 1 ||
      h.n < 1 || h.d < 1 || h.K < 1 || h.dpad < h.d || h.dpad % 64 || h.W != h.dpad / 64 ||
      h.metric > RABITQ_METRIC_COSINE) {
    std::fclose(f);
    return fail(RABITQ_EIO, std::string("not a valid index file (header): ") + path);
  }
  auto* X = new rabitq_index();
  X->n = h.n;
  X->d = h.d;
  X->dpad = h.dpad;
  X->K = h.K;
  X->W = h.W;
  X->metric = (int32_t)h.metric;
  cudaGetDevice(&X->device);
  int st = alloc_index_arrays(X);
  struct Part {
    void* dev;
    size_t bytes;
  };
  const Part parts[] = {
      {X->data_b, sizeof(float) * X->n * X->d},     {X->codes, sizeof(uint64_t) * X->n * X->W},
      {X->factors, sizeof(float4) * X->n},          {X->perm, sizeof(int32_t) * X->n},
      {X->bucket_off, sizeof(int32_t) * (X->K + 1)}, {X->assign, sizeof(int32_t) * X->n},
      {X->centroids, sizeof(float) * X->K * X->d},  {X->ptc, sizeof(float) * X->K * X->dpad},
      {X->P64, sizeof(double) * X->dpad * X->dpad}};
  uint32_t crc = 0;
  uint64_t total = 0;
  std::vector<uint8_t> buf;
  for (const Part& p : parts) {
    if (st != RABITQ_OK) break;
    buf.resize(p.bytes);
    if (std::fread(buf.data(), 1, p.bytes, f) != p.bytes) {
      st = fail(RABITQ_EIO, std::string("truncated index file: ") + path);
      break;
    }
    crc = crc32_update(crc, buf.data(), p.bytes);
    total += p.bytes;
    if (cudaMemcpy(p.dev, buf.data(), p.bytes, cudaMemcpyHostToDevice) != cudaSuccess)
      st = fail(RABITQ_ECUDA, "copy of the index to the device failed");
  }
  std::fclose(f);
  if (st == RABITQ_OK && (crc != h.payload_crc || total != h.payload_bytes))
    st = fail(RABITQ_EIO, std::string("index file checksum mismatch: ") + path);
  if (st == RABITQ_OK) st = transpose_f32(X->centroids, X->K, X->d, X->centroids_t, nullptr);
  if (st == RABITQ_OK) st = pack_centroids(X, nullptr);
  if (st == RABITQ_OK) st = invert_perm(X->perm, X->n, X->inv_perm, nullptr);
  if (st == RABITQ_OK) {
    const int64_t tot = (int64_t)X->dpad * X->dpad;
    std::vector<double> p64(tot);
    std::vector<float> p32(tot);
    cudaMemcpy(p64.data(), X->P64, sizeof(double) * tot, cudaMemcpyDeviceToHost);
    for (int64_t i = 0; i < tot; ++i) p32[i] = (float)p64[i];
    if (cudaMemcpy(X->P32, p32.data(), sizeof(float) * tot, cudaMemcpyHostToDevice) != cudaSuccess)
      st = fail(RABITQ_ECUDA, "copy of P to the device failed");
    if (st == RABITQ_OK) st = pack_pt(X, nullptr);
  }
  if (st == RABITQ_OK) st = max_bucket_size(X, nullptr);
  if (st != RABITQ_OK) {
    free_index_arrays(X);
    delete X;
    return st;
  }
  *out = X;
  return RABITQ_OK;
}

void rabitq_free(rabitq_index* X) {
  if (!X) return;
  cudaDeviceSynchronize();
  free_index_arrays(X);
  delete X;
}

}  // extern "C"
