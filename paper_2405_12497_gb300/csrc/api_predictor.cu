// api_predictor.cu -- C-ABI entry points of the learned probe count: training,
// creation from given parameters, accessors, probe-count prediction, labels,
// and the single-pass gradient / Adam calls used to check the training
// kernels against an independent implementation.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

using namespace rbq;

namespace {

bool device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void free_predictor(rabitq_predictor* pr) {
  if (!pr) return;
  cudaFree(pr->params);
  cudaFree(pr->params_bf16);
  delete pr;
}

int new_predictor(int32_t K, int32_t nprobe_max, rabitq_predictor** out) {
  int dev = 0;
  RBQ_CUDA(cudaGetDevice(&dev));
  auto* pr = new rabitq_predictor();
  pr->device = dev;
  pr->K = K;
  pr->nprobe_max = nprobe_max;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&pr->params), sizeof(float) * kMlpParams);
  if (e == cudaSuccess) e = cudaMalloc(&pr->params_bf16, sizeof(uint16_t) * kMlpParams);
  if (e != cudaSuccess) {
    free_predictor(pr);
    return fail(RABITQ_ENOMEM, std::string("predictor allocation failed: ") + cudaGetErrorString(e));
  }
  *out = pr;
  return RABITQ_OK;
}

}  // namespace

extern "C" {

void rabitq_predictor_opts_default(rabitq_predictor_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->k = 100;
  o->target_recall = 0.95f;
  o->epochs = 30;
  o->batch = 1024;
  o->lr = 1e-3f;
  o->val_fraction = 0.1f;
  o->seed = 5;
}

int rabitq_predictor_train(const rabitq_index* X, const float* train_q, int64_t nt,
                           const rabitq_predictor_opts* opts_in, rabitq_predictor** out) {
  set_error("");
  if (!out) return fail(RABITQ_EINVAL, "rabitq_predictor_train: out is null");
  *out = nullptr;
  if (!X || !train_q) return fail(RABITQ_EINVAL, "rabitq_predictor_train: null index or queries");
  RBQ_CHECK(check_device(X->device, "rabitq_predictor_train"));
  if (X->metric != RABITQ_METRIC_L2)
    return fail(RABITQ_EUNSUPPORTED, "rabitq_predictor_train: learned probe counts need a squared-distance (L2) index");
  rabitq_predictor_opts o;
  rabitq_predictor_opts_default(&o);
  if (opts_in) o = *opts_in;
  const int nmax = o.nprobe_max ? o.nprobe_max : std::min(X->K, 512);
  if (nt < 2) return fail(RABITQ_EINVAL, "rabitq_predictor_train: need at least 2 queries");
  if (o.k < 1 || o.k > 1024) return fail(RABITQ_EINVAL, "rabitq_predictor_train: need 1 <= k <= 1024");
  if (!(o.target_recall > 0.0f && o.target_recall <= 1.0f))
    return fail(RABITQ_EINVAL, "rabitq_predictor_train: target_recall must be in (0, 1]");
  if (nmax < 1 || nmax > X->K || nmax > 16384)
    return fail(RABITQ_EINVAL, "rabitq_predictor_train: need 1 <= nprobe_max <= min(K, 16384)");
  if (o.epochs < 0 || o.epochs > 100000 || o.batch < 1 || o.batch > 65536)
    return fail(RABITQ_EINVAL, "rabitq_predictor_train: need 0 <= epochs, 1 <= batch <= 65536");
  if (!(o.lr > 0.0f) || !std::isfinite(o.lr))
    return fail(RABITQ_EINVAL, "rabitq_predictor_train: lr must be finite and > 0");
  if (!(o.val_fraction >= 0.0f && o.val_fraction < 1.0f))
    return fail(RABITQ_EINVAL, "rabitq_predictor_train: val_fraction must be in [0, 1)");
  cudaStream_t s = static_cast<cudaStream_t>(o.stream);
  const int d = X->d;
  DevBuf qb, gb;
  const float* dq = train_q;
  const int64_t* dgt = o.gt_ids;
  if (o.io_on_device) {
    if (!device_ptr(train_q) || (o.gt_ids && !device_ptr(o.gt_ids)))
      return fail(RABITQ_EINVAL, "rabitq_predictor_train: io_on_device set but a pointer is not "
                                 "device memory");
  } else {
    RBQ_CHECK(qb.alloc(sizeof(float) * nt * d, s));
    RBQ_CUDA(cudaMemcpyAsync(qb.p, train_q, sizeof(float) * nt * d, cudaMemcpyHostToDevice, s));
    dq = qb.as<float>();
    if (o.gt_ids) {
      RBQ_CHECK(gb.alloc(sizeof(int64_t) * nt * o.k, s));
      RBQ_CUDA(cudaMemcpyAsync(gb.p, o.gt_ids, sizeof(int64_t) * nt * o.k, cudaMemcpyHostToDevice,
                               s));
      dgt = gb.as<int64_t>();
    }
  }
  bool finite = true;
  RBQ_CHECK(check_finite(dq, nt * d, s, &finite));
  if (!finite) return fail(RABITQ_EINVAL, "rabitq_predictor_train: non-finite query value");
  rabitq_predictor* pr = nullptr;
  RBQ_CHECK(new_predictor(X->K, nmax, &pr));
  pr->k = o.k;
  pr->target_recall = o.target_recall;
  int st = predictor_train_dev(X, dq, nt, dgt, o, pr, s);
  if (st == RABITQ_OK && cudaStreamSynchronize(s) != cudaSuccess)
    st = fail(RABITQ_ECUDA, "rabitq_predictor_train: stream error");
  if (st != RABITQ_OK) {
    free_predictor(pr);
    return st;
  }
  *out = pr;
  return RABITQ_OK;
}

int rabitq_predictor_create(const float* params, float s0, float mult, int32_t nprobe_max,
                            int32_t n_clusters, rabitq_predictor** out) {
  set_error("");
  if (!out || !params) return fail(RABITQ_EINVAL, "rabitq_predictor_create: null pointer");
  *out = nullptr;
  if (!(s0 > 0.0f) || !std::isfinite(s0) || !(mult > 0.0f) || !std::isfinite(mult))
    return fail(RABITQ_EINVAL, "rabitq_predictor_create: s0 and mult must be finite and > 0");
  if (n_clusters < 1 || nprobe_max < 1 || nprobe_max > n_clusters || nprobe_max > 16384)
    return fail(RABITQ_EINVAL, "rabitq_predictor_create: need 1 <= nprobe_max <= min(K, 16384)");
  for (int i = 0; i < kMlpParams; ++i)
    if (!std::isfinite(params[i]))
      return fail(RABITQ_EINVAL, "rabitq_predictor_create: non-finite parameter");
  rabitq_predictor* pr = nullptr;
  RBQ_CHECK(new_predictor(n_clusters, nprobe_max, &pr));
  pr->s0 = s0;
  pr->mult = mult;
  int st = RABITQ_OK;
  if (cudaMemcpy(pr->params, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice) !=
      cudaSuccess)
    st = fail(RABITQ_ECUDA, "rabitq_predictor_create: copy failed");
  if (st == RABITQ_OK) st = mlp_pack_bf16(pr, nullptr);
  if (st == RABITQ_OK && cudaDeviceSynchronize() != cudaSuccess)
    st = fail(RABITQ_ECUDA, "rabitq_predictor_create: device error");
  if (st != RABITQ_OK) {
    free_predictor(pr);
    return st;
  }
  *out = pr;
  return RABITQ_OK;
}

int rabitq_predictor_get_info(const rabitq_predictor* pr, rabitq_predictor_info* out) {
  if (!pr || !out) return fail(RABITQ_EINVAL, "rabitq_predictor_get_info: null pointer");
  out->n_clusters = pr->K;
  out->k = pr->k;
  out->nprobe_max = pr->nprobe_max;
  out->target_recall = pr->target_recall;
  out->s0 = pr->s0;
  out->mult = pr->mult;
  out->train_loss = pr->train_loss;
  out->val_loss = pr->val_loss;
  out->val_recall = pr->val_recall;
  out->val_mean_nprobe = pr->val_mean_nprobe;
  out->n_train = pr->n_train;
  out->n_val = pr->n_val;
  return RABITQ_OK;
}

int rabitq_predictor_get_params(const rabitq_predictor* pr, float* out) {
  if (!pr || !out) return fail(RABITQ_EINVAL, "rabitq_predictor_get_params: null pointer");
  RBQ_CUDA(cudaMemcpy(out, pr->params, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
  return RABITQ_OK;
}

int rabitq_predictor_set_mult(rabitq_predictor* pr, float mult) {
  if (!pr) return fail(RABITQ_EINVAL, "rabitq_predictor_set_mult: null predictor");
  if (!(mult > 0.0f) || !std::isfinite(mult))
    return fail(RABITQ_EINVAL, "rabitq_predictor_set_mult: mult must be finite and > 0");
  pr->mult = mult;
  return RABITQ_OK;
}

void rabitq_predictor_free(rabitq_predictor* pr) {
  if (!pr) return;
  cudaDeviceSynchronize();
  free_predictor(pr);
}

int rabitq_predict_nprobe(const rabitq_index* X, const rabitq_predictor* pr,
                          const float* queries, int64_t nq, int32_t* out_nprobe,
                          float* out_features, float* out_y, const rabitq_search_opts* opts_in) {
  set_error("");
  if (!X || !pr) return fail(RABITQ_EINVAL, "rabitq_predict_nprobe: null index or predictor");
  RBQ_CHECK(check_device(X->device, "rabitq_predict_nprobe"));
  RBQ_CHECK(check_device(pr->device, "rabitq_predict_nprobe (predictor)"));
  if (pr->K != X->K)
    return fail(RABITQ_EINVAL, "rabitq_predict_nprobe: predictor made for another bucket count");
  if (X->metric != RABITQ_METRIC_L2)
    return fail(RABITQ_EUNSUPPORTED, "rabitq_predict_nprobe: learned probe counts need a squared-distance (L2) index");
  if (nq < 0) return fail(RABITQ_EINVAL, "rabitq_predict_nprobe: nq < 0");
  if (nq == 0) return RABITQ_OK;
  if (!queries || !out_nprobe) return fail(RABITQ_EINVAL, "rabitq_predict_nprobe: null pointer");
  rabitq_search_opts opts;
  rabitq_search_opts_default(&opts);
  if (opts_in) opts = *opts_in;
  cudaStream_t s = static_cast<cudaStream_t>(opts.stream);
  const int d = X->d;
  DevBuf qb, nb, fb, yb;
  const float* dq = queries;
  int32_t* dn = out_nprobe;
  float* df = out_features;
  float* dy = out_y;
  if (opts.io_on_device) {
    if (!device_ptr(queries) || !device_ptr(out_nprobe) ||
        (out_features && !device_ptr(out_features)) || (out_y && !device_ptr(out_y)))
      return fail(RABITQ_EINVAL, "rabitq_predict_nprobe: io_on_device set but a pointer is not "
                                 "device memory");
  } else {
    RBQ_CHECK(qb.alloc(sizeof(float) * nq * d, s));
    RBQ_CHECK(nb.alloc(sizeof(int32_t) * nq, s));
    RBQ_CUDA(cudaMemcpyAsync(qb.p, queries, sizeof(float) * nq * d, cudaMemcpyHostToDevice, s));
    dq = qb.as<float>();
    dn = nb.as<int32_t>();
    if (out_features) {
      RBQ_CHECK(fb.alloc(sizeof(float) * nq * kMlpIn, s));
      df = fb.as<float>();
    }
    if (out_y) {
      RBQ_CHECK(yb.alloc(sizeof(float) * nq, s));
      dy = yb.as<float>();
    }
  }
  RBQ_CHECK(predict_dev(X, pr, dq, nq, dn, df, dy, s));
  if (!opts.io_on_device) {
    RBQ_CUDA(cudaMemcpyAsync(out_nprobe, dn, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, s));
    if (out_features)
      RBQ_CUDA(cudaMemcpyAsync(out_features, df, sizeof(float) * nq * kMlpIn,
                               cudaMemcpyDeviceToHost, s));
    if (out_y)
      RBQ_CUDA(cudaMemcpyAsync(out_y, dy, sizeof(float) * nq, cudaMemcpyDeviceToHost, s));
    RBQ_CUDA(cudaStreamSynchronize(s));
  }
  return RABITQ_OK;
}

int rabitq_compute_labels(const rabitq_index* X, const float* queries, int64_t nq,
                          const int64_t* gt_ids, int32_t k, float target_recall,
                          int32_t nprobe_max, int32_t* ranks, int32_t* label_r) {
  set_error("");
  if (!X) return fail(RABITQ_EINVAL, "rabitq_compute_labels: index is null");
  RBQ_CHECK(check_device(X->device, "rabitq_compute_labels"));
  if (X->metric != RABITQ_METRIC_L2)
    return fail(RABITQ_EUNSUPPORTED, "rabitq_compute_labels: learned probe counts need a squared-distance (L2) index");
  if (nq < 0) return fail(RABITQ_EINVAL, "rabitq_compute_labels: nq < 0");
  if (nq == 0) return RABITQ_OK;
  if (!queries || !gt_ids || !ranks || !label_r)
    return fail(RABITQ_EINVAL, "rabitq_compute_labels: null pointer");
  if (k < 1 || k > 1024) return fail(RABITQ_EINVAL, "rabitq_compute_labels: need 1 <= k <= 1024");
  if (!(target_recall > 0.0f && target_recall <= 1.0f))
    return fail(RABITQ_EINVAL, "rabitq_compute_labels: target_recall must be in (0, 1]");
  if (nprobe_max < 1 || nprobe_max > X->K || nprobe_max > 16384)
    return fail(RABITQ_EINVAL, "rabitq_compute_labels: need 1 <= nprobe_max <= min(K, 16384)");
  cudaStream_t s = nullptr;
  DevBuf qb, gb, rb, lb;
  RBQ_CHECK(qb.alloc(sizeof(float) * nq * X->d, s));
  RBQ_CHECK(gb.alloc(sizeof(int64_t) * nq * k, s));
  RBQ_CHECK(rb.alloc(sizeof(int32_t) * nq * k, s));
  RBQ_CHECK(lb.alloc(sizeof(int32_t) * nq, s));
  RBQ_CUDA(cudaMemcpyAsync(qb.p, queries, sizeof(float) * nq * X->d, cudaMemcpyHostToDevice, s));
  RBQ_CUDA(cudaMemcpyAsync(gb.p, gt_ids, sizeof(int64_t) * nq * k, cudaMemcpyHostToDevice, s));
  RBQ_CHECK(mlp_labels_dev(X, qb.as<float>(), nq, gb.as<int64_t>(), k,
                           mlp_need(target_recall, k), nprobe_max, rb.as<int32_t>(),
                           lb.as<int32_t>(), s));
  RBQ_CUDA(cudaMemcpyAsync(ranks, rb.p, sizeof(int32_t) * nq * k, cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaMemcpyAsync(label_r, lb.p, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaStreamSynchronize(s));
  return RABITQ_OK;
}

int rabitq_mlp_grad(const float* params, const float* X, const float* t, int64_t B, float* y,
                    float* grads, float* loss) {
  set_error("");
  if (!params || !X || !t) return fail(RABITQ_EINVAL, "rabitq_mlp_grad: null input");
  if (B < 1 || B > (int64_t(1) << 20))
    return fail(RABITQ_EINVAL, "rabitq_mlp_grad: need 1 <= B <= 2^20");
  cudaStream_t s = nullptr;
  DevBuf pb, xb, tb, gb, lb;
  RBQ_CHECK(pb.alloc(sizeof(float) * kMlpParams, s));
  RBQ_CHECK(xb.alloc(sizeof(float) * B * kMlpIn, s));
  RBQ_CHECK(tb.alloc(sizeof(float) * B, s));
  RBQ_CHECK(gb.alloc(sizeof(float) * kMlpParams, s));
  RBQ_CHECK(lb.alloc(sizeof(double), s));
  RBQ_CUDA(cudaMemcpyAsync(pb.p, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, s));
  RBQ_CUDA(cudaMemcpyAsync(xb.p, X, sizeof(float) * B * kMlpIn, cudaMemcpyHostToDevice, s));
  RBQ_CUDA(cudaMemcpyAsync(tb.p, t, sizeof(float) * B, cudaMemcpyHostToDevice, s));
  MlpWork w;
  RBQ_CHECK(w.alloc(B, s));
  RBQ_CHECK(mlp_backward(pb.as<float>(), xb.as<float>(), tb.as<float>(), B, gb.as<float>(), w, s));
  RBQ_CHECK(mlp_sum_sq_err(w.y, tb.as<float>(), B, lb.as<double>(), s));
  double sse = 0.0;
  if (y) RBQ_CUDA(cudaMemcpyAsync(y, w.y, sizeof(float) * B, cudaMemcpyDeviceToHost, s));
  if (grads)
    RBQ_CUDA(cudaMemcpyAsync(grads, gb.p, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaMemcpyAsync(&sse, lb.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaStreamSynchronize(s));
  if (loss) *loss = (float)(sse / (double)B);
  return RABITQ_OK;
}

int rabitq_mlp_adam(float* master, float* m1, float* m2, const float* grads, int32_t step,
                    float lr, float* work) {
  set_error("");
  if (!master || !m1 || !m2 || !grads || !work)
    return fail(RABITQ_EINVAL, "rabitq_mlp_adam: null pointer");
  if (step < 1) return fail(RABITQ_EINVAL, "rabitq_mlp_adam: step must be >= 1");
  if (!(lr > 0.0f) || !std::isfinite(lr))
    return fail(RABITQ_EINVAL, "rabitq_mlp_adam: lr must be finite and > 0");
  cudaStream_t s = nullptr;
  const size_t bytes = sizeof(float) * kMlpParams;
  DevBuf buf;
  RBQ_CHECK(buf.alloc(bytes * 5, s));
  float* dm = buf.as<float>();
  float* d1 = dm + kMlpParams;
  float* d2 = d1 + kMlpParams;
  float* dg = d2 + kMlpParams;
  float* dw = dg + kMlpParams;
  RBQ_CUDA(cudaMemcpyAsync(dm, master, bytes, cudaMemcpyHostToDevice, s));
  RBQ_CUDA(cudaMemcpyAsync(d1, m1, bytes, cudaMemcpyHostToDevice, s));
  RBQ_CUDA(cudaMemcpyAsync(d2, m2, bytes, cudaMemcpyHostToDevice, s));
  RBQ_CUDA(cudaMemcpyAsync(dg, grads, bytes, cudaMemcpyHostToDevice, s));
  RBQ_CHECK(mlp_adam(dm, dw, dg, d1, d2, lr, step, s));
  RBQ_CUDA(cudaMemcpyAsync(master, dm, bytes, cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaMemcpyAsync(m1, d1, bytes, cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaMemcpyAsync(m2, d2, bytes, cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaMemcpyAsync(work, dw, bytes, cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaStreamSynchronize(s));
  return RABITQ_OK;
}

}  // extern "C"
