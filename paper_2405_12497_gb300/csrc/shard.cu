// shard.cu -- bucket sharding of the IVF index across GPUs (or any set of
// index pieces): the clusters are split into size-balanced shards, each
// shard is an index of its clusters' points built with the global centroids
// and the global rotation (so its codes, factors, probe lists and random
// quantization streams are those of the unsharded index), every shard is
// searched on its own (its threshold tau_ub is the k-th smallest upper bound
// of its own codes, at least the global one, so its candidate set is a
// superset of the global one restricted to the shard), and the per-shard
// top-k lists are merged by (distance, id). The exchange is one gather of
// nq x k (id, distance) per shard.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace {

using namespace rbq;

// One CTA per query: the n_lists x k_in candidates (ids mapped through the
// lists' labels) as keys (score key << 32 | id), sorted in shared memory,
// the k smallest written out. The score is the distance, or the negated
// inner product (IP metrics return inner products, largest first). Ids are
// at most 2^32 - 2 (the all-ones id is the padding's).
__global__ void merge_topk_kernel(const float* __restrict__ dist, const int64_t* __restrict__ ids,
                                  int n_lists, int64_t nq, int k_in, int k,
                                  const int64_t* const* __restrict__ labels, int ip,
                                  int sort_n, int64_t* __restrict__ out_ids,
                                  float* __restrict__ out_dist) {
  extern __shared__ unsigned long long keys[];
  const int64_t q = blockIdx.x;
  const int n = n_lists * k_in;
  for (int i = threadIdx.x; i < sort_n; i += blockDim.x) {
    unsigned long long key = ~0ull;
    if (i < n) {
      const int l = i / k_in, j = i - l * k_in;
      const int64_t src = ((int64_t)l * nq + q) * k_in + j;
      int64_t id = ids[src];
      if (id >= 0) {
        if (labels && labels[l]) id = labels[l][id];
        const float v = dist[src];
        key = ((unsigned long long)float_key(ip ? -v : v) << 32) | (uint32_t)id;
      }
    }
    keys[i] = key;
  }
  __syncthreads();
  block_bitonic_sort_u64(keys, sort_n);
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const unsigned long long key = keys[j];
    const bool ok = key != ~0ull;
    out_ids[q * k + j] = ok ? (int64_t)(key & 0xffffffffu) : -1;
    const float v = ok ? key_float((uint32_t)(key >> 32)) : __int_as_float(0x7f800000);
    out_dist[q * k + j] = ip ? -v : v;
  }
}

}  // namespace

extern "C" {

int rabitq_shard_clusters(const int32_t* sizes, int32_t K, int32_t S, int32_t* shard_of,
                          int64_t* shard_points) {
  if (!sizes || !shard_of || K < 1 || S < 1 || S > K)
    return fail(RABITQ_EINVAL, "rabitq_shard_clusters: need sizes, shard_of and 1 <= S <= K");
  std::vector<int32_t> order(K);
  for (int32_t c = 0; c < K; ++c) {
    if (sizes[c] < 0) return fail(RABITQ_EINVAL, "rabitq_shard_clusters: negative cluster size");
    order[c] = c;
  }
  // longest processing time first: the largest cluster goes to the shard
  // with the fewest points so far (ties: lower cluster id, lower shard)
  std::stable_sort(order.begin(), order.end(),
                   [sizes](int32_t a, int32_t b) { return sizes[a] > sizes[b]; });
  std::vector<int64_t> load(S, 0);
  for (int32_t c : order) {
    int32_t best = 0;
    for (int32_t s = 1; s < S; ++s)
      if (load[s] < load[best]) best = s;
    shard_of[c] = best;
    load[best] += sizes[c];
  }
  if (shard_points)
    for (int32_t s = 0; s < S; ++s) shard_points[s] = load[s];
  return RABITQ_OK;
}

int rabitq_merge_topk(const float* dist, const int64_t* ids, int32_t n_lists, int64_t nq,
                      int32_t k_in, int32_t k, const int64_t* const* labels, int32_t metric,
                      int64_t* out_ids, float* out_dist, void* stream) {
  set_error("");
  if (nq < 0 || nq > 0x7fffffff)
    return fail(RABITQ_EINVAL, "rabitq_merge_topk: need 0 <= nq <= 2^31 - 1 (one CTA per query)");
  if (nq == 0) return RABITQ_OK;
  if (!dist || !ids || !out_ids || !out_dist)
    return fail(RABITQ_EINVAL, "rabitq_merge_topk: null pointer");
  if (n_lists < 1 || k_in < 1 || k < 1 || k > 1024 || (int64_t)n_lists * k_in > 8192)
    return fail(RABITQ_EINVAL,
                "rabitq_merge_topk: need n_lists, k_in >= 1, 1 <= k <= 1024, n_lists * k_in <= 8192");
  if (metric < RABITQ_METRIC_L2 || metric > RABITQ_METRIC_COSINE)
    return fail(RABITQ_EINVAL, "rabitq_merge_topk: unknown metric");
  int sort_n = 1;
  while (sort_n < n_lists * k_in || sort_n < k) sort_n <<= 1;
  const size_t smem = sizeof(unsigned long long) * sort_n;
  RBQ_CUDA(cudaFuncSetAttribute(merge_topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  merge_topk_kernel<<<(unsigned)nq, 256, smem, static_cast<cudaStream_t>(stream)>>>(
      dist, ids, n_lists, nq, k_in, k, labels, metric != RABITQ_METRIC_L2 ? 1 : 0, sort_n, out_ids,
      out_dist);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

}  // extern "C"
