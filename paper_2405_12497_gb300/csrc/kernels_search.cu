// kernels_search.cu -- query phase (Alg. 2 of the paper with the IVF probing
// and error-bound re-ranking of §4).
//
// Stages per batch of queries:
//   1. TF32 tensor-core products <q, c> with every centroid (kernels_tc.cu);
//   2. probe selection: the nprobe nearest centroids by canonical (distance,
//      id), exactly, from bounds on those products (probe_select_kernel);
//      with learned probe counts, the 64 nearest first (the network's
//      features), then each query's count;
//   3. query rotation P^{-1}[q_r; 0] (kernels_gemm.cu FP32 canonical, or
//      kernels_tc.cu BF16 / TF32);
//   4. one persistent fused kernel, a CTA per query at a time: randomized
//      B_q-bit quantization of q' per probed cluster (§3.3.1), bucket scan
//      with the bit-plane popcount form of <x_b, q_u> (§3.3.2), the unbiased
//      estimator and its error bound (Theorem 3.2), the k-th smallest upper
//      bound tau, the survivors LB <= tau, their exact distances and the
//      top-k by (distance, id).
// Also here: the split-mode merge, the bucket-major tensor-core scan path,
// the single-code estimator (§3.3.2, first case) and the host launchers.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"
#include "tc_util.cuh"

namespace rbq {
namespace {

constexpr int kThreads = 256;

// ------------------------------------------------------------ selection
// Top-nsel of K scores score(c) by (score, id): radix select of the nsel-th
// smallest key, collection of everything below it plus the lowest ids among
// its ties, then a bitonic sort of the selection (sel: sort_n entries of
// shared memory). Writes nprobe slots of out_ids/out_dist (-1/+inf after
// nsel). Whole block.
template <class F>
__device__ void select_row(F score, int K, int nsel, int nprobe, int sort_n,
                           unsigned long long* sel, int32_t* out_ids, float* out_dist) {
  __shared__ int hist[256];
  __shared__ uint32_t s_prefix, s_mask;
  __shared__ int s_remaining, s_less, s_tie_base;
  __syncthreads();
  if (threadIdx.x == 0) {
    s_prefix = 0;
    s_mask = 0;
    s_remaining = nsel;
    s_less = 0;
    s_tie_base = 0;
  }
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const uint32_t prefix = s_prefix, mask = s_mask;
    for (int c = threadIdx.x; c < K; c += blockDim.x) {
      const uint32_t key = float_key(score(c));
      if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int rem = s_remaining, b = 0;
      while (b < 255 && hist[b] < rem) {
        rem -= hist[b];
        ++b;
      }
      s_remaining = rem;
      s_prefix = prefix | ((uint32_t)b << shift);
      s_mask = mask | (255u << shift);
    }
    __syncthreads();
  }
  const uint32_t T = s_prefix;
  const int need_ties = s_remaining;  // ties with key T to take, lowest ids first
  for (int i = threadIdx.x; i < sort_n; i += blockDim.x) sel[i] = ~0ull;
  __syncthreads();
  const int n_less = nsel - need_ties;
  for (int c = threadIdx.x; c < K; c += blockDim.x) {
    const uint32_t key = float_key(score(c));
    if (key < T) sel[atomicAdd(&s_less, 1)] = ((unsigned long long)key << 32) | (uint32_t)c;
  }
  __syncthreads();
  // ties in ascending id order, chunk by chunk
  __shared__ int warp_cnt[kThreads / 32];
  for (int c0 = 0; c0 < K; c0 += blockDim.x) {
    if (s_tie_base >= need_ties) break;
    const int c = c0 + threadIdx.x;
    const bool tie = (c < K) && float_key(score(c)) == T;
    const unsigned b = __ballot_sync(kFull, tie);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_cnt[wid] = __popc(b);
    __syncthreads();
    int before = s_tie_base;
    for (int w = 0; w < wid; ++w) before += warp_cnt[w];
    const int rank = before + __popc(b & ((1u << lane) - 1u));
    if (tie && rank < need_ties)
      sel[n_less + rank] = ((unsigned long long)T << 32) | (uint32_t)c;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += warp_cnt[w];
      s_tie_base += tot;
    }
    __syncthreads();
  }
  __syncthreads();
  block_bitonic_sort_u64(sel, sort_n);
  for (int j = threadIdx.x; j < nprobe; j += blockDim.x) {
    const bool ok = j < nsel;
    out_ids[j] = ok ? (int32_t)(sel[j] & 0xffffffffu) : -1;
    out_dist[j] = ok ? key_float((uint32_t)(sel[j] >> 32)) : __int_as_float(0x7f800000);
  }
  __syncthreads();
}


// ------------------------------------------------------ fused query kernel
// Shared state of the block radix select.
struct SelState {
  int hist[256];
  int bin, rem, tie_taken;
  int warp_cnt[kThreads / 32];
  unsigned long long wmin[kThreads / 32], wmax[kThreads / 32];
};

struct FusedParams {
  const float* queries;     // nq x d
  const float* rq;          // nq x dpad
  const int32_t* probe_ids; // nq x nprobe
  const float* probe_dist;  // nq x nprobe: centroid scores, the estimator's additive term
  const float* probe_nq2;   // nq x nprobe ||q_r - c||^2 (IP metric), null = probe_dist
  const int32_t* nprobe_q;  // nq or null
  const float* ptc;         // K x dpad
  const uint64_t* codes;    // n x W (bucket order)
  const float4* factors;    // n (bucket order)
  const float* data_b;      // n x d (bucket order)
  const int32_t* perm;      // n: position -> id
  const int32_t* inv_perm;  // n: id -> position
  const int32_t* bucket_off;
  int64_t nq, q_offset;
  int d, dpad, W, bq, k, m, nprobe, pch, cu, ce, ct;
  float eps0;
  uint64_t seed;
  int cand_cap;
  int metric;               // 0: squared distance; 1: inner product (score -<o_r, q_r>)
  int4* cand;               // gridDim.x x cand_cap: {pos, LB, estimate, -}
  int64_t* out_ids;
  float* out_dist;
  int* err;
  rabitq_trace tr;
  // query scheduling: CTAs take the next query from *next (zeroed before the
  // launch) in the order `order` (null = ascending); next == null = static
  // striding by gridDim.x
  const int32_t* order;
  int* next;
  int scap;  // shared-memory capacity for the tail's candidate list (0 = none)
  // Split mode (split > 1, for batches too small to fill the GPU): work item
  // i scans probe slice i % split of query i / split into candidate region i
  // and writes the slice's k smallest upper-bound keys to ub_out[i k ...] and
  // {keys written, candidates} to slice_cnt[2 i ...]; split_merge_kernel
  // then finishes each query from its slices. cand2: one merged-list region
  // of cand_cap entries per query.
  int split;
  uint32_t* ub_out;
  int* slice_cnt;
  int4* cand2;
  // Warp-per-query kernel: candidate region of capw entries per warp; a
  // query whose list outgrows it goes to redo[*redo_cnt++]. The CTA kernel
  // redoing them reads its query count from *nq_dev when that is set.
  int4* candw;
  int capw;
  int32_t* redo;
  int* redo_cnt;
  const int* nq_dev;
};

struct FusedSmem {
  uint64_t* planes;  // pch x bq x W
  float4* pmeta;     // pch: A, B, E, nq2
  int* psum;         // pch
  int* pbeg;         // pch
  int* pref;         // pch + 1
  float* qv;         // d
  SelState* sel;     // radix-select scratch
  uint32_t* ubk;     // cu: upper-bound keys
  unsigned long long* estk;  // ce: the pilot list, (id << 32) | position
  unsigned long long* topk;  // ct: (exact distance key << 32) | id
  int4* scand;               // scap: the candidate list staged for the tail
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline size_t fused_smem_bytes(int pch, int bq, int W, int d, int cu, int ce,
                                                   int ct, int nwarps,
                                                   size_t* off /* 10 entries or null */,
                                                   int scap = 0) {
  size_t o = 0, offs[10];
  (void)nwarps;
  offs[0] = o; o = align_up(o + sizeof(uint64_t) * pch * bq * W, 16);
  offs[1] = o; o = align_up(o + sizeof(float4) * pch, 16);
  offs[2] = o; o = align_up(o + sizeof(int) * pch, 16);
  offs[3] = o; o = align_up(o + sizeof(int) * pch, 16);
  offs[4] = o; o = align_up(o + sizeof(int) * (pch + 1), 16);
  offs[5] = o; o = align_up(o + sizeof(float) * d, 16);
  offs[6] = o; o = align_up(o + sizeof(uint32_t) * cu, 16);
  offs[7] = o; o = align_up(o + sizeof(unsigned long long) * ce, 16);
  offs[8] = o; o = align_up(o + sizeof(unsigned long long) * ct, 16);
  offs[9] = o; o = align_up(o + sizeof(int4) * scap, 16);
  if (off)
    for (int i = 0; i < 10; ++i) off[i] = offs[i];
  return o;
}

// Randomized B_q-bit quantization of q' for one probed cluster with one warp
// (§3.3.1): qd = rq - P^T c, v_l = min qd, v_r = max qd, Delta = (v_r -
// v_l)/(2^B_q - 1), q_u[k] = min(floor((qd[k] - v_l)/Delta + u_k), 2^B_q - 1)
// with u_k from Philox(seed; k/4, query, cluster, 3). Lane l holds elements
// k = 128 i + 4 l + r (r = 0..3), so the four u_k of one Philox call belong to
// one lane; emit(i, k0, qu) receives them block by block (warp-uniform).
// Returns sum(q_u) in every lane; writes v_l and Delta.
template <class Emit>
__device__ __forceinline__ int quant_core(const float* rq, const float* pc, int dpad, int bq,
                                          uint64_t seed, uint64_t gq, int c, float* vl_out,
                                          float* delta_out, Emit emit) {
  const int lane = threadIdx.x & 31;
  const int nblk = (dpad + 127) >> 7;
  float vl = __int_as_float(0x7f800000), vr = __int_as_float(0xff800000);
  for (int kk = lane; kk < dpad; kk += 32) {
    const float v = __fsub_rn(rq[kk], pc[kk]);
    vl = fminf(vl, v);
    vr = fmaxf(vr, v);
  }
  vl = warp_min_f(vl);
  vr = warp_max_f(vr);
  const int qmax = (1 << bq) - 1;
  const float delta = __fdiv_rn(__fsub_rn(vr, vl), (float)qmax);
  int sum = 0;
  for (int i = 0; i < nblk; ++i) {
    const int k0 = 128 * i + 4 * lane;
    int qu[4] = {0, 0, 0, 0};
    if (delta > 0.0f && k0 < dpad) {
      float qd[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) qd[r] = (k0 + r < dpad) ? __fsub_rn(rq[k0 + r], pc[k0 + r]) : 0.0f;
      const U4 w = philox4x32_10(seed, (uint32_t)(k0 >> 2), (uint32_t)gq, (uint32_t)c, kTagQuant);
      const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (k0 + r < dpad) {
          const float u = __fmul_rn(__uint2float_rn(ws[r] >> 8), 0x1.0p-24f);
          const float x = __fdiv_rn(__fsub_rn(qd[r], vl), delta);
          const int v = __float2int_rd(__fadd_rn(x, u));
          qu[r] = v > qmax ? qmax : v;
        }
      }
    }
    sum += qu[0] + qu[1] + qu[2] + qu[3];
    emit(i, k0, qu);
  }
  *vl_out = vl;
  *delta_out = delta;
  return warp_sum_i(sum);
}

// Per-(query, cluster) constants of the estimator: A = Delta/sqrt(D'),
// B = v_l/sqrt(D'), E = ||q_r - c|| 2 eps0/sqrt(D'-1) and the additive term
// add: ||q_r - c||^2 for distances, -<q_r, c> for inner products (§6).
__device__ __forceinline__ float4 quant_meta(float delta, float vl, float nq2, float add,
                                             float eps0, int dpad) {
  const float sqd = __fsqrt_rn((float)dpad);
  const float keps = __fdiv_rn(__fmul_rn(2.0f, eps0), __fsqrt_rn((float)(dpad - 1)));
  const float n_q = __fsqrt_rn(nq2);
  return make_float4(__fdiv_rn(delta, sqd), __fdiv_rn(vl, sqd), __fmul_rn(n_q, keps), add);
}

// Quantize for the popcount scan: B_q bit-planes of q_u into shared memory.
__device__ __forceinline__ void quantize_probe(const FusedParams& P, const FusedSmem& S, int64_t q,
                                               int j, int jg, int c, float nq2, float add) {
  const int lane = threadIdx.x & 31;
  const int dpad = P.dpad, W = P.W, bq = P.bq;
  uint64_t* planes = S.planes + (size_t)j * bq * W;
  float vl, delta;
  const int sum = quant_core(
      P.rq + q * dpad, P.ptc + (int64_t)c * dpad, dpad, bq, P.seed, (uint64_t)(P.q_offset + q), c,
      &vl, &delta, [&](int i, int, const int* qu) {
        // the nibble of lane l sits at bits 4l..4l+3 of the 128-bit block
        for (int b = 0; b < bq; ++b) {
          const uint32_t nib = ((qu[0] >> b) & 1) | (((qu[1] >> b) & 1) << 1) |
                               (((qu[2] >> b) & 1) << 2) | (((qu[3] >> b) & 1) << 3);
          const uint32_t part = nib << (4 * (lane & 7));
          const uint32_t q0 = __reduce_or_sync(kFull, lane < 8 ? part : 0u);
          const uint32_t q1 = __reduce_or_sync(kFull, (lane >= 8 && lane < 16) ? part : 0u);
          const uint32_t q2 = __reduce_or_sync(kFull, (lane >= 16 && lane < 24) ? part : 0u);
          const uint32_t q3 = __reduce_or_sync(kFull, lane >= 24 ? part : 0u);
          if (lane == 0) {
            const int w0 = 2 * i;
            if (w0 < W) planes[b * W + w0] = ((uint64_t)q1 << 32) | q0;
            if (w0 + 1 < W) planes[b * W + w0 + 1] = ((uint64_t)q3 << 32) | q2;
          }
        }
      });
  if (lane == 0) {
    const float4 m = quant_meta(delta, vl, nq2, add, P.eps0, dpad);
    S.pmeta[j] = m;
    S.psum[j] = sum;
    S.pbeg[j] = P.bucket_off[c];
    S.pref[j + 1] = P.bucket_off[c + 1] - P.bucket_off[c];  // length; prefix-summed later
    if (P.tr.sum_qu) P.tr.sum_qu[q * P.nprobe + jg] = sum;
    if (P.tr.meta) {
      float* tm = P.tr.meta + (q * P.nprobe + jg) * 4;
      tm[0] = m.x; tm[1] = m.y; tm[2] = m.z; tm[3] = m.w;
    }
  }
  __syncwarp();
  if (P.tr.planes) {
    uint64_t* tp = P.tr.planes + (q * P.nprobe + jg) * (int64_t)bq * W;
    for (int t = lane; t < bq * W; t += 32) tp[t] = planes[t];
  }
}

// Warp-aggregated slot reservation: lanes with `want` get consecutive slots
// from one atomicAdd per warp (shared-memory counters are hot).
__device__ __forceinline__ int warp_reserve(bool want, int* counter) {
  const unsigned m = __ballot_sync(kFull, want);
  if (m == 0) return -1;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(counter, __popc(m));
  base = __shfl_sync(kFull, base, leader);
  return want ? base + __popc(m & ((1u << lane) - 1u)) : -1;
}


// ---------------------------------------------------------- block select
// The want-th smallest (1-based, want <= n) of the n keys a[0..n) by an
// MSD radix select, 8 bits per pass; histogram updates are aggregated per
// warp by digit. On return st.rem = how many keys equal to the result are
// among the `want` smallest. Whole block; synchronized on return.
template <class K, class F>
__device__ K block_select_f(int n, int want, SelState& st, F keyf) {
  constexpr int NB = (int)sizeof(K) * 8;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // The leading bits where the smallest and the largest key agree are common
  // to every key and need no histogram pass: one min/max pass finds them.
  K kmin = ~(K)0, kmax = 0;
  for (int i = tid; i < n; i += blockDim.x) {
    const K key = keyf(i);
    kmin = key < kmin ? key : kmin;
    kmax = key > kmax ? key : kmax;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const K a = __shfl_xor_sync(kFull, kmin, o), b = __shfl_xor_sync(kFull, kmax, o);
    kmin = a < kmin ? a : kmin;
    kmax = b > kmax ? b : kmax;
  }
  if (lane == 0) {
    st.wmin[wid] = kmin;
    st.wmax[wid] = kmax;
  }
  __syncthreads();
  kmin = ~(K)0;
  kmax = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    kmin = (K)st.wmin[w] < kmin ? (K)st.wmin[w] : kmin;
    kmax = (K)st.wmax[w] > kmax ? (K)st.wmax[w] : kmax;
  }
  if (kmin == kmax) {  // all keys equal: the answer, with every key a tie
    __syncthreads();
    if (tid == 0) {
      st.bin = (int)(kmin & 255);
      st.hist[st.bin] = n;
      st.rem = want;
    }
    __syncthreads();
    return kmin;
  }
  const K diff = kmin ^ kmax;
  const int top = NB - 1 - (sizeof(K) == 8 ? __clzll((long long)diff) : __clz((int)diff));
  const int start = (top / 8) * 8;  // the byte holding the highest differing bit
  K mask = start + 8 >= NB ? (K)0 : ~(((K)1 << (start + 8)) - 1);
  K prefix = kmin & mask;
  int rem = want;
  for (int shift = start; shift >= 0; shift -= 8) {
    for (int i = tid; i < 256; i += blockDim.x) st.hist[i] = 0;
    __syncthreads();
    for (int b0 = 0; b0 < n; b0 += blockDim.x) {
      const int i = b0 + tid;
      K key = 0;
      bool v = false;
      if (i < n) {
        key = keyf(i);
        v = (key & mask) == prefix;
      }
      const int dig = v ? (int)((key >> shift) & 255) : 256 + lane;
      const unsigned grp = __match_any_sync(kFull, dig);
      if (v && lane == __ffs(grp) - 1) atomicAdd(&st.hist[dig], __popc(grp));
    }
    __syncthreads();
    if (tid < 32) {
      int c[8], sum = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        c[u] = st.hist[lane * 8 + u];
        sum += c[u];
      }
      int incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      const unsigned hit = __ballot_sync(kFull, incl >= rem);
      if (lane == __ffs(hit) - 1) {
        int cum = incl - sum;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (cum + c[u] >= rem) {
            st.bin = lane * 8 + u;
            st.rem = rem - cum;
            break;
          }
          cum += c[u];
        }
      }
    }
    __syncthreads();
    prefix |= (K)st.bin << shift;
    mask |= (K)255 << shift;
    rem = st.rem;
    __syncthreads();
  }
  return prefix;
}

template <class K>
__device__ K block_select(const K* a, int n, int want, SelState& st) {
  return block_select_f<K>(n, want, st, [a](int i) { return a[i]; });
}

// The want-th smallest (1-based, want <= n) of n 32-bit keys: one histogram
// of kHistBins equal-width bins over [min, max] (bin = (key - min) kHistBins
// / (max - min + 1): monotone in the key, so the bins order the keys), then
// an exact selection among the keys of the boundary bin, collected into coll
// (ranked directly when they fit one per thread). rem = how many keys equal
// to the result are among the want smallest, eq = how many keys equal it in
// all. hist: kHistBins ints; coll: coll_cap keys. Falls back to the radix
// select when the boundary bin does not fit coll. Whole block (kThreads
// threads); synchronized on return.
constexpr int kHistBins = 1024;
template <class F>
__device__ uint32_t hist_select(int n, int want, SelState& st, int* hist, uint32_t* coll,
                                int coll_cap, int& rem, int& eq, F keyf) {
  static_assert(kHistBins == 4 * kThreads, "four bins per thread");
  __shared__ int s_hs[5];  // boundary bin, keys below it, fill, rem, eq
  __shared__ uint32_t s_T;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  uint32_t kmin = 0xffffffffu, kmax = 0u;
  for (int i = tid; i < n; i += blockDim.x) {
    const uint32_t key = keyf(i);
    kmin = key < kmin ? key : kmin;
    kmax = key > kmax ? key : kmax;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint32_t a = __shfl_xor_sync(kFull, kmin, o), b = __shfl_xor_sync(kFull, kmax, o);
    kmin = a < kmin ? a : kmin;
    kmax = b > kmax ? b : kmax;
  }
  if (lane == 0) {
    st.wmin[wid] = kmin;
    st.wmax[wid] = kmax;
  }
  __syncthreads();
  kmin = 0xffffffffu;
  kmax = 0u;
  for (int w = 0; w < nw; ++w) {
    kmin = (uint32_t)st.wmin[w] < kmin ? (uint32_t)st.wmin[w] : kmin;
    kmax = (uint32_t)st.wmax[w] > kmax ? (uint32_t)st.wmax[w] : kmax;
  }
  if (kmin == kmax) {  // all keys equal
    rem = want;
    eq = n;
    __syncthreads();
    return kmin;
  }
  const uint64_t span = (uint64_t)(kmax - kmin) + 1u;
  auto bin_of = [kmin, span](uint32_t key) {
    return (int)(((uint64_t)(key - kmin) * (uint64_t)kHistBins) / span);
  };
  for (int i = tid; i < kHistBins; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) atomicAdd(&hist[bin_of(keyf(i))], 1);
  __syncthreads();
  // the bin holding the want-th key: four bins per thread, block prefix sum
  int c[4], sum = 0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    c[u] = hist[4 * tid + u];
    sum += c[u];
  }
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) st.warp_cnt[wid] = incl;
  __syncthreads();
  for (int w = 0; w < wid; ++w) incl += st.warp_cnt[w];
  const int excl = incl - sum;
  if (excl < want && incl >= want) {  // exactly one thread
    int cum = excl;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (cum + c[u] >= want) {
        s_hs[0] = 4 * tid + u;
        s_hs[1] = cum;
        break;
      }
      cum += c[u];
    }
  }
  if (tid == 0) s_hs[2] = 0;
  __syncthreads();
  const int B = s_hs[0], below = s_hs[1], nB = hist[B], want_b = want - below;
  uint32_t T;
  if (nB <= coll_cap) {
    for (int b0 = 0; b0 < n; b0 += blockDim.x) {
      const int i = b0 + tid;
      uint32_t key = 0u;
      bool in = false;
      if (i < n) {
        key = keyf(i);
        in = bin_of(key) == B;
      }
      const int slot = warp_reserve(in, &s_hs[2]);
      if (in) coll[slot] = key;
    }
    __syncthreads();
    if (nB <= (int)blockDim.x) {  // rank each key of the bin against the others
      if (tid < nB) {
        const uint32_t mine = coll[tid];
        int lt = 0, le = 0;
        for (int j = 0; j < nB; ++j) {
          const uint32_t v = coll[j];
          lt += v < mine ? 1 : 0;
          le += v <= mine ? 1 : 0;
        }
        if (lt < want_b && want_b <= le) {  // the threads holding the result
          s_T = mine;
          s_hs[3] = want_b - lt;
          s_hs[4] = le - lt;
        }
      }
      __syncthreads();
      T = s_T;
      rem = s_hs[3];
      eq = s_hs[4];
    } else {
      T = block_select_f<uint32_t>(nB, want_b, st, [coll](int i) { return coll[i]; });
      rem = st.rem;
      eq = st.hist[st.bin];
    }
  } else {
    T = block_select_f<uint32_t>(n, want, st, keyf);
    rem = st.rem;
    eq = st.hist[st.bin];
  }
  __syncthreads();
  return T;
}

// In place, keep the keys below T and `ties` of the keys equal to T; returns
// the new count (whole block; synchronized on return).
template <class K>
__device__ int block_keep_below(K* a, int n, K T, int ties, SelState& st) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) st.tie_taken = 0;
  __syncthreads();
  int out = 0;
  for (int b0 = 0; b0 < n; b0 += blockDim.x) {
    const int i = b0 + tid;
    K key = 0;
    bool keep = false;
    if (i < n) {
      key = a[i];
      keep = key < T || (key == T && atomicAdd(&st.tie_taken, 1) < ties);
    }
    const unsigned bal = __ballot_sync(kFull, keep);
    if (lane == 0) st.warp_cnt[wid] = __popc(bal);
    __syncthreads();
    int before = out, tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      if (w < wid) before += st.warp_cnt[w];
      tot += st.warp_cnt[w];
    }
    if (keep) a[before + __popc(bal & ((1u << lane) - 1u))] = key;
    out += tot;
    __syncthreads();
  }
  return out;
}

// Keep the `keep` smallest of the *cnt keys (no order); returns the
// keep-th smallest key (or ~0 if there are fewer than keep keys).
template <class K>
__device__ K select_keep(K* a, int* cnt, int keep, SelState& st) {
  const int n = *cnt;
  if (n < keep) {
    __syncthreads();
    return ~(K)0;
  }
  const K T = block_select<K>(a, n, keep, st);
  const int kept = block_keep_below<K>(a, n, T, st.rem, st);
  if (threadIdx.x == 0) *cnt = kept;
  __syncthreads();
  return T;
}

// select_keep for 32-bit keys by the histogram select (hist, coll: shared
// memory the caller has free at this point).
__device__ uint32_t select_keep_h(uint32_t* a, int* cnt, int keep, SelState& st, int* hist,
                                  uint32_t* coll, int coll_cap) {
  const int n = *cnt;
  if (n < keep) {
    __syncthreads();
    return 0xffffffffu;
  }
  int rem = 0, eq = 0;
  const uint32_t T =
      hist_select(n, keep, st, hist, coll, coll_cap, rem, eq, [a](int i) { return a[i]; });
  const int kept = block_keep_below<uint32_t>(a, n, T, rem, st);
  if (threadIdx.x == 0) *cnt = kept;
  __syncthreads();
  return T;
}

// Keep the `keep` smallest of the *cnt distinct (distance key << 32 | id)
// keys of a: a 32-bit select on the distance half (by the histogram select
// when hist/coll are given, else the radix select), then -- only when more
// keys share the boundary distance than are kept -- one on the id half of
// those. Returns the keep-th smallest key (~0 if there are fewer than keep).
// Whole block; synchronized on return.
__device__ unsigned long long select_keep_dk(unsigned long long* a, int* cnt, int keep,
                                             SelState& st, int* hist = nullptr,
                                             uint32_t* coll = nullptr, int coll_cap = 0) {
  const int n = *cnt;
  if (n < keep) {
    __syncthreads();
    return ~0ull;
  }
  uint32_t Td;
  int ties = 0, eqn = 0;
  if (hist) {
    Td = hist_select(n, keep, st, hist, coll, coll_cap, ties, eqn,
                     [a](int i) { return (uint32_t)(a[i] >> 32); });
  } else {
    Td = block_select_f<uint32_t>(n, keep, st, [a](int i) { return (uint32_t)(a[i] >> 32); });
    ties = st.rem;
    eqn = st.hist[st.bin];
  }
  uint32_t Tid = 0xffffffffu;
  if (eqn > ties)
    Tid = block_select_f<uint32_t>(n, ties, st, [a, Td](int i) {
      return (uint32_t)(a[i] >> 32) == Td ? (uint32_t)(a[i] & 0xffffffffu) : 0xffffffffu;
    });
  unsigned long long T = ((unsigned long long)Td << 32) | Tid;
  if (Tid == 0xffffffffu) {  // every key at the boundary distance is kept
    T = ((unsigned long long)Td << 32) | 0xffffffffu;
  }
  const int kept = block_keep_below<unsigned long long>(a, n, T, 1, st);
  if (threadIdx.x == 0) *cnt = kept;
  __syncthreads();
  if (Tid == 0xffffffffu) {
    // the keep-th smallest key itself: the largest kept key
    __shared__ unsigned long long s_max;
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    unsigned long long mx = 0;
    for (int i = threadIdx.x; i < kept; i += blockDim.x) mx = a[i] > mx ? a[i] : mx;
    atomicMax(&s_max, mx);
    __syncthreads();
    T = s_max;
    __syncthreads();
  }
  return T;
}

// Sort the first pow2(keep) slots of a shared key buffer holding *cnt <=
// keep keys (padded with the maximum key). Whole block; synchronized on return.
__device__ __forceinline__ void sort_kept_u64(unsigned long long* a, int cnt, int keep) {
  int n = 1;
  while (n < keep) n <<= 1;
  for (int i = cnt + threadIdx.x; i < n; i += blockDim.x) a[i] = ~0ull;
  __syncthreads();
  block_bitonic_sort_u64(a, n);
  __syncthreads();
}

// In-place, order-keeping compaction of the candidate list with predicate f:
// blocks of kCompactU x blockDim entries (kCompactU loads in flight per
// thread, two barriers per block); every read of a block precedes its
// writes, which land below the block's end. scratch: kCompactU x
// (blockDim / 32) ints. (Two entries per thread: four cost the fused kernel
// register spills that outweighed the fewer barriers.)
constexpr int kCompactU = 2;
template <class F>
__device__ __forceinline__ void compact_cand(int4* cand, int* cnt, int cap, int* scratch, F keep_f) {
  const int n = min(*cnt, cap);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned below = (1u << lane) - 1u;
  int out = 0;
  __syncthreads();
  for (int b = 0; b < n; b += kCompactU * blockDim.x) {
    int4 e[kCompactU];
    bool keep[kCompactU];
#pragma unroll
    for (int u = 0; u < kCompactU; ++u) {
      const int i = b + u * blockDim.x + threadIdx.x;
      e[u] = make_int4(0, 0, 0, 0);
      keep[u] = false;
      if (i < n) {
        e[u] = cand[i];
        keep[u] = keep_f(e[u]);
      }
    }
    unsigned bal[kCompactU];
#pragma unroll
    for (int u = 0; u < kCompactU; ++u) {
      bal[u] = __ballot_sync(kFull, keep[u]);
      if (lane == 0) scratch[u * nw + wid] = __popc(bal[u]);
    }
    __syncthreads();
    // entry (u, thread) follows every kept entry of sub-blocks < u and of
    // the warps before it in sub-block u
#pragma unroll
    for (int u = 0; u < kCompactU; ++u) {
      int before = out, tot = 0;
      for (int w = 0; w < nw; ++w) {
        const int c = scratch[u * nw + w];
        if (w < wid) before += c;
        tot += c;
      }
      if (keep[u]) cand[before + __popc(bal[u] & below)] = e[u];
      out += tot;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *cnt = out;
  __syncthreads();
}

// One term of the canonical exact score: squared distance, fold of
// (q - x)^2; inner product, fold of q x (negated at the end).
template <bool IP>
__device__ __forceinline__ float score_step(float acc, float q, float x) {
  if (IP) return __fmaf_rn(q, x, acc);
  const float t = __fsub_rn(q, x);
  return __fmaf_rn(t, t, acc);
}

// Canonical exact score of row x against the query qv (shared memory), in
// ascending dimension order: ||q - x||^2, or -<q, x> for inner products.
// 32-byte loads, four in flight, when d is a multiple of 8 (rows, in
// cudaMalloc'ed arrays, then start on 32-byte boundaries); 16-byte loads,
// eight in flight, when d is a multiple of 4.
template <bool IP>
__device__ __forceinline__ float row_score(const float* __restrict__ x, const float* qv, int d) {
  float acc = 0.0f;
  if ((d & 7) == 0) {
    // (qv: 16-byte aligned shared memory, read as float4)
    const float4* q4 = reinterpret_cast<const float4*>(qv);
    auto fold8 = [&](const unsigned long long (&v)[4], int c) {
      const float4 qa = q4[c >> 2], qb = q4[(c >> 2) + 1];
      const float qq[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
#pragma unroll
      for (int e = 0; e < 8; ++e)
        acc = score_step<IP>(acc, qq[e], __int_as_float((int)(uint32_t)(v[e >> 1] >> (32 * (e & 1)))));
    };
    int c = 0;
    for (; c + 32 <= d; c += 32) {
      unsigned long long v[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        asm volatile("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];"
                     : "=l"(v[u][0]), "=l"(v[u][1]), "=l"(v[u][2]), "=l"(v[u][3])
                     : "l"(x + c + 8 * u));
#pragma unroll
      for (int u = 0; u < 4; ++u) fold8(v[u], c + 8 * u);
    }
    for (; c < d; c += 8) {
      unsigned long long v[4];
      asm volatile("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];"
                   : "=l"(v[0]), "=l"(v[1]), "=l"(v[2]), "=l"(v[3])
                   : "l"(x + c));
      fold8(v, c);
    }
  } else if ((d & 3) == 0) {
    const float4* x4 = reinterpret_cast<const float4*>(x);
    const float4* q4 = reinterpret_cast<const float4*>(qv);
    int c = 0;
    for (; c + 8 <= (d >> 2); c += 8) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldg(x4 + c + u);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float4 qq = q4[c + u];
        acc = score_step<IP>(acc, qq.x, v[u].x);
        acc = score_step<IP>(acc, qq.y, v[u].y);
        acc = score_step<IP>(acc, qq.z, v[u].z);
        acc = score_step<IP>(acc, qq.w, v[u].w);
      }
    }
    for (; c < (d >> 2); ++c) {
      const float4 vv = __ldg(x4 + c), qq = q4[c];
      acc = score_step<IP>(acc, qq.x, vv.x);
      acc = score_step<IP>(acc, qq.y, vv.y);
      acc = score_step<IP>(acc, qq.z, vv.z);
      acc = score_step<IP>(acc, qq.w, vv.w);
    }
  } else {
    for (int dd = 0; dd < d; ++dd) acc = score_step<IP>(acc, qv[dd], __ldg(x + dd));
  }
  return IP ? -acc : acc;
}

// Exact scores of a list of rows: each lane streams its own row (a warp has
// 256 rows' worth of loads outstanding) and folds it in ascending dimension
// order. Keys (score, id) go to the top-k buffer.
// SRC 0: the pilot (ids in S.estk); SRC 1: the candidate list (positions).
// kmax: keys above it cannot enter the result and are not kept (the rest
// of the re-rank set, once the pilot's k smallest keys are known).
template <int SRC>
__device__ void rerank_rows(const FusedParams& P, const FusedSmem& S, int64_t q, int count,
                            const int4* cand, int* top_cnt, int* surv_cnt,
                            unsigned long long kmax = ~0ull) {
  const int d = P.d;
  // Ask L2 for the rows of the first two rounds (no registers held, no
  // waiting): their loads then find most rows in L2 instead of waiting on
  // DRAM four loads at a time. (Asking for a whole set of thousands of rows
  // at once, or two rounds ahead every round, measured slower.)
  const int row_bytes = d * (int)sizeof(float);
  for (int i = threadIdx.x; i < min(count, 2 * (int)blockDim.x); i += blockDim.x) {
    const int pos = SRC == 0 ? (int)(S.estk[i] & 0xffffffffu) : (cand[i].x & 0x7fffffff);
    const char* x = reinterpret_cast<const char*>(P.data_b + (int64_t)pos * d);
    for (int o = 0; o < row_bytes; o += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(x + o));
  }
  for (int r0 = 0; r0 < count; r0 += blockDim.x) {
    const int i = r0 + threadIdx.x;
    const bool valid = i < count;
    int pos = 0, id = 0;
    if (valid) {
      if (SRC == 0) {
        const unsigned long long e = S.estk[i];
        id = (int)(e >> 32);
        pos = (int)(e & 0xffffffffu);
      } else {
        pos = cand[i].x & 0x7fffffff;
        id = P.perm[pos];
      }
    }
    float acc = 0.0f;
    if (valid) {
      const float* x = P.data_b + (int64_t)pos * d;
      acc = P.metric ? row_score<true>(x, S.qv, d) : row_score<false>(x, S.qv, d);
    }
    const unsigned long long key = ((unsigned long long)float_key(acc) << 32) | (uint32_t)id;
    const bool take = valid && key <= kmax;
    const int slot = warp_reserve(take, top_cnt);
    if (take) S.topk[slot] = key;
    if (valid) {
      const int si = i + (SRC == 0 ? 0 : *surv_cnt);
      if (P.tr.surv_ids && si < P.tr.surv_cap) P.tr.surv_ids[q * P.tr.surv_cap + si] = id;
    }
    __syncthreads();
    const int tc = *top_cnt;  // read between barriers (see the scan's upkeep)
    __syncthreads();
    if (tc > P.ct - (int)blockDim.x) select_keep_dk(S.topk, top_cnt, P.k, *S.sel);
  }
  __syncthreads();
  if (threadIdx.x == 0) *surv_cnt += count;
  __syncthreads();
}

// ------------------------------------------------------------ probe selection
// The nsel nearest centroids of each query (§4's probe; for inner products
// the largest <q_r, c>), exactly as a full canonical scan would rank them,
// from tensor-core scores. For centroid c the TF32 product <q, c>~ (inputs
// rounded to 10-bit mantissas, FP32 accumulation) gives the approximate score
// s~ = ||q||^2 + ||c||^2 - 2 <q, c>~ (or -<q, c>~), within eps_c of the
// canonical FP32 score (the bound is derived below). U_c = s~ + eps_c is an
// upper and L_c = s~ - eps_c a lower bound of c's canonical score, so any T
// at least the nsel-th smallest upper bound is at least the nsel-th smallest
// canonical score, and every centroid of the exact top nsel has L_c <= T --
// the same bound-and-filter step as the paper's re-ranking (§4). T is the
// nsel-th smallest of a pool of upper bounds (the kProbePool smallest of
// every 128 centroids, taken in the tensor-core kernel's epilogue),
// or, when nsel exceeds the pool, the upper edge of the histogram bin of all
// upper bounds that holds the nsel-th smallest. The candidates with
// L_c <= T get their canonical scores (the fold the full scan uses) and the
// nsel smallest (score, id) are written in order.
// If the candidates exceed the shared-memory list, the row select ranks every
// centroid by its canonical score (computed on the fly). keys: nq x K keys
// of U_c, formed in the tensor-core kernel's epilogue (probe_keys_tc) with
// eps_c from ProbeEps and each query's FP32 ||q||^2 (nq2), together with
// the pool (pool_n keys per query) and each query's key range [kmin, kmax]
// (read only).
//
// The bound: |t - x| <= 2^-11 |x| for each TF32 operand t, the products of
// two TF32 values are exact in FP32, and the accumulation of d products in
// FP32 is taken to lose at most (d + 2) 2^-21 of sum |q_i c_i| <= ||q|| ||c||
// (four units of FP32 rounding per addition, to cover accumulation orders the
// hardware does not document), so |<q,c>~ - <q,c>| <= a ||q|| ||c|| with
// a = 2^-10 + (d + 2) 2^-21. The canonical dot and squared distance are
// within d 2^-23 ||q|| ||c|| and (d + 2) 2^-24 (||q|| + ||c||)^2 of exact,
// and the FP32 operations forming s~, U and L add a few units of
// 2^-24 (||q|| + ||c||)^2; eps_c takes all of these with a 5% margin.
constexpr int kProbeCandMax = 2048;  // candidates kept in shared memory

__global__ void __launch_bounds__(kThreads) probe_select_kernel(
    const float* __restrict__ Q, int d, const uint32_t* __restrict__ keys,
    const uint32_t* __restrict__ pool, int pool_n, const uint32_t* __restrict__ kmin_q,
    const uint32_t* __restrict__ kmax_q, const float* __restrict__ nq2_q,
    const float* __restrict__ C, const float* __restrict__ cnorm,
    const float* __restrict__ cnorm_max, int K, int metric, int nprobe,
    const int32_t* __restrict__ nprobe_q, int sort_n, const int32_t* __restrict__ pre_ids,
    const float* __restrict__ pre_dist, int pre_n, int32_t* __restrict__ out_ids,
    float* __restrict__ out_dist) {
  extern __shared__ __align__(16) unsigned char psm[];
  // layout: q (d floats) | the pool (pool_n entries) | work area: the
  // histogram, then the candidates, or the fallback's sort buffer
  float* qs = reinterpret_cast<float*>(psm);
  uint32_t* sp = reinterpret_cast<uint32_t*>(psm + align_up(sizeof(float) * d, 16));
  unsigned char* work = psm + align_up(sizeof(float) * d, 16) + align_up(sizeof(uint32_t) * pool_n, 16);
  __shared__ SelState st;
  __shared__ int s_nc, s_bin, s_np, s_nsat;
  __shared__ uint32_t s_pmin, s_pmax;
  __shared__ int s_sat[64];  // saturated groups of 128 centroids (scanned in full)
  const int q = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const float* qg = Q + (int64_t)q * d;
  const uint32_t* row = keys + (int64_t)q * K;
  int nsel = nprobe;
  if (nprobe_q) nsel = min(max(nprobe_q[q], 1), nprobe);
  nsel = min(nsel, K);
  if (pre_ids && nsel <= pre_n) {
    // a list of this query's pre_n best is already selected: its prefix is
    // the answer (the same order by (score, id))
    for (int j = tid; j < nprobe; j += blockDim.x) {
      const bool ok = j < nsel;
      out_ids[(int64_t)q * nprobe + j] = ok ? pre_ids[(int64_t)q * pre_n + j] : -1;
      out_dist[(int64_t)q * nprobe + j] =
          ok ? pre_dist[(int64_t)q * pre_n + j] : __int_as_float(0x7f800000);
    }
    return;
  }
  for (int i = tid; i < d; i += blockDim.x) qs[i] = qg[i];
  if (tid == 0) {
    s_nc = 0;
    s_np = 0;
    s_nsat = 0;
    s_pmin = 0xffffffffu;
    s_pmax = 0u;
  }
  const ProbeEps eps(metric, __fsqrt_rn(nq2_q[q]), d);
  constexpr int kSelU = 8;  // keys per thread in flight in a pass
  int* hist = reinterpret_cast<int*>(work);
  for (int i = tid; i < kHistBins; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  // the pool, with the number and range of its real entries (an entry is
  // at least its centroid's key: the key rounded up, then the index bits)
  {
    int cnt = 0;
    uint32_t pmin = 0xffffffffu, pmax = 0u;
    for (int i = tid; i < pool_n; i += blockDim.x) {
      const uint32_t e = __ldg(pool + (int64_t)q * pool_n + i);
      sp[i] = e;
      if (e != 0xffffffffu) {
        ++cnt;
        pmin = e < pmin ? e : pmin;
        pmax = e > pmax ? e : pmax;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      cnt += __shfl_xor_sync(kFull, cnt, o);
      const uint32_t a = __shfl_xor_sync(kFull, pmin, o), b = __shfl_xor_sync(kFull, pmax, o);
      pmin = a < pmin ? a : pmin;
      pmax = b > pmax ? b : pmax;
    }
    if (lane == 0) {
      atomicAdd(&s_np, cnt);
      atomicMin(&s_pmin, pmin);
      atomicMax(&s_pmax, pmax);
    }
  }
  __syncthreads();
  const bool from_pool = nsel <= s_np;
  // T bounds the nsel-th smallest upper bound of all centroids from above.
  // From the pool (distinct centroids): the last value of the histogram bin
  // (over the pool's range) holding the nsel-th smallest entry, so at least
  // nsel centroids have keys <= T. Otherwise: the same over all K keys.
  const uint32_t kmin = from_pool ? s_pmin : kmin_q[q], kmax = from_pool ? s_pmax : kmax_q[q];
  const uint32_t span1 = kmax - kmin;  // span - 1
  int shift = 0;
  while ((span1 >> shift) >= (uint32_t)kHistBins) ++shift;
  if (from_pool) {
    for (int i = tid; i < pool_n; i += blockDim.x) {
      const uint32_t e = sp[i];
      if (e != 0xffffffffu) atomicAdd(&hist[(e - kmin) >> shift], 1);
    }
  } else {
    for (int c0 = 0; c0 < K; c0 += kSelU * blockDim.x) {
      uint32_t kv[kSelU];
#pragma unroll
      for (int u = 0; u < kSelU; ++u) {
        const int c = c0 + u * blockDim.x + tid;
        kv[u] = c < K ? __ldg(row + c) : 0u;
      }
#pragma unroll
      for (int u = 0; u < kSelU; ++u) {
        const int c = c0 + u * blockDim.x + tid;
        if (c < K) atomicAdd(&hist[(kv[u] - kmin) >> shift], 1);
      }
    }
  }
  __syncthreads();
  {
    int cb[4], sum = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      cb[u] = hist[4 * tid + u];
      sum += cb[u];
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) st.warp_cnt[wid] = incl;
    __syncthreads();
    for (int w = 0; w < wid; ++w) incl += st.warp_cnt[w];
    const int excl = incl - sum;
    if (excl < nsel && incl >= nsel) {  // exactly one thread
      int cum = excl;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (cum + cb[u] >= nsel) {
          s_bin = 4 * tid + u;
          break;
        }
        cum += cb[u];
      }
    }
  }
  __syncthreads();
  // keys of bin B are at most kmin + ((B + 1) << shift) - 1
  const uint64_t edge = (uint64_t)kmin + ((uint64_t)(s_bin + 1) << shift) - 1u;
  const uint32_t T = (uint32_t)min((uint64_t)kmax, edge);
  // Candidates, L_c <= T (ids now, (score key, id) after the refine).
  // L_c = U_c - 2 eps_c (its rounding is inside the bound's margin) needs
  // ||c||; since eps_c is at most eps(max ||c||), only keys U_c <= Tpre =
  // T + 2 eps(max ||c||) (with a margin for the rounding of the subtraction)
  // can pass. From the pool: a group of 128 centroids whose largest pooled
  // entry, rounded down to its key part, is <= Tpre + 128 may hold more
  // such keys (an entry's key part exceeds its key by less than 128) and is
  // scanned in full; the others' keys <= Tpre are all pooled, and a pooled
  // entry whose key part is <= Tpre + 128 has its exact key read.
  const float Tf = key_float(T), e2max = __fmul_rn(2.0f, eps(__ldg(cnorm_max)));
  const uint32_t Tpre =
      float_key(__fadd_ru(__fadd_ru(Tf, e2max), __fmul_ru(0x1.0p-20f, __fadd_ru(fabsf(Tf), e2max))));
  unsigned long long* ckey = reinterpret_cast<unsigned long long*>(work);
  __syncthreads();  // (the histogram is read)
  auto consider = [&](bool pass_pre, int c) {
    bool in = false;
    if (pass_pre)
      in = float_key(__fsub_rn(key_float(row[c]), __fmul_rn(2.0f, eps(__ldg(cnorm + c))))) <= T;
    const int slot = warp_reserve(in, &s_nc);
    if (in && slot < kProbeCandMax) ckey[slot] = (unsigned long long)(uint32_t)c;
  };
  bool scan_all = !from_pool;
  if (from_pool) {
    const uint64_t lim = (uint64_t)Tpre + 128u;
    for (int i0 = 0; i0 < pool_n; i0 += blockDim.x) {
      const int i = i0 + tid;
      bool pre = false;
      int c = 0;
      if (i < pool_n) {
        const uint32_t e = sp[i];
        const int g = i / kProbePool, j = i % kProbePool;
        const uint32_t last = sp[g * kProbePool + kProbePool - 1];
        const bool sat = last != 0xffffffffu && (uint64_t)(last & ~127u) <= lim;
        if (sat && j == 0) {
          const int slot = atomicAdd(&s_nsat, 1);
          if (slot < 64) s_sat[slot] = g;
        }
        c = g * 128 + (int)(e & 127u);
        pre = !sat && e != 0xffffffffu && (uint64_t)(e & ~127u) <= lim;
      }
      consider(pre && row[c] <= Tpre, c);
    }
    __syncthreads();
    const int nsat = s_nsat;
    if (nsat > 64) {
      scan_all = true;  // many saturated groups: one pass over all keys instead
      __syncthreads();
      if (tid == 0) s_nc = 0;
      __syncthreads();
    } else {
      for (int t = 0; t < nsat; ++t) {
        const int g = s_sat[t];
        for (int c0 = g * 128; c0 < min(K, g * 128 + 128); c0 += blockDim.x) {
          const int c = c0 + tid;
          const bool ok = c < min(K, g * 128 + 128);
          consider(ok && row[c] <= Tpre, ok ? c : 0);
        }
      }
    }
  }
  if (scan_all) {
    for (int c0 = 0; c0 < K; c0 += kSelU * blockDim.x) {
      uint32_t kv[kSelU];
#pragma unroll
      for (int u = 0; u < kSelU; ++u) {
        const int c = c0 + u * blockDim.x + tid;
        kv[u] = c < K ? __ldg(row + c) : 0xffffffffu;
      }
#pragma unroll
      for (int u = 0; u < kSelU; ++u) {
        const int c = c0 + u * blockDim.x + tid;
        consider(c < K && kv[u] <= Tpre, c < K ? c : 0);
      }
    }
  }
  __syncthreads();
  const int nc = s_nc;
  int32_t* oid = out_ids + (int64_t)q * nprobe;
  float* od = out_dist + (int64_t)q * nprobe;
  if (nc <= kProbeCandMax) {
    // canonical scores of the candidates (one thread each, the full scan's
    // fold); every line of their rows is requested first
    for (int i = tid; i < nc; i += blockDim.x) {
      const char* x = reinterpret_cast<const char*>(C + (int64_t)(uint32_t)ckey[i] * d);
      for (int o = 0; o < d * (int)sizeof(float); o += 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(x + o));
    }
    for (int i = tid; i < nc; i += blockDim.x) {
      const int c = (int)(uint32_t)ckey[i];
      const float* x = C + (int64_t)c * d;
      const float a = metric ? row_score<true>(x, qs, d) : row_score<false>(x, qs, d);
      ckey[i] = ((unsigned long long)float_key(a) << 32) | (uint32_t)c;
    }
    __syncthreads();
    // rank each candidate among all of them (distinct keys: the ids differ)
    for (int i = tid; i < nc; i += blockDim.x) {
      const unsigned long long mine = ckey[i];
      int r = 0;
      for (int j = 0; j < nc; ++j) r += ckey[j] < mine ? 1 : 0;
      if (r < nsel) {
        oid[r] = (int32_t)(mine & 0xffffffffu);
        od[r] = key_float((uint32_t)(mine >> 32));
      }
    }
    for (int j = nsel + tid; j < nprobe; j += blockDim.x) {
      oid[j] = -1;
      od[j] = __int_as_float(0x7f800000);
    }
  } else {
    // too many candidates: the row select over canonical scores computed on
    // the fly (every pass refolds them; a rare path)
    select_row(
        [qs, C, d, metric](int c) {
          const float* x = C + (int64_t)c * d;
          return metric ? row_score<true>(x, qs, d) : row_score<false>(x, qs, d);
        },
        K, nsel, nprobe, sort_n, reinterpret_cast<unsigned long long*>(work), oid, od);
  }
}

// Shared memory of probe_select_kernel for dimension d, sort size sort_n and
// pool_n pooled entries.
inline size_t probe_select_smem(int d, int sort_n, int pool_n) {
  const size_t work = std::max({sizeof(int) * kHistBins, sizeof(unsigned long long) * kProbeCandMax,
                                sizeof(unsigned long long) * (size_t)sort_n});
  return align_up(sizeof(float) * d, 16) + align_up(sizeof(uint32_t) * (size_t)pool_n, 16) + work;
}

// Shared counters the per-query finishing step works with.
struct TailShared {
  int* cand_cnt;
  int* top_cnt;
  int* surv;
  int* scratch;  // kCompactU x kThreads / 32 ints
};

// The per-query end of the search (§4, reading R1): given the list of
// candidates {position, LB, estimate, UB} that contains every code with
// LB <= tau_ub, keep LB <= tau_ub; pilot = the m smallest (estimate, id);
// exact distances of the pilot give tau1; tau = min(tau_ub, tau1); exact
// distances of the other codes with LB <= tau; top-k by (distance, id).
// The pilot mark is bit 31 of the position. Whole block.
__device__ void finish_query(const FusedParams& P, const FusedSmem& S, int64_t q, int4* cand,
                             int cand_cap, float tau_ub, const TailShared& ts,
                             bool filtered = false) {
  const int tid = threadIdx.x;
  const int k = P.k, m = P.m;
  if (tid == 0) {
    *ts.top_cnt = 0;
    *ts.surv = 0;
  }
  __syncthreads();
  if (!filtered)  // (a list staged with LB <= tau_ub is already filtered)
    compact_cand(cand, ts.cand_cnt, cand_cap, ts.scratch,
                 [tau_ub](const int4& e) { return __int_as_float(e.y) <= tau_ub; });
  // pilot: the m smallest (estimate, id) of the list
  const int nl = *ts.cand_cnt;
  const bool pilot_all = nl <= m;
  uint32_t T_e = 0xffffffffu, T_id = 0xffffffffu;
  if (!pilot_all) {
    // the top-k buffer is free until the pilot's re-rank: histogram and
    // boundary-bin keys go there
    int ties = 0, eqn = 0;
    T_e = hist_select(nl, m, *S.sel, reinterpret_cast<int*>(S.topk),
                      reinterpret_cast<uint32_t*>(S.topk) + kHistBins, 2 * P.ct - kHistBins, ties,
                      eqn, [cand](int i) { return float_key(__int_as_float(cand[i].z)); });
    // among the list entries whose estimate equals the m-th one, the
    // `ties` smallest ids belong to the pilot; when all of them belong (the
    // usual case: one entry) no id selection is needed
    if (eqn > ties)
      T_id = block_select_f<uint32_t>(nl, ties, *S.sel, [cand, T_e, &P](int i) {
        const int4 e = cand[i];
        return float_key(__int_as_float(e.z)) == T_e ? (uint32_t)__ldg(P.perm + e.x) : 0xffffffffu;
      });
  }
  // write the pilot's (id, position) pairs to the pilot list, mark them
  __shared__ int s_pilot;
  if (tid == 0) s_pilot = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nl; b0 += blockDim.x) {
    const int i = b0 + tid;
    bool in = false;
    int4 e = make_int4(0, 0, 0, 0);
    if (i < nl) {
      e = cand[i];
      const uint32_t ek = float_key(__int_as_float(e.z));
      in = pilot_all || ek < T_e || (ek == T_e && (uint32_t)__ldg(P.perm + e.x) <= T_id);
    }
    const int slot = warp_reserve(in, &s_pilot);
    if (in) {
      S.estk[slot] = (uint32_t)e.x;
      cand[i].x = e.x | (int)0x80000000;
    }
  }
  __syncthreads();
  const int pilot = s_pilot;
  // the pilot's ids, all loads in flight together
  for (int i = tid; i < pilot; i += blockDim.x) {
    const unsigned long long e = S.estk[i];
    S.estk[i] = ((unsigned long long)(uint32_t)__ldg(P.perm + (uint32_t)e) << 32) | e;
  }
  __syncthreads();
  // exact distances of the pilot; tau1 = k-th smallest of them
  rerank_rows<0>(P, S, q, pilot, cand, ts.top_cnt, ts.surv);
  // tau1: the k-th smallest exact distance of the pilot; only the k smallest
  // pilot keys can be in the result, so the rest are dropped here
  // (the pilot list is free now and holds the histogram when large enough;
  // the upper-bound buffer, free since tau_ub, holds the boundary keys)
  const bool hsel = 2 * P.ce >= kHistBins && P.cu >= 256;
  const unsigned long long T1 =
      (pilot >= k) ? select_keep_dk(S.topk, ts.top_cnt, k, *S.sel,
                                    hsel ? reinterpret_cast<int*>(S.estk) : nullptr, S.ubk, P.cu)
                   : ~0ull;
  const float tau1 = (pilot >= k) ? key_float((uint32_t)(T1 >> 32)) : __int_as_float(0x7f800000);
  const float tau = fminf(tau_ub, tau1);
  // the rest of the re-rank set: LB <= tau, outside the pilot
  compact_cand(cand, ts.cand_cnt, cand_cap, ts.scratch,
               [tau](const int4& e) { return e.x >= 0 && __int_as_float(e.y) <= tau; });
  // with k pilot keys kept, a key above the k-th of them cannot be in the
  // result (keys are distinct): such keys are not kept
  rerank_rows<1>(P, S, q, *ts.cand_cnt, cand, ts.top_cnt, ts.surv, T1);
  const int n_top = *ts.top_cnt;
  if (n_top <= (int)blockDim.x) {
    // few keys (the usual case): each thread ranks its key against all of
    // them (distinct keys, so the ranks are a permutation) and writes it to
    // its place in the result
    const bool has = tid < n_top;
    const unsigned long long mine = has ? S.topk[tid] : 0ull;
    int r = 0;
    if (has)
      for (int j2 = 0; j2 < n_top; ++j2) r += S.topk[j2] < mine ? 1 : 0;
    if (has && r < k) {
      P.out_ids[q * k + r] = (int64_t)(mine & 0xffffffffu);
      const float v = key_float((uint32_t)(mine >> 32));
      P.out_dist[q * k + r] = P.metric ? -v : v;  // inner products: <o_r, q_r>
    }
    for (int j2 = n_top + tid; j2 < k; j2 += blockDim.x) {
      P.out_ids[q * k + j2] = -1;
      P.out_dist[q * k + j2] = P.metric ? __int_as_float(0xff800000) : __int_as_float(0x7f800000);
    }
  } else {
    select_keep_dk(S.topk, ts.top_cnt, k, *S.sel);
    const int got = min(*ts.top_cnt, k);
    sort_kept_u64(S.topk, got, k);
    for (int j2 = tid; j2 < k; j2 += blockDim.x) {
      const bool ok = j2 < got;
      P.out_ids[q * k + j2] = ok ? (int64_t)(S.topk[j2] & 0xffffffffu) : -1;
      const float v = ok ? key_float((uint32_t)(S.topk[j2] >> 32)) : __int_as_float(0x7f800000);
      P.out_dist[q * k + j2] = P.metric ? -v : v;  // inner products: <o_r, q_r>, -inf pads
    }
  }
  if (tid == 0) {
    if (P.tr.tau_ub) P.tr.tau_ub[q] = tau_ub;
    if (P.tr.tau1) P.tr.tau1[q] = tau1;
    if (P.tr.tau) P.tr.tau[q] = tau;
    if (P.tr.n_surv) P.tr.n_surv[q] = *ts.surv;
  }
  __syncthreads();
}

// Code words of one code held in registers (WT > 0: compile-time length,
// loaded as 16-byte vectors; WT = 0: generic length, read in place).
template <int WT>
struct CodeRegs {
  uint64_t c[WT > 0 ? WT : 1];
};

template <int WT>
__device__ __forceinline__ void load_code(CodeRegs<WT>& r, const uint64_t* __restrict__ code) {
  if constexpr (WT == 4) {  // one 32-byte load (codes are 32-byte aligned)
    asm volatile("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];"
                 : "=l"(r.c[0]), "=l"(r.c[1]), "=l"(r.c[2]), "=l"(r.c[3])
                 : "l"(code));
  } else if constexpr (WT > 0) {
    if constexpr (WT % 2 == 0) {
#pragma unroll
      for (int w = 0; w < WT; w += 2) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(code) + w / 2);
        r.c[w] = ((uint64_t)v.y << 32) | v.x;
        r.c[w + 1] = ((uint64_t)v.w << 32) | v.z;
      }
    } else {
#pragma unroll
      for (int w = 0; w < WT; ++w) r.c[w] = __ldg(code + w);
    }
  }
}

// <x_b, q_u> of one code against the bit-planes of its probe (§3.3.2):
// sum_j 2^j popcount(x_b AND q_u^(j)), unrolled for a compile-time code length
// (WT words) and B_q (BQT planes); WT = 0 / BQT = 0 use the runtime values.
template <int WT, int BQT>
__device__ __forceinline__ int code_ip(const CodeRegs<WT>& r, const uint64_t* __restrict__ code,
                                       const uint64_t* pl, int W, int bq) {
  if constexpr (WT > 0 && BQT > 0) {
    int ip = 0;
#pragma unroll
    for (int b = 0; b < BQT; ++b) {
      uint64_t pw[WT];
      if constexpr (WT % 2 == 0) {
#pragma unroll
        for (int w = 0; w < WT; w += 2) {
          const uint4 v = *reinterpret_cast<const uint4*>(pl + b * WT + w);
          pw[w] = ((uint64_t)v.y << 32) | v.x;
          pw[w + 1] = ((uint64_t)v.w << 32) | v.z;
        }
      } else {
#pragma unroll
        for (int w = 0; w < WT; ++w) pw[w] = pl[b * WT + w];
      }
      int pb = 0;
#pragma unroll
      for (int w = 0; w < WT; ++w) pb += __popcll(r.c[w] & pw[w]);
      ip += pb << b;
    }
    return ip;
  } else {
    int ip = 0;
    for (int b = 0; b < bq; ++b) {
      int pb = 0;
      for (int w = 0; w < W; ++w) pb += __popcll(code[w] & pl[b * W + w]);
      ip += pb << b;
    }
    return ip;
  }
}

// <x_b, q_u> of two codes of the same probe: each plane word is read from
// shared memory once for both (D' = 128 / 256, B_q = 4).
template <int WT>
__device__ __forceinline__ void code_ip2(const CodeRegs<WT>& r0, const CodeRegs<WT>& r1,
                                         const uint64_t* pl, int& i0, int& i1) {
  i0 = 0;
  i1 = 0;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    uint64_t pw[WT];
#pragma unroll
    for (int w = 0; w < WT; w += 2) {
      const uint4 v = *reinterpret_cast<const uint4*>(pl + b * WT + w);
      pw[w] = ((uint64_t)v.y << 32) | v.x;
      pw[w + 1] = ((uint64_t)v.w << 32) | v.z;
    }
    int p0 = 0, p1 = 0;
#pragma unroll
    for (int w = 0; w < WT; ++w) {
      p0 += __popcll(r0.c[w] & pw[w]);
      p1 += __popcll(r1.c[w] & pw[w]);
    }
    i0 += p0 << b;
    i1 += p1 << b;
  }
}

constexpr int kPPT = 4;  // most appends per thread between two buffer upkeeps (sizing)

// Pairs per thread per round: two (four cost spills at the four-CTA register
// budget), one for codes longer than 512 bits.
template <int WT>
__host__ __device__ constexpr int pairs_per_thread() {
  return WT == 0 ? 2 : (WT <= 4 ? 2 : (WT <= 8 ? 2 : 1));
}

// Residency: 4 CTAs per SM for the short codes (D' <= 256), 3 otherwise.
template <int WT>
constexpr int fused_min_blocks() {
  return (WT > 0 && WT <= 4) ? 4 : 3;
}

// ---- bulk-copy staging of the scan rounds (STG kernels, D' = 128 / 256)
// Round r of a probe chunk covers pairs [r * step, (r + 1) * step) of the
// chunk's pair sequence (probe order, then bucket order); their codes and
// factors are runs of consecutive bucket positions, one run per probed
// bucket the round touches. Warp 0 copies the runs of round r + 1 into the
// other of two shared-memory stages with cp.async.bulk (one per run and
// array, completion counted in bytes on the stage's mbarrier) while the
// block evaluates round r from its stage. Every wait is bounded (about a
// second); a wait that expires sets the error flag to 2.
__device__ __forceinline__ bool stage_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t b = smem_u32(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(b), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}

// Issue the copies of pairs [b0, b0 + cnt) of the chunk into stage buf
// (codes at stg + buf * step * CB, factors after both code stages). Warp 0.
template <int WT>
__device__ __forceinline__ void stage_issue(const FusedParams& P, const FusedSmem& S,
                                            unsigned char* stg, uint64_t* bars, int b0, int cnt,
                                            int npc, int buf, int step) {
  constexpr int CB = WT * 8;  // code bytes
  const int lane = threadIdx.x & 31;
  const uint32_t dc = smem_u32(stg) + (uint32_t)(buf * step * CB);
  const uint32_t df = smem_u32(stg) + (uint32_t)(2 * step * CB + buf * step * 16);
  const uint32_t bar = smem_u32(&bars[buf]);
  if (lane == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"((uint32_t)cnt * (uint32_t)(CB + 16))
                 : "memory");
  }
  __syncwarp();
  // the last probe whose pairs start at or before b0
  int lo = 0, hi = npc - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (S.pref[mid] <= b0) lo = mid; else hi = mid - 1;
  }
  for (int j = lo + lane; j < npc; j += 32) {
    const int ps = S.pref[j], pe = S.pref[j + 1];
    if (ps >= b0 + cnt) break;
    const int t0 = max(ps, b0), t1 = min(pe, b0 + cnt);
    if (t1 <= t0) continue;
    const int pos0 = S.pbeg[j] + (t0 - ps);
    const uint32_t n = (uint32_t)(t1 - t0);
    const uint64_t* src_c = P.codes + (size_t)pos0 * WT;
    const float4* src_f = P.factors + pos0;
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dc + (uint32_t)((t0 - b0) * CB)), "l"(src_c), "r"(n * (uint32_t)CB), "r"(bar)
        : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(df + (uint32_t)((t0 - b0) * 16)), "l"(src_f), "r"(n * 16u), "r"(bar)
        : "memory");
  }
}

template <int WT>
__host__ __device__ constexpr int stage_bytes(int step) {
  return 2 * step * (WT * 8 + 16);
}

template <int WT, int BQT, bool STG = false>
__global__ void __launch_bounds__(kThreads, fused_min_blocks<WT>()) fused_search_kernel(FusedParams P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ int s_ub_cnt, s_cand_cnt, s_top_cnt, s_surv, s_overflow;
  __shared__ float s_tau;
  __shared__ int s_scratch[kCompactU * kThreads / 32];
  __shared__ SelState s_sel;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarps = blockDim.x >> 5;
  size_t off[10];
  fused_smem_bytes(P.pch, P.bq, P.W, P.d, P.cu, P.ce, P.ct, nwarps, off, P.scap);
  FusedSmem S;
  S.planes = reinterpret_cast<uint64_t*>(smem + off[0]);
  S.pmeta = reinterpret_cast<float4*>(smem + off[1]);
  S.psum = reinterpret_cast<int*>(smem + off[2]);
  S.pbeg = reinterpret_cast<int*>(smem + off[3]);
  S.pref = reinterpret_cast<int*>(smem + off[4]);
  S.qv = reinterpret_cast<float*>(smem + off[5]);
  S.sel = &s_sel;
  S.ubk = reinterpret_cast<uint32_t*>(smem + off[6]);
  S.estk = reinterpret_cast<unsigned long long*>(smem + off[7]);
  S.topk = reinterpret_cast<unsigned long long*>(smem + off[8]);
  S.scand = reinterpret_cast<int4*>(smem + off[9]);
  const int W = P.W, bq = P.bq, k = P.k;
  int4* cand = P.cand + (int64_t)blockIdx.x * P.cand_cap;
  // staging (STG): two stages in the tail's candidate area, one mbarrier each
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ int s_stg_fail;
  unsigned char* stg = reinterpret_cast<unsigned char*>(S.scand);
  uint32_t par = 0;  // bit b: parity of stage b's next completion
  if constexpr (STG) {
    if (tid == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&s_bar[0])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&s_bar[1])), "r"(1));
      asm volatile("fence.mbarrier_init.release.cluster;");
      s_stg_fail = 0;
    }
    __syncthreads();
  }

  __shared__ int s_next, s_next_fill;
  // next work item: dynamic (one atomic per query, taken by thread 0 and
  // broadcast) or static striding
  auto fetch = [&](int64_t cur) -> int64_t {
    if (!P.next) return cur + gridDim.x;
    __syncthreads();
    if (tid == 0) s_next = atomicAdd(P.next, 1);
    __syncthreads();
    return s_next;
  };
  const int split = P.split > 1 ? P.split : 1;
  const int64_t n_items = (P.nq_dev ? (int64_t)*P.nq_dev : P.nq) * split;
  for (int64_t it = P.next ? fetch(0) : (int64_t)blockIdx.x; it < n_items; it = fetch(it)) {
    const int64_t qi = it / split;
    const int sl = (int)(it % split);
    const int64_t q = P.order ? (int64_t)P.order[qi] : qi;
    int np = P.nprobe;
    if (P.nprobe_q) np = min(max(P.nprobe_q[q], 1), P.nprobe);
    // this item's probes: all of them, or slice sl of `split`
    const int pb = (int)((int64_t)np * sl / split), pe = (int)((int64_t)np * (sl + 1) / split);
    if (split > 1) cand = P.cand + it * P.cand_cap;
    for (int i = tid; i < P.d; i += blockDim.x) S.qv[i] = P.queries[q * P.d + i];
    if (tid == 0) {
      s_ub_cnt = 0;
      s_cand_cnt = 0;
      s_top_cnt = 0;
      s_surv = 0;
      s_overflow = 0;
      s_tau = __int_as_float(0x7f800000);
    }
    __syncthreads();
    int pairs_done = 0;
    for (int pc0 = pb; pc0 < pe; pc0 += P.pch) {
      const int npc = min(P.pch, pe - pc0);
      for (int j = wid; j < npc; j += nwarps) {
        const int jg = pc0 + j;
        const int64_t pj = q * P.nprobe + jg;
        const int c = P.probe_ids[pj];
        const float add = P.probe_dist[pj];
        quantize_probe(P, S, q, j, jg, c, P.probe_nq2 ? P.probe_nq2[pj] : add, add);
      }
      __syncthreads();
      if (wid == 0) {  // inclusive prefix of the bucket lengths, 32 at a time
        int carry = 0;
        if (lane == 0) S.pref[0] = 0;
        for (int j0 = 0; j0 < npc; j0 += 32) {
          const int jj = j0 + lane;
          int v = (jj < npc) ? S.pref[jj + 1] : 0;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, v, o);
            if (lane >= o) v += y;
          }
          if (jj < npc) S.pref[jj + 1] = carry + v;
          carry += __shfl_sync(kFull, v, 31);
        }
      }
      __syncthreads();
      const int total = S.pref[npc];
      int j = 0;
      constexpr int PPT = STG ? 1 : pairs_per_thread<WT>();
      const int step = PPT * blockDim.x;
      if constexpr (STG) {
        if (wid == 0 && total > 0) stage_issue<WT>(P, S, stg, s_bar, 0, min(step, total), npc, 0, step);
      }
      int rnd = 0;
      // Pairs of a round. Direct loads: warp w takes the block [base + 32 PPT w,
      // base + 32 PPT (w + 1)) and lane l its pairs l, l + 32, ..., so that
      // each load instruction of a warp covers consecutive codes; a block
      // inside one probe (the usual case) shares that probe's position,
      // bit-planes and bounds across the warp, and each plane word is read
      // once for a thread's two pairs. Staged rounds: thread tid takes the
      // stage slots tid PPT ... The warps run unsynchronized between the
      // buffer upkeep points (every kUpkeep rounds, every round when staged);
      // the buffers have room for the appends in between.
      constexpr int kUpkeep = STG ? 1 : 2;
      static_assert(kUpkeep * PPT <= kPPT, "buffer room between upkeeps");
      const bool tracing = P.tr.pair_id != nullptr;
      for (int base = 0; base < total; base += step, ++rnd) {
        const int buf = rnd & 1;
        if constexpr (STG) {
          // the next round's copies go out now (its stage was last read in
          // the round before this one, which ended with a barrier); then
          // this round's stage is waited for
          if (wid == 0 && base + step < total)
            stage_issue<WT>(P, S, stg, s_bar, base + step, min(step, total - base - step), npc,
                            buf ^ 1, step);
          if (!stage_wait(&s_bar[buf], (par >> buf) & 1u)) s_stg_fail = 1;
          par ^= 1u << buf;
        }
        // every load of this thread's PPT pairs is issued first (they are
        // independent), then the pairs are evaluated
        int posv[PPT], jv[PPT], tv[PPT], ipv[PPT];
        CodeRegs<WT> cr[PPT];
        float4 fv[PPT];
        bool one_probe = false;
        if constexpr (STG) {
          // consecutive pairs advance through a bucket: the prefix array is
          // consulted again only at a bucket boundary
          const int t0 = base + tid * PPT;
          int pos = 0, next_b = 0;
#pragma unroll
          for (int pp = 0; pp < PPT; ++pp) {
            const int t = t0 + pp;
            posv[pp] = -1;
            jv[pp] = 0;
            tv[pp] = t;
            if (t < total) {
              if (pp == 0 || t >= next_b) {
                while (S.pref[j + 1] <= t) ++j;
                pos = S.pbeg[j] + (t - S.pref[j]);
                next_b = S.pref[j + 1];
              } else {
                ++pos;
              }
              posv[pp] = pos;
              jv[pp] = j;
              // this pair's slot in the round's stage (shared memory: plain
              // loads, not the read-only global path)
              const int r = t - base;
              const uint4* cs = reinterpret_cast<const uint4*>(stg + (size_t)(buf * step + r) * (WT * 8));
#pragma unroll
              for (int w = 0; w < WT; w += 2) {
                const uint4 v = cs[w / 2];
                cr[pp].c[w] = ((uint64_t)v.y << 32) | v.x;
                cr[pp].c[w + 1] = ((uint64_t)v.w << 32) | v.z;
              }
              fv[pp] = reinterpret_cast<const float4*>(stg + (size_t)2 * step * (WT * 8))[buf * step + r];
            }
          }
        } else {
          const int blk = base + wid * (32 * PPT);
          // the probe of the block's first pair; every lane's j is at most
          // that probe, so after this walk j is the same in all lanes
          if (blk < total)
            while (S.pref[j + 1] <= blk) ++j;
          one_probe = blk + 32 * PPT <= min(total, S.pref[j + 1]);  // warp-uniform
          if (one_probe) {
            const int p0 = S.pbeg[j] + (blk - S.pref[j]) + lane;
#pragma unroll
            for (int pp = 0; pp < PPT; ++pp) {
              posv[pp] = p0 + 32 * pp;
              jv[pp] = j;
              tv[pp] = blk + 32 * pp + lane;
              load_code<WT>(cr[pp], P.codes + (size_t)(uint32_t)posv[pp] * (uint32_t)W);
              fv[pp] = __ldg(P.factors + (uint32_t)posv[pp]);
            }
          } else {
#pragma unroll
            for (int pp = 0; pp < PPT; ++pp) {
              const int t = blk + 32 * pp + lane;
              posv[pp] = -1;
              jv[pp] = 0;
              tv[pp] = t;
              if (t < total) {
                while (S.pref[j + 1] <= t) ++j;
                posv[pp] = S.pbeg[j] + (t - S.pref[j]);
                jv[pp] = j;
                load_code<WT>(cr[pp], P.codes + (size_t)(uint32_t)posv[pp] * (uint32_t)W);
                fv[pp] = __ldg(P.factors + (uint32_t)posv[pp]);
              }
            }
          }
        }
        // A block inside one probe (direct loads, D' = 128 / 256, B_q = 4):
        // every pair valid, the probe's bounds shared, each plane word read
        // once for both pairs, appends reserved from ballots.
        bool evaluated = false;
        if constexpr (!STG && PPT == 2 && (WT == 2 || WT == 4) && BQT == 4) {
          if (one_probe) {
            evaluated = true;
            code_ip2<WT>(cr[0], cr[1], S.planes + (size_t)j * (4 * WT), ipv[0], ipv[1]);
            const float4 mt = S.pmeta[j];
            const int psum = S.psum[j];
            const float tau = s_tau;
            float dv[2], lv[2], uv[2];
#pragma unroll
            for (int pp = 0; pp < 2; ++pp) {
              const float4 f = fv[pp];
              // estimator (§3.3.2 + Theorem 3.2) and its bound, fixed FP32 order
              const float t1 = (float)(2 * ipv[pp] - psum);
              const float xq = __fadd_rn(__fmul_rn(mt.x, t1), __fmul_rn(mt.y, f.w));
              dv[pp] = __fsub_rn(__fadd_rn(f.x, mt.w), __fmul_rn(f.y, xq));
              const float e = __fmul_rn(f.z, mt.z);
              lv[pp] = __fsub_rn(dv[pp], e);
              uv[pp] = __fadd_rn(dv[pp], e);
            }
            const unsigned lt = (1u << lane) - 1u;
            const unsigned mu0 = __ballot_sync(kFull, uv[0] < tau);
            const unsigned mu1 = __ballot_sync(kFull, uv[1] < tau);
            if (mu0 | mu1) {
              int b = 0;
              if (lane == 0) b = atomicAdd(&s_ub_cnt, __popc(mu0) + __popc(mu1));
              b = __shfl_sync(kFull, b, 0);
              if (uv[0] < tau) S.ubk[b + __popc(mu0 & lt)] = float_key(uv[0]);
              if (uv[1] < tau) S.ubk[b + __popc(mu0) + __popc(mu1 & lt)] = float_key(uv[1]);
            }
            const unsigned mc0 = __ballot_sync(kFull, lv[0] <= tau);
            const unsigned mc1 = __ballot_sync(kFull, lv[1] <= tau);
            if (mc0 | mc1) {
              int b = 0;
              if (lane == 0) b = atomicAdd(&s_cand_cnt, __popc(mc0) + __popc(mc1));
              b = __shfl_sync(kFull, b, 0);
#pragma unroll
              for (int pp = 0; pp < 2; ++pp) {
                if (lv[pp] <= tau) {
                  const int slot = b + (pp == 0 ? __popc(mc0 & lt) : __popc(mc0) + __popc(mc1 & lt));
                  if (slot < P.cand_cap)
                    cand[slot] = make_int4(posv[pp], __float_as_int(lv[pp]), __float_as_int(dv[pp]),
                                           __float_as_int(uv[pp]));
                  else
                    s_overflow = 1;
                }
              }
            }
            if (tracing) {
#pragma unroll
              for (int pp = 0; pp < 2; ++pp) {
                const int64_t tt = pairs_done + tv[pp];
                if (tt < P.tr.pair_cap) {
                  const int64_t o = q * P.tr.pair_cap + tt;
                  P.tr.pair_id[o] = __ldg(P.perm + posv[pp]);
                  P.tr.pair_ip[o] = ipv[pp];
                  P.tr.pair_est[3 * o] = dv[pp];
                  P.tr.pair_est[3 * o + 1] = lv[pp];
                  P.tr.pair_est[3 * o + 2] = uv[pp];
                }
              }
            }
          }
        }
        if (!evaluated) {
        // <x_b, q_u> of every pair (§3.3.2)
        {
#pragma unroll
          for (int pp = 0; pp < PPT; ++pp)
            ipv[pp] = posv[pp] < 0 ? 0
                                   : code_ip<WT, BQT>(cr[pp], P.codes + (size_t)(uint32_t)posv[pp] * (uint32_t)W,
                                                      S.planes + (size_t)jv[pp] * bq * W, W, bq);
        }
        // the estimator and its bounds for every pair of the round
        float distv[PPT], lbv[PPT], ubv[PPT];
        const float tau = s_tau;
#pragma unroll
        for (int pp = 0; pp < PPT; ++pp) {
          distv[pp] = 0.0f;
          lbv[pp] = __int_as_float(0x7f800000);
          ubv[pp] = __int_as_float(0x7f800000);
          if (posv[pp] >= 0) {
            const int jj = jv[pp];
            const int ip = ipv[pp];
            const float4 mt = S.pmeta[jj];
            const int psum = S.psum[jj];
            const float4 f = fv[pp];
            // estimator (§3.3.2 + Theorem 3.2) and its bound, fixed FP32 order
            const float t1 = (float)(2 * ip - psum);
            const float xq = __fadd_rn(__fmul_rn(mt.x, t1), __fmul_rn(mt.y, f.w));
            const float dist = __fsub_rn(__fadd_rn(f.x, mt.w), __fmul_rn(f.y, xq));
            const float e = __fmul_rn(f.z, mt.z);
            distv[pp] = dist;
            lbv[pp] = __fsub_rn(dist, e);
            ubv[pp] = __fadd_rn(dist, e);
          }
        }
        // one packed warp scan reserves the slots of both buffers
        int nu = 0, nc = 0;
#pragma unroll
        for (int pp = 0; pp < PPT; ++pp) {
          if (posv[pp] < 0) continue;
          nu += ubv[pp] < tau;
          nc += lbv[pp] <= tau;
        }
        const int packed = nu | (nc << 16);
        int incl = packed;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += y;
        }
        const int tot = __shfl_sync(kFull, incl, 31);
        const int excl = incl - packed;
        int bu = 0, bc = 0;
        if (lane == 0) {
          if (tot & 0xffff) bu = atomicAdd(&s_ub_cnt, tot & 0xffff);
          if (tot >> 16) bc = atomicAdd(&s_cand_cnt, tot >> 16);
        }
        bu = __shfl_sync(kFull, bu, 0) + (excl & 0xffff);
        bc = __shfl_sync(kFull, bc, 0) + (excl >> 16);
#pragma unroll
        for (int pp = 0; pp < PPT; ++pp) {
          if (posv[pp] < 0) continue;
          if (ubv[pp] < tau) S.ubk[bu++] = float_key(ubv[pp]);
          if (lbv[pp] <= tau) {
            if (bc < P.cand_cap)
              cand[bc] = make_int4((int)posv[pp], __float_as_int(lbv[pp]),
                                   __float_as_int(distv[pp]), __float_as_int(ubv[pp]));
            else
              s_overflow = 1;
            ++bc;
          }
          if (tracing) {
            const int64_t tt = pairs_done + tv[pp];
            if (tt < P.tr.pair_cap) {
              const int64_t o = q * P.tr.pair_cap + tt;
              P.tr.pair_id[o] = __ldg(P.perm + posv[pp]);
              P.tr.pair_ip[o] = ipv[pp];
              P.tr.pair_est[3 * o] = distv[pp];
              P.tr.pair_est[3 * o + 1] = lbv[pp];
              P.tr.pair_est[3 * o + 2] = ubv[pp];
            }
          }
        }
        }  // !evaluated
        if (rnd % kUpkeep != kUpkeep - 1 && base + step < total) continue;
        // Buffer upkeep. The counters are read between two barriers: after
        // every append before this point and before any append after it, so
        // that every thread takes the same branches (a warp that ran ahead
        // must not change what a slower one reads).
        __syncthreads();
        const int room = kUpkeep * step;
        const int ub_cnt = s_ub_cnt, c_cnt = s_cand_cnt;
        bool ovf = s_overflow != 0;
        __syncthreads();
        if (ub_cnt > P.cu - room) {  // keep the k smallest upper bounds
          // (the top-k buffer is free during the scan)
          const uint32_t T = select_keep_h(S.ubk, &s_ub_cnt, k, *S.sel,
                                           reinterpret_cast<int*>(S.topk),
                                           reinterpret_cast<uint32_t*>(S.topk) + kHistBins,
                                           2 * P.ct - kHistBins);
          if (tid == 0) s_tau = key_float(T);
          __syncthreads();
        }
        if (c_cnt > P.cand_cap - room) {
          const float tau = s_tau;
          compact_cand(cand, &s_cand_cnt, P.cand_cap, s_scratch,
                       [tau](const int4& e) { return __int_as_float(e.y) <= tau; });
          if (s_cand_cnt > P.cand_cap - room) ovf = true;  // same value in every thread
          __syncthreads();
          if (ovf && tid == 0) s_overflow = 1;
        }
        if (ovf) {
          if constexpr (STG) {  // the next round's copies are in flight: let them land
            if (base + step < total) {
              if (!stage_wait(&s_bar[buf ^ 1], (par >> (buf ^ 1)) & 1u)) s_stg_fail = 1;
              par ^= 1u << (buf ^ 1);
            }
          }
          break;
        }
      }
      pairs_done += total;
      __syncthreads();
      if (s_overflow) break;
    }
    if (split > 1) {  // a slice: hand its k smallest upper bounds and its list to the merge
      if (s_ub_cnt > k) select_keep<uint32_t>(S.ubk, &s_ub_cnt, k, *S.sel);
      const int nk = min(s_ub_cnt, k);
      for (int i = tid; i < nk; i += blockDim.x) P.ub_out[it * k + i] = S.ubk[i];
      if (tid == 0) {
        if (STG && s_stg_fail) atomicExch(P.err, 2);
        P.slice_cnt[2 * it] = nk;
        P.slice_cnt[2 * it + 1] = min(s_cand_cnt, P.cand_cap);
        if (s_overflow) atomicExch(P.err, 1);
      }
      __syncthreads();
      continue;
    }
    // tau_ub: k-th smallest upper bound; pilot: the m smallest estimates
    const int n_ub = s_ub_cnt;
    int ub_rem = 0, ub_eq = 0;
    const uint32_t T_ub =
        (n_ub >= k) ? hist_select(n_ub, k, *S.sel, reinterpret_cast<int*>(S.topk),
                                  reinterpret_cast<uint32_t*>(S.topk) + kHistBins,
                                  2 * P.ct - kHistBins, ub_rem, ub_eq,
                                  [&S](int i) { return S.ubk[i]; })
                    : 0u;
    const float tau_ub = (n_ub >= k) ? key_float(T_ub) : __int_as_float(0x7f800000);
    TailShared ts{&s_cand_cnt, &s_top_cnt, &s_surv, s_scratch};
    // Stage the entries with LB <= tau_ub in shared memory (one pass with
    // four loads in flight per thread) so that the tail's selections and
    // compactions read shared memory; if they do not fit, the tail works on
    // the list in global memory, which this pass only reads.
    int4* tcand = cand;
    int tcap = P.cand_cap;
    if (P.scap > 0) {
      const int n_c = min(s_cand_cnt, P.cand_cap);
      if (tid == 0) s_next_fill = 0;
      __syncthreads();
      for (int b = 0; b < n_c; b += 4 * blockDim.x) {
        int4 e[4];
        bool keep[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = b + u * blockDim.x + tid;
          keep[u] = false;
          if (i < n_c) {
            e[u] = cand[i];
            keep[u] = __int_as_float(e[u].y) <= tau_ub;
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int slot = warp_reserve(keep[u], &s_next_fill);
          if (keep[u] && slot < P.scap) S.scand[slot] = e[u];
        }
      }
      __syncthreads();
      if (s_next_fill <= P.scap) {
        tcand = S.scand;
        tcap = P.scap;
        __syncthreads();
        if (tid == 0) s_cand_cnt = s_next_fill;
      }
      __syncthreads();
    }
    finish_query(P, S, q, tcand, tcap, tau_ub, ts, tcand == S.scand);
    if (tid == 0) {
      if (STG && s_stg_fail) atomicExch(P.err, 2);
      if (s_overflow) atomicExch(P.err, 1);
      if (P.tr.n_pairs) P.tr.n_pairs[q] = pairs_done;
    }
    __syncthreads();
  }
}


// The end of a split search: one CTA per query gathers its slices' upper
// bounds (the union holds the query's k smallest, so tau_ub is exact),
// stages the slices' candidates with LB <= tau_ub (shared memory when they
// fit, else the query's merged-list region), and finishes the query like the
// fused kernel. Results are identical to an unsplit search.
__global__ void __launch_bounds__(kThreads) split_merge_kernel(FusedParams P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ int s_cand_cnt, s_top_cnt, s_surv, s_fill;
  __shared__ int s_scratch[kCompactU * kThreads / 32];
  __shared__ SelState s_sel;
  __shared__ int s_off[33];
  const int tid = threadIdx.x;
  size_t off[10];
  fused_smem_bytes(P.pch, P.bq, P.W, P.d, P.cu, P.ce, P.ct, blockDim.x >> 5, off, P.scap);
  FusedSmem S;
  S.planes = nullptr;
  S.pmeta = nullptr;
  S.psum = nullptr;
  S.pbeg = nullptr;
  S.pref = nullptr;
  S.qv = reinterpret_cast<float*>(smem + off[5]);
  S.sel = &s_sel;
  S.ubk = reinterpret_cast<uint32_t*>(smem + off[6]);
  S.estk = reinterpret_cast<unsigned long long*>(smem + off[7]);
  S.topk = reinterpret_cast<unsigned long long*>(smem + off[8]);
  S.scand = reinterpret_cast<int4*>(smem + off[9]);
  const int k = P.k, split = P.split;
  for (int64_t qi = blockIdx.x; qi < P.nq; qi += gridDim.x) {
    const int64_t q = P.order ? (int64_t)P.order[qi] : qi;
    for (int i = tid; i < P.d; i += blockDim.x) S.qv[i] = P.queries[q * P.d + i];
    if (tid == 0) {
      s_off[0] = 0;
      for (int sl = 0; sl < split; ++sl) s_off[sl + 1] = s_off[sl] + P.slice_cnt[2 * (qi * split + sl)];
      s_top_cnt = 0;
      s_surv = 0;
      s_fill = 0;
    }
    __syncthreads();
    const int n_ub = s_off[split];
    for (int sl = 0; sl < split; ++sl)
      for (int i = tid; i < s_off[sl + 1] - s_off[sl]; i += blockDim.x)
        S.ubk[s_off[sl] + i] = P.ub_out[(qi * split + sl) * k + i];
    __syncthreads();
    const uint32_t T_ub = (n_ub >= k) ? block_select<uint32_t>(S.ubk, n_ub, k, *S.sel) : 0u;
    const float tau_ub = (n_ub >= k) ? key_float(T_ub) : __int_as_float(0x7f800000);
    int4* merged = P.cand2 + qi * P.cand_cap;
    for (int sl = 0; sl < split; ++sl) {
      const int64_t item = qi * split + sl;
      const int4* src = P.cand + item * P.cand_cap;
      const int n_c = P.slice_cnt[2 * item + 1];
      for (int b = 0; b < n_c; b += blockDim.x) {
        const int i = b + tid;
        int4 e = make_int4(0, 0, 0, 0);
        bool keep = false;
        if (i < n_c) {
          e = src[i];
          keep = __int_as_float(e.y) <= tau_ub;
        }
        const int slot = warp_reserve(keep, &s_fill);
        if (keep) {
          if (slot < P.scap) S.scand[slot] = e;
          if (slot < P.cand_cap) merged[slot] = e;
        }
      }
    }
    __syncthreads();
    const int nf = s_fill;
    if (nf > P.cand_cap && tid == 0) atomicExch(P.err, 1);
    const bool in_smem = nf <= P.scap;
    if (tid == 0) s_cand_cnt = min(nf, P.cand_cap);
    __syncthreads();
    TailShared ts{&s_cand_cnt, &s_top_cnt, &s_surv, s_scratch};
    finish_query(P, S, q, in_smem ? S.scand : merged, in_smem ? P.scap : P.cand_cap, tau_ub, ts,
                 true);
    __syncthreads();
  }
}

// ------------------------------------------------ warp-per-query fused scan
// The same search as fused_search_kernel with one WARP per query instead of
// one CTA, for the common shapes (D' = 128 or 256, B_q = 4, k <= 128): no
// block barrier anywhere. Per probe the warp quantizes the query against the
// bucket's centroid with its lanes owning dimensions 32 r + lane, so that
// each bit-plane word of q_u is one ballot and the planes sit in registers;
// the bucket's codes are then scanned with lanes on consecutive codes
// (coalesced 16-byte loads, PPL codes per lane per step). The warp keeps the
// exact running k-th smallest upper bound tau (a 256-key buffer, sorted when
// full) and appends every code with LB <= tau to its own candidate region
// (compacted by the current tau when full). The end of the query follows the
// same rule as finish_query (§4, reading R1): tau_ub, the pilot, tau1, the
// rest of the re-rank set and the top-k by (distance, id). A query whose
// candidates do not fit the region is handed to the CTA kernel (redo list).
constexpr int kWarpMaxK = 128;     // largest k of the warp kernel
constexpr int kWarpBuf = 256;      // keys per per-warp buffer
constexpr int kWarpThreads = 128;  // 4 warps (queries) per CTA

struct __align__(16) WarpSmem {
  uint32_t ubk[kWarpBuf];               // running upper-bound keys
  unsigned long long top[kWarpBuf];     // (exact score key << 32) | id
  int hist[256];                        // radix-select histogram / row staging
  float qv[256];                        // the query (d <= 256)
};

// Ascending bitonic sort of the first n (<= 256) keys of buf in place (the
// other slots of the 256 become `pad`, the largest key): 36 compare-exchange
// steps over shared memory, four pairs per lane per step. One out-of-line
// copy per key type keeps the kernel's code small. Whole warp.
template <class T>
__device__ __noinline__ void warp_sort_buf(T* buf, int n, T pad) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  for (int e = n + lane; e < kWarpBuf; e += 32) buf[e] = pad;
  __syncwarp();
#pragma unroll 1
  for (int size = 2; size <= kWarpBuf; size <<= 1) {
#pragma unroll 1
    for (int j = size >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int t = lane + 32 * u;            // pair index, 0..127
        const int lo = 2 * t - (t & (j - 1));
        const int hi = lo + j;
        const bool up = (lo & size) == 0;
        const T a = buf[lo], b = buf[hi];
        if (up ? (b < a) : (a < b)) {
          buf[lo] = b;
          buf[hi] = a;
        }
      }
      __syncwarp();
    }
  }
}

// The want-th smallest (1-based, want <= n) of n 32-bit keys keyf(i), by an
// MSD radix select over the bits below the keys' common prefix (hist: 256
// ints of per-warp shared memory). ties: how many keys equal to the result
// are among the want smallest; eqn: how many keys equal it. Whole warp.
template <class F>
__device__ uint32_t warp_select_u32(int* hist, int n, int want, int& ties, int& eqn, F keyf) {
  const int lane = threadIdx.x & 31;
  uint32_t mn = 0xffffffffu, mx = 0u;
  for (int i = lane; i < n; i += 32) {
    const uint32_t k = keyf(i);
    mn = min(mn, k);
    mx = max(mx, k);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(kFull, mn, o));
    mx = max(mx, __shfl_xor_sync(kFull, mx, o));
  }
  if (mn == mx) {
    ties = want;
    eqn = n;
    return mn;
  }
  const int hb = 31 - __clz(mn ^ mx);  // highest bit where keys differ
  int shift = hb + 1;
  uint32_t mask = hb == 31 ? 0u : ~((2u << hb) - 1u);
  uint32_t prefix = mn & mask;
  int rem = want, last = 0;
  while (shift > 0) {
    const int nb = shift >= 8 ? 8 : shift;
    shift -= nb;
    const uint32_t dm = (1u << nb) - 1u;
    __syncwarp();
    for (int t = lane; t < 256; t += 32) hist[t] = 0;
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      const uint32_t k = keyf(i);
      if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & dm], 1);
    }
    __syncwarp();
    int c[8], s = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      c[t] = hist[8 * lane + t];
      s += c[t];
    }
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    const int excl = incl - s;
    const unsigned bal = __ballot_sync(kFull, excl < rem && rem <= incl);
    const int src = __ffs(bal) - 1;
    int digit = 0, nrem = 0, cnt = 0;
    if (lane == src) {
      int cum = excl;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (digit == 0 && nrem == 0 && cum + c[t] >= rem) {
          digit = 8 * lane + t;
          nrem = rem - cum;
          cnt = c[t];
        }
        cum += c[t];
      }
    }
    digit = __shfl_sync(kFull, digit, src);
    rem = __shfl_sync(kFull, nrem, src);
    last = __shfl_sync(kFull, cnt, src);
    prefix |= (uint32_t)digit << shift;
    mask |= dm << shift;
  }
  ties = rem;
  eqn = last;
  return prefix;
}

// In-place stable compaction of the first n entries of L by keep(e).
template <class F>
__device__ __forceinline__ int warp_compact(int4* L, int n, F keep_f) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  int out = 0;
  __syncwarp();  // entries other lanes wrote are visible
  for (int b0 = 0; b0 < n; b0 += 32) {
    const int i = b0 + lane;
    int4 e = make_int4(0, 0, 0, 0);
    bool keep = false;
    if (i < n) {
      e = L[i];
      keep = keep_f(e);
    }
    const unsigned bal = __ballot_sync(kFull, keep);
    if (keep) L[out + __popc(bal & lt)] = e;
    out += __popc(bal);
  }
  __syncwarp();
  return out;
}

// Randomized B_q = 4 quantization of the query against cluster c (§3.3.1)
// with the same arithmetic and random stream as quant_core, lane l owning the
// dimensions 32 r + l (r < NW): the Philox call of dimensions 4m..4m+3 is
// computed by lane m % 32 and its words are exchanged by shuffles. Plane b's
// u32 word r is then one ballot. Returns sum(q_u); writes the planes and the
// estimator constants (quant_meta).
template <int NW>
__device__ __forceinline__ int quant_warp(const FusedParams& P, int64_t q, int c, float nq2,
                                          float add, uint32_t (&pl)[4][NW], float4* meta) {
  const int lane = threadIdx.x & 31;
  constexpr int dpad = 32 * NW;
  const float* rq = P.rq + q * dpad;
  const float* pc = P.ptc + (int64_t)c * dpad;
  float qd[NW];
  float vl = __int_as_float(0x7f800000), vr = __int_as_float(0xff800000);
#pragma unroll
  for (int r = 0; r < NW; ++r) {
    qd[r] = __fsub_rn(rq[32 * r + lane], pc[32 * r + lane]);
    vl = fminf(vl, qd[r]);
    vr = fmaxf(vr, qd[r]);
  }
  vl = warp_min_f(vl);
  vr = warp_max_f(vr);
  const float delta = __fdiv_rn(__fsub_rn(vr, vl), 15.0f);
  const uint64_t gq = (uint64_t)(P.q_offset + q);
  U4 w[NW / 4];
#pragma unroll
  for (int cc = 0; cc < NW / 4; ++cc)
    w[cc] = philox4x32_10(P.seed, (uint32_t)(lane + 32 * cc), (uint32_t)gq, (uint32_t)c, kTagQuant);
  int sum = 0;
  int qu[NW];
#pragma unroll
  for (int r = 0; r < NW; ++r) {
    // dimension 32 r + lane: Philox call 8 r + lane / 4 (lane 8 (r % 4) + lane / 4,
    // call index r / 4), word lane % 4
    const int src = 8 * (r & 3) + (lane >> 2);
    const uint32_t a0 = __shfl_sync(kFull, w[r >> 2].x, src);
    const uint32_t a1 = __shfl_sync(kFull, w[r >> 2].y, src);
    const uint32_t a2 = __shfl_sync(kFull, w[r >> 2].z, src);
    const uint32_t a3 = __shfl_sync(kFull, w[r >> 2].w, src);
    const int s = lane & 3;
    const uint32_t word = s == 0 ? a0 : (s == 1 ? a1 : (s == 2 ? a2 : a3));
    int v = 0;
    if (delta > 0.0f) {
      const float u = __fmul_rn(__uint2float_rn(word >> 8), 0x1.0p-24f);
      const float x = __fdiv_rn(__fsub_rn(qd[r], vl), delta);
      v = __float2int_rd(__fadd_rn(x, u));
      v = v > 15 ? 15 : v;
    }
    qu[r] = v;
    sum += v;
  }
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int r = 0; r < NW; ++r) pl[b][r] = __ballot_sync(kFull, (qu[r] >> b) & 1);
  *meta = quant_meta(delta, vl, nq2, add, P.eps0, dpad);
  return warp_sum_i(sum);
}

// Exact scores of staged rows: stage[0..n) hold bucket positions (n <= 32),
// lane l scores row l; keys <= kmax are appended to the top buffer. Returns
// the new buffer count (whole warp; the buffer keeps room for 32).
__device__ __noinline__ int warp_score_rows(const FusedParams& P, WarpSmem& S, const int* stage,
                                               int n, int tn, unsigned long long kmax) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  unsigned long long key = ~0ull;
  const bool valid = lane < n;
  if (valid) {
    const int pos = stage[lane];
    const float* x = P.data_b + (int64_t)pos * P.d;
    const float acc = P.metric ? row_score<true>(x, S.qv, P.d) : row_score<false>(x, S.qv, P.d);
    const int id = __ldg(P.perm + pos);
    key = ((unsigned long long)float_key(acc) << 32) | (uint32_t)id;
  }
  const bool take = valid && key <= kmax;
  const unsigned bal = __ballot_sync(kFull, take);
  if (take) S.top[tn + __popc(bal & lt)] = key;
  __syncwarp();
  return tn + __popc(bal);
}

// Keep the k smallest keys of the top buffer (sorted); returns the k-th
// smallest (all ones if fewer than k).
__device__ __noinline__ unsigned long long warp_top_keep(WarpSmem& S, int& tn, int k) {
  warp_sort_buf<unsigned long long>(S.top, tn, ~0ull);
  const unsigned long long T = tn >= k ? S.top[k - 1] : ~0ull;
  tn = min(tn, k);
  return T;
}

// List entries per lane per step in the passes of the warp's query end (so
// that a pass over a few thousand entries is a few dependent steps, not one
// per 32 entries).
constexpr int kTU = 4;

// Stage the rows of the entries with in[u] for exact scoring (32 at a time;
// stage: 64 ints); each staged row is requested from L2 at once.
template <int U>
__device__ __forceinline__ int warp_stage_rows(const FusedParams& P, WarpSmem& S, const int (&pos)[U],
                                               const bool (&in)[U], int& staged, int tn,
                                               unsigned long long kmax) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  int* stage = S.hist;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const unsigned bal = __ballot_sync(kFull, in[u]);
    if (in[u]) {
      stage[staged + __popc(bal & lt)] = pos[u];
      const char* x = reinterpret_cast<const char*>(P.data_b + (int64_t)pos[u] * P.d);
      for (int o = 0; o < P.d * (int)sizeof(float); o += 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(x + o));
    }
    staged += __popc(bal);
    __syncwarp();
    if (staged >= 32) {
      if (tn > kWarpBuf - 32) warp_top_keep(S, tn, P.k);
      tn = warp_score_rows(P, S, stage, 32, tn, kmax);
      staged -= 32;
      const int mv = lane < staged ? stage[32 + lane] : 0;
      __syncwarp();
      if (lane < staged) stage[lane] = mv;
      __syncwarp();
    }
  }
  return tn;
}

// The end of one query (the rule of finish_query, for one warp): L holds
// every code with LB <= tau_ub (n entries {position, LB, estimate, UB}).
// Passes over the list, kTU entries per lane per step: keep LB <= tau_ub
// (with the range of the kept estimates); a 256-bin histogram of their
// estimate keys finds the bin of the m-th smallest; that bin's entries are
// ranked exactly by (estimate, id) (a radix select if more than 256 share
// it); the pilot's rows are scored as they are found; then the rest.
__device__ __noinline__ void warp_finish(const FusedParams& P, WarpSmem& S, int64_t q, int4* L,
                                        int n, int ubn) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int k = P.k, m = P.m;
  float tau_ub = __int_as_float(0x7f800000);
  if (ubn >= k) {
    warp_sort_buf<uint32_t>(S.ubk, ubn, 0xffffffffu);
    tau_ub = key_float(S.ubk[k - 1]);
  }
  // keep LB <= tau_ub, with the smallest and largest estimate key kept
  uint32_t kmin = 0xffffffffu, kmax = 0u;
  {
    int out = 0;
    __syncwarp();
    for (int b0 = 0; b0 < n; b0 += 32 * kTU) {
      int4 e[kTU];
      bool keep[kTU];
#pragma unroll
      for (int u = 0; u < kTU; ++u) {
        const int i = b0 + 32 * u + lane;
        keep[u] = false;
        if (i < n) {
          e[u] = L[i];
          keep[u] = __int_as_float(e[u].y) <= tau_ub;
        }
      }
#pragma unroll
      for (int u = 0; u < kTU; ++u) {
        const unsigned bal = __ballot_sync(kFull, keep[u]);
        if (keep[u]) {
          L[out + __popc(bal & lt)] = e[u];
          const uint32_t ek = float_key(__int_as_float(e[u].z));
          kmin = min(kmin, ek);
          kmax = max(kmax, ek);
        }
        out += __popc(bal);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      kmin = min(kmin, __shfl_xor_sync(kFull, kmin, o));
      kmax = max(kmax, __shfl_xor_sync(kFull, kmax, o));
    }
    n = out;
    __syncwarp();
  }
  // pilot threshold: the m-th smallest (estimate key, id) of the list
  uint32_t T_e = 0xffffffffu, T_id = 0xffffffffu;
  const bool pilot_all = n <= m;
  if (!pilot_all) {
    const uint64_t range = (uint64_t)(kmax - kmin) + 1u;
    auto bin_of = [kmin, range](uint32_t ek) { return (int)(((uint64_t)(ek - kmin) << 8) / range); };
    int* hist = S.hist;
    for (int t = lane; t < 256; t += 32) hist[t] = 0;
    __syncwarp();
    for (int b0 = 0; b0 < n; b0 += 32 * kTU) {
      uint32_t ek[kTU];
#pragma unroll
      for (int u = 0; u < kTU; ++u) {
        const int i = b0 + 32 * u + lane;
        ek[u] = i < n ? float_key(__int_as_float(L[i].z)) : 0u;
      }
#pragma unroll
      for (int u = 0; u < kTU; ++u)
        if (b0 + 32 * u + lane < n) atomicAdd(&hist[bin_of(ek[u])], 1);
    }
    __syncwarp();
    int c[8], sum = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      c[t] = hist[8 * lane + t];
      sum += c[t];
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    const int excl = incl - sum;
    const int src = __ffs(__ballot_sync(kFull, excl < m && m <= incl)) - 1;
    int bstar = 0, need = 0, cnt = 0;
    if (lane == src) {
      int cum = excl;
      bool found = false;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (!found && cum + c[t] >= m) {
          found = true;
          bstar = 8 * lane + t;
          need = m - cum;
          cnt = c[t];
        }
        cum += c[t];
      }
    }
    bstar = __shfl_sync(kFull, bstar, src);
    need = __shfl_sync(kFull, need, src);
    cnt = __shfl_sync(kFull, cnt, src);
    if (cnt <= kWarpBuf) {
      // the boundary bin's entries, ranked by (estimate key, id)
      int got = 0;
      for (int b0 = 0; b0 < n; b0 += 32 * kTU) {
        int4 e[kTU];
        bool in[kTU];
#pragma unroll
        for (int u = 0; u < kTU; ++u) {
          const int i = b0 + 32 * u + lane;
          in[u] = false;
          if (i < n) {
            e[u] = L[i];
            in[u] = bin_of(float_key(__int_as_float(e[u].z))) == bstar;
          }
        }
#pragma unroll
        for (int u = 0; u < kTU; ++u) {
          const unsigned bal = __ballot_sync(kFull, in[u]);
          if (in[u])
            S.top[got + __popc(bal & lt)] =
                ((unsigned long long)float_key(__int_as_float(e[u].z)) << 32) |
                (uint32_t)__ldg(P.perm + e[u].x);
          got += __popc(bal);
        }
      }
      warp_sort_buf<unsigned long long>(S.top, got, ~0ull);
      const unsigned long long T = S.top[need - 1];
      T_e = (uint32_t)(T >> 32);
      T_id = (uint32_t)T;
    } else {  // many equal estimates: radix selects by key, then by id
      int ties = 0, eqn = 0;
      T_e = warp_select_u32(S.hist, n, m, ties, eqn,
                            [L](int i) { return float_key(__int_as_float(L[i].z)); });
      if (eqn > ties) {
        int t2 = 0, e2 = 0;
        T_id = warp_select_u32(S.hist, n, ties, t2, e2, [L, T_e, &P](int i) {
          const int4 e = L[i];
          return float_key(__int_as_float(e.z)) == T_e ? (uint32_t)__ldg(P.perm + e.x) : 0xffffffffu;
        });
      }
    }
  }
  // the pilot: marked (bit 31 of the position) and scored as found;
  // tau1 = the k-th smallest of its exact scores
  int tn = 0, staged = 0;
  for (int b0 = 0; b0 < n; b0 += 32 * kTU) {
    int pos[kTU];
    bool in[kTU];
#pragma unroll
    for (int u = 0; u < kTU; ++u) {
      const int i = b0 + 32 * u + lane;
      in[u] = false;
      pos[u] = 0;
      if (i < n) {
        const int4 e = L[i];
        pos[u] = e.x;
        const uint32_t ek = float_key(__int_as_float(e.z));
        in[u] = pilot_all || ek < T_e || (ek == T_e && (uint32_t)__ldg(P.perm + e.x) <= T_id);
        if (in[u]) L[i].x = e.x | (int)0x80000000;
      }
    }
    tn = warp_stage_rows<kTU>(P, S, pos, in, staged, tn, ~0ull);
  }
  if (staged > 0) {
    if (tn > kWarpBuf - 32) warp_top_keep(S, tn, k);
    tn = warp_score_rows(P, S, S.hist, staged, tn, ~0ull);
    staged = 0;
  }
  const unsigned long long T1 = warp_top_keep(S, tn, k);
  const float tau1 = T1 != ~0ull ? key_float((uint32_t)(T1 >> 32)) : __int_as_float(0x7f800000);
  const float tau = fminf(tau_ub, tau1);
  // the rest of the re-rank set (LB <= tau, outside the pilot); keys above
  // the pilot's k-th cannot enter the result
  __syncwarp();
  for (int b0 = 0; b0 < n; b0 += 32 * kTU) {
    int pos[kTU];
    bool in[kTU];
#pragma unroll
    for (int u = 0; u < kTU; ++u) {
      const int i = b0 + 32 * u + lane;
      in[u] = false;
      pos[u] = 0;
      if (i < n) {
        const int4 e = L[i];
        pos[u] = e.x & 0x7fffffff;
        in[u] = e.x >= 0 && __int_as_float(e.y) <= tau;
      }
    }
    tn = warp_stage_rows<kTU>(P, S, pos, in, staged, tn, T1);
  }
  if (staged > 0) {
    if (tn > kWarpBuf - 32) warp_top_keep(S, tn, k);
    tn = warp_score_rows(P, S, S.hist, staged, tn, T1);
  }
  warp_sort_buf<unsigned long long>(S.top, tn, ~0ull);
  const int got = min(tn, k);
  for (int j = lane; j < k; j += 32) {
    const bool ok = j < got;
    const unsigned long long key = ok ? S.top[j] : 0ull;
    P.out_ids[q * k + j] = ok ? (int64_t)(key & 0xffffffffu) : -1;
    const float v = ok ? key_float((uint32_t)(key >> 32)) : __int_as_float(0x7f800000);
    P.out_dist[q * k + j] = P.metric ? -v : v;
  }
  __syncwarp();
}

template <int WT>
constexpr int warp_min_blocks() {
  return WT <= 2 ? 8 : 6;
}

// PPL: codes per lane per step (their loads are in flight together).
template <int WT, int PPL>
__global__ void __launch_bounds__(kWarpThreads, warp_min_blocks<WT>()) fused_warp_kernel(FusedParams P) {
  constexpr int NW = 2 * WT;                // u32 words per code and per plane
  __shared__ WarpSmem sm[kWarpThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  WarpSmem& S = sm[wid];
  const int64_t gw = (int64_t)blockIdx.x * (kWarpThreads / 32) + wid;
  int4* L = P.candw + gw * P.capw;
  const unsigned lt = (1u << lane) - 1u;
  const int k = P.k;
  const int room = P.capw - 32 * PPL;
  for (;;) {
    int qi = 0;
    if (lane == 0) qi = atomicAdd(P.next, 1);
    qi = __shfl_sync(kFull, qi, 0);
    if (qi >= P.nq) break;
    const int64_t q = P.order ? (int64_t)P.order[qi] : (int64_t)qi;
    int np = P.nprobe;
    if (P.nprobe_q) np = min(max(P.nprobe_q[q], 1), P.nprobe);
    __syncwarp();
    for (int i = lane; i < P.d; i += 32) S.qv[i] = P.queries[q * P.d + i];
    __syncwarp();
    int ubn = 0, nc = 0;
    float tau = __int_as_float(0x7f800000);
    bool ovf = false;
    for (int j = 0; j < np && !ovf; ++j) {
      const int64_t pj = q * P.nprobe + j;
      const int c = P.probe_ids[pj];
      const float add = P.probe_dist[pj];
      const float nq2 = P.probe_nq2 ? P.probe_nq2[pj] : add;
      uint32_t pl[4][NW];
      float4 mt;
      const int psum = quant_warp<NW>(P, q, c, nq2, add, pl, &mt);
      const int beg = P.bucket_off[c], end = P.bucket_off[c + 1];
      for (int base = beg; base < end; base += 32 * PPL) {
        int pos[PPL];
        uint32_t cw[PPL][NW];
        float4 f[PPL];
#pragma unroll
        for (int u = 0; u < PPL; ++u) {
          pos[u] = base + 32 * u + lane;
          if (pos[u] < end) {
            const uint4* cp = reinterpret_cast<const uint4*>(P.codes) + (size_t)pos[u] * (NW / 4);
#pragma unroll
            for (int v = 0; v < NW / 4; ++v) {
              const uint4 x = __ldg(cp + v);
              cw[u][4 * v] = x.x;
              cw[u][4 * v + 1] = x.y;
              cw[u][4 * v + 2] = x.z;
              cw[u][4 * v + 3] = x.w;
            }
            f[u] = __ldg(P.factors + pos[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < PPL; ++u) {
          const bool valid = pos[u] < end;
          float est = 0.0f, lb = __int_as_float(0x7f800000), ub = __int_as_float(0x7f800000);
          if (valid) {
            int ip = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              int pb = 0;
#pragma unroll
              for (int r = 0; r < NW; ++r) pb += __popc(cw[u][r] & pl[b][r]);
              ip += pb << b;
            }
            // estimator (§3.3.2 + Theorem 3.2) and its bound, fixed FP32 order
            const float t1 = (float)(2 * ip - psum);
            const float xq = __fadd_rn(__fmul_rn(mt.x, t1), __fmul_rn(mt.y, f[u].w));
            est = __fsub_rn(__fadd_rn(f[u].x, mt.w), __fmul_rn(f[u].y, xq));
            const float e = __fmul_rn(f[u].z, mt.z);
            lb = __fsub_rn(est, e);
            ub = __fadd_rn(est, e);
          }
          const bool wu = valid && ub < tau;
          const unsigned bu = __ballot_sync(kFull, wu);
          if (wu) S.ubk[ubn + __popc(bu & lt)] = float_key(ub);
          ubn += __popc(bu);
          const bool wc = valid && lb <= tau;
          const unsigned bc = __ballot_sync(kFull, wc);
          if (wc) {
            const int slot = nc + __popc(bc & lt);
            if (slot < P.capw)
              L[slot] = make_int4(pos[u], __float_as_int(lb), __float_as_int(est), __float_as_int(ub));
          }
          nc += __popc(bc);
        }
        // upkeep (warp-uniform): keep the k smallest upper bounds; compact
        // the candidate list by the current threshold when it fills
        if (ubn > kWarpBuf - 32 * PPL) {
          warp_sort_buf<uint32_t>(S.ubk, ubn, 0xffffffffu);
          tau = key_float(S.ubk[k - 1]);
          ubn = k;
        }
        if (nc > room) {
          const float t = tau;
          nc = warp_compact(L, min(nc, P.capw), [t](const int4& e) { return __int_as_float(e.y) <= t; });
          if (nc > room) {
            ovf = true;
            break;
          }
        }
      }
    }
    if (ovf) {  // the CTA kernel redoes this query
      if (lane == 0) P.redo[atomicAdd(P.redo_cnt, 1)] = (int)q;
      __syncwarp();
      continue;
    }
    warp_finish(P, S, q, L, nc, ubn);
  }
}

// ------------------------------------------- bucket-major tensor-core scan
// The queries probing one bucket share its codes, so the scan becomes a
// product (codes x queries) per bucket: <x_b, q_u> for a tile of 128 codes x
// 128 (query, cluster) pairs is one K = D' tensor-core product with A = the
// codes as BF16 0/1 and B = the quantized query values as BF16 0..15, FP32
// accumulation (exact: every partial sum is an integer below 2^24). The
// epilogue evaluates the estimator and bounds of every (code, query) pair
// exactly as the popcount path does and appends the pairs with LB <= tau'_q
// to the query's candidate list. Pass A covers each query's first probes
// with tau' = +inf; tau'_q is then the k-th smallest UB of its list; pass B
// covers the remaining probes. The list then holds every code with
// LB <= tau_ub (tau_ub <= tau'_q), which is all the per-query end needs.
constexpr int kTsM = 128;        // codes per tile (TMEM lanes)
constexpr int kTsN = 128;        // (query, cluster) pairs per tile (TMEM columns)
constexpr int kTsThreads = 128;  // 4 warps

struct TcScanParams {
  const uint64_t* codes;
  const float4* factors;
  const int32_t* bucket_off;
  int W, dpad, K, nprobe;
  const int32_t* pair_perm;  // pair indices (q * nprobe + rank) sorted by key
  const int32_t* pair_off;   // 2K + 3 key offsets
  int key_base;              // 0 (pass A) or K + 1 (pass B)
  const int32_t* tile_off;   // K + 1 tile offsets of this pass
  const __nv_bfloat16* qub;  // pairs x dpad quantized query values
  const float4* pmeta;       // pairs: A, B, E, nq2
  const int32_t* psum;       // pairs: sum(q_u)
  const float* qtau;         // queries: tau'
  int4* lists;               // queries x cap
  int32_t* lcnt;             // queries
  int cap;
  int* err;
};

__global__ void __launch_bounds__(kTsThreads) tc_scan_kernel(TcScanParams P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint8_t* sA = smem;                 // 128 codes x 128 B (64 BF16 per stage)
  uint8_t* sB = smem + kTsM * 128;    // 128 pairs x 128 B
  __shared__ uint32_t s_taddr;
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ int s_fail;
  __shared__ int s_q[kTsN], s_pp[kTsN], s_sum[kTsN];
  __shared__ float4 s_meta[kTsN];
  __shared__ float s_tau[kTsN];
  __shared__ int s_pos[kTsM];
  __shared__ float4 s_fac[kTsM];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_taddr)),
                 "r"(kTsN));
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
  const uint32_t taddr = s_taddr, bar = smem_u32(&s_bar);
  const uint32_t idesc = make_idesc(1u, kTsM, kTsN);
  const uint32_t lbo = (kTsM / 8) * 128;  // == (kTsN / 8) * 128
  uint32_t phase = 0;
  const int T = P.tile_off[P.K];
  for (int t = blockIdx.x; t < T && !s_fail; t += gridDim.x) {
    // bucket of tile t: the last c with tile_off[c] <= t
    int lo = 0, hi = P.K;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (P.tile_off[mid] <= t) lo = mid; else hi = mid;
    }
    const int c = lo;
    const int cbeg = P.bucket_off[c], Mc = P.bucket_off[c + 1] - cbeg;
    const int pbeg = P.pair_off[P.key_base + c];
    const int Nc = P.pair_off[P.key_base + c + 1] - pbeg;
    const int mt = (Mc + kTsM - 1) / kTsM;
    const int local = t - P.tile_off[c];
    const int m0 = (local % mt) * kTsM, n0 = (local / mt) * kTsN;
    const int rows = min(kTsM, Mc - m0), cols = min(kTsN, Nc - n0);
    {
      const int j = tid;
      if (j < cols) {
        const int pp = P.pair_perm[pbeg + n0 + j];
        const int q = pp / P.nprobe;
        s_pp[j] = pp;
        s_q[j] = q;
        s_meta[j] = P.pmeta[pp];
        s_sum[j] = P.psum[pp];
        s_tau[j] = P.qtau[q];
      }
      const int r = tid;
      if (r < rows) {
        const int pos = cbeg + m0 + r;
        s_pos[r] = pos;
        s_fac[r] = P.factors[pos];
      }
    }
    __syncthreads();
    for (int k0 = 0; k0 < P.dpad; k0 += 64) {
      const int w = k0 >> 6;
      {  // A: the 64 code bits of row `tid` as BF16 0/1 (1.0 = 0x3F80)
        const int r = tid;
        const uint64_t bits = (r < rows) ? __ldg(P.codes + (int64_t)s_pos[r] * P.W + w) : 0ull;
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
          const uint32_t b8 = (uint32_t)(bits >> (8 * ch)) & 0xffu;
          uint32_t v[4];
#pragma unroll
          for (int h = 0; h < 4; ++h)
            v[h] = (((b8 >> (2 * h)) & 1u) ? 0x3F80u : 0u) |
                   (((b8 >> (2 * h + 1)) & 1u) ? 0x3F800000u : 0u);
          *reinterpret_cast<uint4*>(sA + core_off(r, ch, kTsM)) = make_uint4(v[0], v[1], v[2], v[3]);
        }
      }
      {  // B: 64 quantized values of pair column `tid`
        const int j = tid;
        const uint4* src = j < cols ? reinterpret_cast<const uint4*>(P.qub + (int64_t)s_pp[j] * P.dpad + k0)
                                    : nullptr;
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
          const uint4 v = src ? __ldg(src + ch) : make_uint4(0, 0, 0, 0);
          *reinterpret_cast<uint4*>(sB + core_off(j, ch, kTsN)) = v;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (tid == 0) {
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
        for (int st = 0; st < 4; ++st) {  // K = 16 per instruction, 2 chunks each
          const uint64_t da = make_desc(a0 + 2 * st * lbo, lbo, 128);
          const uint64_t db = make_desc(b0 + 2 * st * lbo, lbo, 128);
          const uint32_t acc = (k0 > 0 || st > 0) ? 1u : 0u;
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(taddr),
              "l"(da), "l"(db), "r"(idesc), "r"(acc));
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                bar)
            : "memory");
      }
      if (!mbar_wait(bar, phase)) s_fail = 1;
      phase ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;");
      __syncthreads();
      if (s_fail) break;
    }
    if (s_fail) break;
    // epilogue: thread = code row; 16 pair columns per TMEM load
    const int r = warp * 32 + lane;
    const bool rv = r < rows;
    const float4 f = rv ? s_fac[r] : make_float4(0, 0, 0, 0);
    const int pos = rv ? s_pos[r] : 0;
    for (int c0 = 0; c0 < cols; c0 += 16) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int j = c0 + e;
        const bool valid = rv && j < cols;
        float lb = 0.f, ub = 0.f, dist = 0.f;
        if (valid) {
          const int ip = __float2int_rn(__uint_as_float(v[e]));
          const float4 mt = s_meta[j];
          const float t1 = (float)(2 * ip - s_sum[j]);
          const float xq = __fadd_rn(__fmul_rn(mt.x, t1), __fmul_rn(mt.y, f.w));
          dist = __fsub_rn(__fadd_rn(f.x, mt.w), __fmul_rn(f.y, xq));
          const float er = __fmul_rn(f.z, mt.z);
          lb = __fsub_rn(dist, er);
          ub = __fadd_rn(dist, er);
        }
        const bool app = valid && lb <= s_tau[min(j, kTsN - 1)];
        const unsigned bal = __ballot_sync(kFull, app);
        if (bal) {
          const int q = s_q[j];
          const int leader = __ffs(bal) - 1;
          int base = 0;
          if (lane == leader) base = atomicAdd(P.lcnt + q, __popc(bal));
          base = __shfl_sync(kFull, base, leader);
          if (app) {
            const int slot = base + __popc(bal & ((1u << lane) - 1u));
            if (slot < P.cap)
              P.lists[(int64_t)q * P.cap + slot] =
                  make_int4(pos, __float_as_int(lb), __float_as_int(dist), __float_as_int(ub));
            else
              atomicExch(P.err, 1);
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // TMEM and tile state are reused by the next tile
    asm volatile("tcgen05.fence::after_thread_sync;");
  }
  if (s_fail && tid == 0) atomicExch(P.err, 2);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTsN));
}

// Quantize every (query, cluster) pair to BF16 values (one warp per pair),
// with the same arithmetic as the popcount path.
__global__ void quantize_pairs_kernel(const float* __restrict__ rq,
                                      const int32_t* __restrict__ probe_ids,
                                      const float* __restrict__ probe_dist,
                                      const float* __restrict__ probe_nq2,
                                      const float* __restrict__ ptc, int64_t npairs, int nprobe,
                                      int dpad, int bq, float eps0, uint64_t seed,
                                      int64_t q_offset, __nv_bfloat16* __restrict__ qub,
                                      float4* __restrict__ pmeta, int32_t* __restrict__ psum) {
  const int64_t pp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (pp >= npairs) return;
  const int c = probe_ids[pp];
  if (c < 0) return;
  const int64_t q = pp / nprobe;
  __nv_bfloat16* dst = qub + pp * dpad;
  float vl, delta;
  const int sum = quant_core(rq + q * dpad, ptc + (int64_t)c * dpad, dpad, bq, seed,
                             (uint64_t)(q_offset + q), c, &vl, &delta,
                             [&](int, int k0, const int* qu) {
                               if (k0 < dpad) {  // dpad is a multiple of 64: 4 elements fit
                                 __nv_bfloat162 a = __floats2bfloat162_rn((float)qu[0], (float)qu[1]);
                                 __nv_bfloat162 b = __floats2bfloat162_rn((float)qu[2], (float)qu[3]);
                                 uint2 u;
                                 u.x = *reinterpret_cast<uint32_t*>(&a);
                                 u.y = *reinterpret_cast<uint32_t*>(&b);
                                 *reinterpret_cast<uint2*>(dst + k0) = u;
                               }
                             });
  if (lane == 0) {
    pmeta[pp] = quant_meta(delta, vl, probe_nq2 ? probe_nq2[pp] : probe_dist[pp], probe_dist[pp],
                           eps0, dpad);
    psum[pp] = sum;
  }
}

// Sort keys of the pairs: a pair of probe rank r in pass p (bounds[p] <= r <
// bounds[p + 1]) gets p (K + 1) + cluster; a pair with no probe gets the
// last key, npass (K + 1).
__global__ void pair_keys_kernel(const int32_t* __restrict__ probe_ids, int64_t npairs,
                                 int nprobe, int b1, int b2, int K, int32_t* __restrict__ key) {
  const int64_t pp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pp >= npairs) return;
  const int c = probe_ids[pp];
  const int rank = (int)(pp % nprobe);
  const int pass = rank < b1 ? 0 : (rank < b2 ? 1 : 2);
  key[pp] = c < 0 ? 3 * (K + 1) : pass * (K + 1) + c;
}

// Tiles per bucket of one pass: ceil(codes / 128) * ceil(pairs / 128).
__global__ void tile_count_kernel(const int32_t* __restrict__ bucket_off,
                                  const int32_t* __restrict__ pair_off, int key_base, int K,
                                  int32_t* __restrict__ tiles) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= K) return;
  const int Mc = bucket_off[c + 1] - bucket_off[c];
  const int Nc = pair_off[key_base + c + 1] - pair_off[key_base + c];
  tiles[c] = (Mc > 0 && Nc > 0) ? ((Mc + kTsM - 1) / kTsM) * ((Nc + kTsN - 1) / kTsN) : 0;
}

__global__ void fill_f32_kernel(float* __restrict__ a, int64_t n, float v) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

// Between the passes: tau'_q = k-th smallest UB of the list (if it has k
// entries), and the list keeps LB <= tau'_q. One CTA per query.
__global__ void __launch_bounds__(kThreads) list_threshold_kernel(int4* __restrict__ lists,
                                                                  int32_t* __restrict__ lcnt,
                                                                  int cap, int64_t nq, int k,
                                                                  float* __restrict__ qtau) {
  __shared__ SelState sel;
  __shared__ int s_cnt;
  __shared__ int s_scratch[kCompactU * kThreads / 32];
  for (int64_t q = blockIdx.x; q < nq; q += gridDim.x) {
    int4* L = lists + q * cap;
    if (threadIdx.x == 0) s_cnt = min(lcnt[q], cap);
    __syncthreads();
    const int n = s_cnt;
    float tau = __int_as_float(0x7f800000);
    if (n >= k) {
      const uint32_t T = block_select_f<uint32_t>(
          n, k, sel, [L](int i) { return float_key(__int_as_float(L[i].w)); });
      tau = key_float(T);
      compact_cand(L, &s_cnt, cap, s_scratch,
                   [tau](const int4& e) { return __int_as_float(e.y) <= tau; });
    }
    if (threadIdx.x == 0) {
      qtau[q] = tau;
      lcnt[q] = s_cnt;
    }
    __syncthreads();
  }
}

// The per-query end of a tensor-core search: tau_ub = k-th smallest UB of
// the list, then finish_query. One CTA per query at a time.
__global__ void __launch_bounds__(kThreads) tc_tail_kernel(FusedParams P, int4* lists,
                                                           int32_t* lcnt, int cap) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ int s_cand_cnt, s_top_cnt, s_surv;
  __shared__ int s_scratch[kCompactU * kThreads / 32];
  __shared__ SelState s_sel;
  size_t off[10];
  fused_smem_bytes(P.pch, P.bq, P.W, P.d, P.cu, P.ce, P.ct, blockDim.x >> 5, off);
  FusedSmem S;
  S.planes = nullptr;
  S.pmeta = nullptr;
  S.psum = S.pbeg = S.pref = nullptr;
  S.qv = reinterpret_cast<float*>(smem + off[5]);
  S.sel = &s_sel;
  S.ubk = nullptr;
  S.estk = reinterpret_cast<unsigned long long*>(smem + off[7]);
  S.topk = reinterpret_cast<unsigned long long*>(smem + off[8]);
  for (int64_t q = blockIdx.x; q < P.nq; q += gridDim.x) {
    for (int i = threadIdx.x; i < P.d; i += blockDim.x) S.qv[i] = P.queries[q * P.d + i];
    int4* L = lists + q * cap;
    if (threadIdx.x == 0) s_cand_cnt = min(lcnt[q], cap);
    __syncthreads();
    const int n = s_cand_cnt;
    float tau_ub = __int_as_float(0x7f800000);
    if (n >= P.k)
      tau_ub = key_float(block_select_f<uint32_t>(
          n, P.k, s_sel, [L](int i) { return float_key(__int_as_float(L[i].w)); }));
    TailShared ts{&s_cand_cnt, &s_top_cnt, &s_surv, s_scratch};
    finish_query(P, S, q, L, cap, tau_ub, ts);
    if (P.tr.n_pairs) {  // codes estimated for this query
      int np = P.nprobe;
      if (P.nprobe_q) np = min(max(P.nprobe_q[q], 1), P.nprobe);
      int acc = 0;
      for (int j = threadIdx.x; j < np; j += blockDim.x) {
        const int c = P.probe_ids[q * P.nprobe + j];
        acc += P.bucket_off[c + 1] - P.bucket_off[c];
      }
      acc = warp_sum_i(acc);
      if ((threadIdx.x & 31) == 0) atomicAdd(P.tr.n_pairs + q, acc);
    }
    __syncthreads();
  }
}

typedef void (*FusedFn)(FusedParams);

// Compile-time code lengths of the common shapes (D' = 128, 256, 1024 with
// B_q = 4); everything else runs the generic instance.
FusedFn pick_fused(int W, int bq, bool staged = false) {
  if (bq == 4) {
    if (W == 2) return staged ? fused_search_kernel<2, 4, true> : fused_search_kernel<2, 4>;
    if (W == 4) return staged ? fused_search_kernel<4, 4, true> : fused_search_kernel<4, 4>;
    if (W == 16) return fused_search_kernel<16, 4>;
  }
  return fused_search_kernel<0, 0>;
}

// The warp-per-query kernel for these parameters (null: the CTA kernel
// runs). It covers D' = 128 / 256, B_q = 4, k <= 128, d <= 256, unsplit
// searches without a trace, and batches of at least min_nq queries.
typedef void (*WarpFn)(FusedParams);
constexpr int kWarpCap = 8192;  // candidate entries per warp region (at most max_candidates)

WarpFn pick_warp(const SearchArgs& a) {
  const rabitq_index* X = a.X;
  int32_t path = a.scan_path, layout = a.layout == RABITQ_LAYOUT_AUTO ? a.tile_layout : a.layout,
          ppl = a.ppl, stage = a.stage;
  resolve_tile(X, a.k, a.nprobe, &path, &layout, &ppl, &stage);
  if (layout != RABITQ_LAYOUT_WARP || !a.allow_warp || a.trace || a.bq != 4 ||
      a.k > kWarpMaxK || X->d > 256)
    return nullptr;
  const int lp = ppl ? ppl : (X->W == 2 ? 2 : 1);
  if (X->W == 2) return lp == 1 ? fused_warp_kernel<2, 1> : fused_warp_kernel<2, 2>;
  if (X->W == 4) return lp == 1 ? fused_warp_kernel<4, 1> : fused_warp_kernel<4, 2>;
  return nullptr;
}

int warp_capw(const SearchArgs& a) { return std::min<int>(a.cand_cap, kWarpCap); }

// Resident CTAs of the warp kernel on this device (every SM full).
int warp_ctas(WarpFn fn, int64_t* ctas) {
  int dev = 0, sms = 0, per = 0;
  RBQ_CUDA(cudaGetDevice(&dev));
  RBQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  RBQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kWarpThreads, 0));
  *ctas = (int64_t)sms * std::max(per, 1);
  return RABITQ_OK;
}

// The warp layout pays off once the batch gives every SM several queries
// per scheduler; smaller batches keep eight warps per query (explicit
// RABITQ_LAYOUT_WARP takes it whatever the batch).
bool warp_batch_ok(const SearchArgs& a, int64_t nqc, int64_t ctas) {
  return a.layout == RABITQ_LAYOUT_WARP || nqc * 4 >= ctas * (kWarpThreads / 32);
}

// Work order of the warp layout: each query is one warp's serial work, so
// the batch ends when its longest query does; queries are taken in
// descending order of estimated codes (sum of the probed buckets' sizes, in
// steps of 128; key = kWorkKeys - 1 - steps, sorted stably).
constexpr int kWorkKeys = 1024, kWorkShift = 7;
__global__ void work_key_kernel(const int32_t* __restrict__ probe_ids,
                                const int32_t* __restrict__ npq, int64_t nq, int nprobe,
                                const int32_t* __restrict__ bucket_off, int32_t* __restrict__ key) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int np = npq ? min(max(npq[q], 1), nprobe) : nprobe;
  int64_t w = 0;
  for (int j = 0; j < np; ++j) {
    const int c = probe_ids[q * nprobe + j];
    if (c >= 0) w += bucket_off[c + 1] - bucket_off[c];
  }
  const int64_t steps = w >> kWorkShift;
  key[q] = kWorkKeys - 1 - (int)(steps < kWorkKeys - 1 ? steps : kWorkKeys - 1);
}

// Longest-first order of queries with per-query probe counts: key =
// nprobe - (clamped count), sorted stably (ties keep ascending query id).
__global__ void order_key_kernel(const int32_t* __restrict__ npq, int64_t n, int nprobe,
                                 int32_t* __restrict__ key) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) key[i] = nprobe - min(max(npq[i], 1), nprobe);
}

int pow2_at_least(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// ||q_r - c||^2 of every probed (query, cluster) pair, canonical order (the
// bound's scale for the inner-product metrics, whose probe list holds
// -<q_r, c>); one thread per pair, empty slots (-1) get 0.
__global__ void probe_nq2_kernel(const float* __restrict__ Q, int d,
                                 const float* __restrict__ centroids,
                                 const int32_t* __restrict__ pid, int64_t npairs, int nprobe,
                                 float* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= npairs) return;
  const int c = pid[i];
  float acc = 0.0f;
  if (c >= 0) {
    const float* q = Q + (i / nprobe) * d;
    const float* x = centroids + (int64_t)c * d;
    for (int t = 0; t < d; ++t) acc = score_step<false>(acc, q[t], x[t]);
  }
  out[i] = acc;
}

// ---------------------------------------------------------- single-code estimator
// §3.3.2, first case: one query against one code at a time. One warp per
// (query, slot): the query is quantized against the code's own cluster with
// the bucket scan's arithmetic and random stream (so the values equal the
// scan's), <x_b, q_u> is taken nibble by nibble against the code while the
// quantized values are produced, and lane 0 evaluates the estimator.
struct EstParams {
  const float* queries;     // nq x d (unit rows for the cosine metric)
  const float* rq;          // nq x dpad
  const int64_t* ids;       // nq x m
  const int32_t* inv_perm;  // id -> bucket position
  const int32_t* assign;    // id -> cluster
  const uint64_t* codes;    // bucket order
  const float4* factors;    // bucket order
  const float* centroids;   // K x d
  const float* ptc;         // K x dpad
  int64_t nq, n, q_offset;  // q_offset: stream index of the first query
  int m, d, dpad, bq, metric;
  float eps0;
  uint64_t seed;
  float* out;               // nq x m x 3
  int* err;                 // set to 1 for an id outside [-1, n)
};

__global__ void __launch_bounds__(256) estimate_kernel(EstParams E) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= E.nq * E.m) return;
  const int64_t q = w / E.m;
  const int64_t id = E.ids[w];
  float* o = E.out + 3 * w;
  if (id < 0 || id >= E.n) {
    if (lane == 0) {
      o[0] = o[1] = o[2] = __int_as_float(0x7fc00000);
      if (id != -1) atomicExch(E.err, 1);
    }
    return;
  }
  const int c = E.assign[id];
  const int64_t pos = E.inv_perm[id];
  const int dpad = E.dpad;
  // ||q_r - c||^2 and the additive term (-<q_r, c> for inner products):
  // sequential folds, so one lane
  float nq2 = 0.0f, qc = 0.0f;
  if (lane == 0) {
    const float* qv = E.queries + q * E.d;
    const float* cv = E.centroids + (int64_t)c * E.d;
    for (int t = 0; t < E.d; ++t) {
      const float a = qv[t], b = cv[t];
      nq2 = score_step<false>(nq2, a, b);
      qc = score_step<true>(qc, a, b);
    }
  }
  const uint32_t* code32 = reinterpret_cast<const uint32_t*>(E.codes + pos * (dpad >> 6));
  int ipl = 0;
  float vl, delta;
  const int sum = quant_core(
      E.rq + q * dpad, E.ptc + (int64_t)c * dpad, dpad, E.bq, E.seed, (uint64_t)(E.q_offset + q),
      c, &vl, &delta,
      [&](int, int k0, const int* qu) {
        if (k0 < dpad) {  // the lane's four coordinates k0..k0+3 (code bit k at word k/32)
          const uint32_t nib = (__ldg(code32 + (k0 >> 5)) >> (k0 & 31)) & 0xfu;
          for (int b = 0; b < E.bq; ++b) {
            const uint32_t qn = ((qu[0] >> b) & 1) | (((qu[1] >> b) & 1) << 1) |
                                (((qu[2] >> b) & 1) << 2) | (((qu[3] >> b) & 1) << 3);
            ipl += __popc(qn & nib) << b;
          }
        }
      });
  const int ip = warp_sum_i(ipl);
  if (lane == 0) {
    const float add = E.metric ? -qc : nq2;
    const float4 mt = quant_meta(delta, vl, nq2, add, E.eps0, dpad);
    const float4 f = E.factors[pos];
    // the bucket scan's estimator, same FP32 order
    const float t1 = (float)(2 * ip - sum);
    const float xq = __fadd_rn(__fmul_rn(mt.x, t1), __fmul_rn(mt.y, f.w));
    const float dist = __fsub_rn(__fadd_rn(f.x, mt.w), __fmul_rn(f.y, xq));
    const float e = __fmul_rn(f.z, mt.z);
    const float lb = __fsub_rn(dist, e), ub = __fadd_rn(dist, e);
    if (E.metric) {  // inner product <o_r, q_r> = -score, bounds swapped
      o[0] = -dist;
      o[1] = -ub;
      o[2] = -lb;
    } else {
      o[0] = dist;
      o[1] = lb;
      o[2] = ub;
    }
  }
}

// Shape of the fused kernel for a search: probes staged per chunk, buffer
// sizes, and the shared-memory capacity for staging the tail's candidate
// list -- the largest of 4096, 2048, 1024 entries that keeps the residency
// the kernel has without it (0 if none does). The kernel's dynamic
// shared-memory limit is set once to the device maximum, so concurrent
// searches with different shapes never lower it under each other.
struct FusedShape {
  int pch, pilot_m, cu, ce, ct, scap, per_sm;
  size_t smem;
  FusedFn fn;
};

int fused_shape(const SearchArgs& a, FusedShape* f) {
  const rabitq_index* X = a.X;
  const int nprobe = std::min(a.nprobe, X->K), W = X->W;
  const int plane_bytes = a.bq * W * 8;
  f->pch = std::max(1, std::min(nprobe, (32 * 1024) / plane_bytes));
  f->pilot_m = 4 * a.k;
  f->cu = std::max(1024, pow2_at_least(a.k + kPPT * kThreads));
  f->ce = pow2_at_least(f->pilot_m);
  f->ct = std::max(1024, pow2_at_least(a.k + kThreads));
  // bulk-copy staging of the scan rounds (D' = 128 / 256, B_q = 4): its two
  // stages live in the tail's candidate area, which must hold them
  const bool staged = a.stage == RABITQ_STAGING_BULK && a.bq == 4 && (W == 2 || W == 4);
  const int min_scap = !staged ? 0 : (W == 2 ? stage_bytes<2>(kThreads) : stage_bytes<4>(kThreads)) / 16;
  f->fn = pick_fused(W, a.bq, staged);
  int dev = 0, optin = 0;
  RBQ_CUDA(cudaGetDevice(&dev));
  RBQ_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  RBQ_CUDA(cudaFuncGetAttributes(&fa, f->fn));
  optin -= (int)fa.sharedSizeBytes;  // the limit counts dynamic shared memory only
  RBQ_CUDA(cudaFuncSetAttribute(f->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  const size_t base =
      fused_smem_bytes(f->pch, a.bq, W, X->d, f->cu, f->ce, f->ct, kThreads / 32, nullptr);
  int per_base = 0;
  RBQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_base, f->fn, kThreads, base));
  f->scap = 0;
  f->smem = base;
  f->per_sm = std::max(per_base, 1);
  for (int scap = 4096; scap >= 1024; scap /= 2) {
    if (scap < min_scap) break;
    const size_t sm = fused_smem_bytes(f->pch, a.bq, W, X->d, f->cu, f->ce, f->ct, kThreads / 32,
                                       nullptr, scap);
    if (sm > (size_t)optin) continue;
    int per = 0;
    RBQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f->fn, kThreads, sm));
    if (per >= per_base && per >= 1) {
      f->scap = scap;
      f->smem = sm;
      break;
    }
  }
  if (staged && f->scap < min_scap) {  // the stages first, residency second
    int scap = 1024;
    while (scap < min_scap) scap *= 2;
    f->scap = scap;
    f->smem = fused_smem_bytes(f->pch, a.bq, W, X->d, f->cu, f->ce, f->ct, kThreads / 32, nullptr,
                               scap);
    int per = 0;
    RBQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f->fn, kThreads, f->smem));
    f->per_sm = std::max(per, 1);
  }
  return RABITQ_OK;
}

// Probe lists from the probe keys in cd (probe_keys_tc):
// the nsel (= nprobe, or npq[q] clamped to it) best centroids of each query
// by exact canonical score, ascending (score, id), in rows of nprobe. With
// pre_ids/pre_dist (rows of pre_n such lists), a query with nsel <= pre_n
// copies its prefix instead.
int probe_select(const rabitq_index* X, const float* Q, int64_t nqc, const float* cd, int nprobe,
                 const int32_t* npq, int32_t* ids, float* dist, cudaStream_t s,
                 const int32_t* pre_ids = nullptr, const float* pre_dist = nullptr,
                 int pre_n = 0) {
  if (nqc <= 0) return RABITQ_OK;
  const int sort_n = pow2_at_least(nprobe);
  int dev = 0, optin = 0;
  RBQ_CUDA(cudaGetDevice(&dev));
  RBQ_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  RBQ_CUDA(cudaFuncGetAttributes(&fa, probe_select_kernel));
  const size_t limit = (size_t)(optin - (int)fa.sharedSizeBytes);
  RBQ_CUDA(cudaFuncSetAttribute(probe_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)limit));
  const ProbeScratch v = probe_scratch(X, nqc, const_cast<float*>(cd));
  const size_t smem = probe_select_smem(X->d, sort_n, v.pool_n);
  if (smem > limit) return fail(RABITQ_EINVAL, "probe selection does not fit shared memory");
  probe_select_kernel<<<(unsigned)nqc, kThreads, smem, s>>>(
      Q, X->d, v.keys, v.pool, v.pool_n, v.kmin, v.kmax, v.nq2, X->centroids, X->cnorm,
      X->cnorm_max, X->K, X->metric != RABITQ_METRIC_L2 ? 1 : 0, nprobe, npq, sort_n, pre_ids,
      pre_dist, pre_n, ids, dist);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

// Learned probe counts of one query chunk from its centroid products cd
// (nqc x K): the min(64, K) nearest buckets, then the fused MLP kernel.
int predict_chunk(const SearchArgs& a, const float* Q, const float* cd, int64_t nqc, int64_t q0,
                  int32_t* fid, float* fdist, cudaStream_t s) {
  const int navail = std::min(kMlpIn, a.X->K);
  RBQ_CHECK(probe_select(a.X, Q, nqc, cd, navail, nullptr, fid, fdist, s));
  return mlp_infer(a.pred, fdist, navail, nqc, navail, a.pred_nprobe + q0, nullptr, nullptr, s);
}

}  // namespace

int search_dev_tc(const SearchArgs& a, cudaStream_t s);

int search_dev_popc(const SearchArgs& a, cudaStream_t s);

namespace {

// Metric plumbing shared by the search paths. COSINE searches the unit
// query (normalized first); the inner-product metrics rank centroids by
// -<q_r, c> and need ||q_r - c||^2 of each probed pair for the bound.
bool metric_ip(const rabitq_index* X) { return X->metric != RABITQ_METRIC_L2; }
bool metric_cos(const rabitq_index* X) { return X->metric == RABITQ_METRIC_COSINE; }

// Q for the search: the caller's rows, or their unit rows in qn (COSINE).
int search_queries(const rabitq_index* X, const float* Q, int64_t nq, float* qn,
                   const float** out, cudaStream_t s) {
  *out = Q;
  if (metric_cos(X)) {
    RBQ_CHECK(normalize_rows(Q, nq, X->d, qn, s));
    *out = qn;
  }
  return RABITQ_OK;
}

// The probe filter's keys for all K centroids from tensor-core products
// (probe_select turns them into exact probe lists).
int centroid_scores(const rabitq_index* X, const float* Q, int64_t nq, float* cd, int* err,
                    cudaStream_t s) {
  return probe_keys_tc(X, Q, nq, cd, err, s);
}

int probe_nq2(const rabitq_index* X, const float* Q, int64_t nq, int nprobe, const int32_t* pid,
              float* out, cudaStream_t s) {
  const int64_t np = nq * nprobe;
  if (np == 0) return RABITQ_OK;
  probe_nq2_kernel<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(Q, X->d, X->centroids, pid, np,
                                                               nprobe, out);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

}  // namespace

namespace {
// Probe slices per query for a chunk of nqc queries: 1 when the queries fill
// the GPU (full = resident CTAs); otherwise up to 16, no more than the probes,
// and the slices' k smallest upper bounds must fit the merge's buffer.
int split_factor(const SearchArgs& a, int64_t nqc, int64_t full, const FusedShape& fs) {
  if (a.trace || !a.allow_split || nqc * 2 > full) return 1;
  int sp = (int)std::min<int64_t>(16, full / std::max<int64_t>(nqc, 1));
  sp = std::min(sp, std::min(a.nprobe, a.X->K));
  sp = std::min(sp, fs.cu / std::max(a.k, 1));
  return std::max(1, sp);
}

int set_merge_attr() {
  int dev = 0, optin = 0;
  RBQ_CUDA(cudaGetDevice(&dev));
  RBQ_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  RBQ_CUDA(cudaFuncGetAttributes(&fa, split_merge_kernel));
  RBQ_CUDA(cudaFuncSetAttribute(split_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes));
  return RABITQ_OK;
}
}  // namespace

// One warp-layout launch for the queries of P (P.next zeroed by the
// caller), then the CTA kernel over the queries it handed back (redo: [0]
// count, [32] work counter, list from [64]; an empty list ends that launch at
// once). Allocation- and synchronization-free (graph capturable).
struct WarpScratch {
  int4* candw;       // per-warp candidate regions
  int capw;
  int* redo;         // [0] count, [32] redo work counter, list from [64]
  int32_t* wkey;     // nq work keys
  int32_t* worder;   // nq: the work order
  int32_t* wooff;    // kWorkKeys + 1
  int32_t* wsortws;  // counting_sort_ws_ints(nq, kWorkKeys)
};

int launch_warp(WarpFn wfn, int64_t wctas, const FusedParams& P, const WarpScratch& ws, FusedFn fn,
                unsigned grid, size_t smem, cudaStream_t s) {
  RBQ_CUDA(cudaMemsetAsync(ws.redo, 0, sizeof(int) * 64, s));
  work_key_kernel<<<(unsigned)((P.nq + 255) / 256), 256, 0, s>>>(
      P.probe_ids, P.nprobe_q, P.nq, P.nprobe, P.bucket_off, ws.wkey);
  RBQ_CUDA(cudaGetLastError());
  RBQ_CHECK(order_sort(ws.wkey, P.nq, kWorkKeys, ws.worder, ws.wooff, ws.wsortws, s));
  int* redo = ws.redo;
  FusedParams W = P;
  W.candw = ws.candw;
  W.capw = ws.capw;
  W.order = ws.worder;
  W.redo = redo + 64;
  W.redo_cnt = redo;
  const int64_t need = (P.nq + (kWarpThreads / 32) - 1) / (kWarpThreads / 32);
  wfn<<<(unsigned)std::min<int64_t>(wctas, need), kWarpThreads, 0, s>>>(W);
  RBQ_CUDA(cudaGetLastError());
  FusedParams R = P;
  R.order = redo + 64;
  R.nq_dev = redo;
  R.next = redo + 32;
  R.split = 1;
  fn<<<grid, kThreads, smem, s>>>(R);
  RBQ_CUDA(cudaGetLastError());
  return RABITQ_OK;
}

// Scan-path choice: the index's tuned choice for AUTO (set by
// rabitq_autotune), the popcount path otherwise; a TC search whose candidate
// lists overflow under AUTO is redone on the popcount path.
int tile_class_k(int k) { return k <= 16 ? 0 : (k <= 64 ? 1 : (k <= 128 ? 2 : 3)); }
int tile_class_np(int nprobe) { return nprobe <= 16 ? 0 : (nprobe <= 64 ? 1 : (nprobe <= 256 ? 2 : 3)); }

// AUTO choices: the tuned tile of the shape's class, else the index-wide
// path choice of rabitq_autotune and the default layout (one warp per
// query for k <= 32, where its shorter tail wins; one CTA per query above).
void resolve_tile(const rabitq_index* X, int k, int nprobe, int32_t* path, int32_t* layout,
                  int32_t* ppl, int32_t* stage) {
  const rabitq_index::Tile& t = X->tune[tile_class_k(k)][tile_class_np(nprobe)];
  if (*path == RABITQ_SCAN_AUTO)
    *path = t.valid ? t.path : (X->tuned_path ? X->tuned_path : RABITQ_SCAN_POPC);
  if (*layout == RABITQ_LAYOUT_AUTO)
    *layout = t.valid ? t.layout
                      : (X->tuned_layout ? X->tuned_layout
                                         : (k <= 32 ? RABITQ_LAYOUT_WARP : RABITQ_LAYOUT_CTA));
  if (*ppl == 0) *ppl = t.valid ? t.ppl : 0;
  if (*stage == RABITQ_STAGING_AUTO)  // bulk staging measured slower on GB300 (tuner only)
    *stage = t.valid && t.stage ? t.stage : RABITQ_STAGING_OFF;
}

int search_dev(const SearchArgs& a_in, cudaStream_t s) {
  SearchArgs a = a_in;
  const bool auto_path = a.scan_path == RABITQ_SCAN_AUTO;
  a.tile_layout = a.layout;
  resolve_tile(a.X, a.k, a.nprobe, &a.scan_path, &a.tile_layout, &a.ppl, &a.stage);
  if (a.scan_path == RABITQ_SCAN_TC) {
    const int st = search_dev_tc(a, s);
    if (!(auto_path && st == RABITQ_EOVERFLOW)) return st;
    a.scan_path = RABITQ_SCAN_POPC;  // a tuned choice that overflowed: redone on popcount
  }
  return search_dev_popc(a, s);
}

int search_dev_popc(const SearchArgs& a, cudaStream_t s) {
  const rabitq_index* X = a.X;
  const int K = X->K, d = X->d, dpad = X->dpad, W = X->W;
  const int nprobe = std::min(a.nprobe, K);
  if (a.nq == 0) return RABITQ_OK;
  int dev = 0, sms = 0;
  RBQ_CUDA(cudaGetDevice(&dev));
  RBQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

  // fused-kernel shape
  FusedShape fs;
  RBQ_CHECK(fused_shape(a, &fs));
  const int pch = fs.pch, pilot_m = fs.pilot_m, cu = fs.cu, ce = fs.ce, ct = fs.ct;
  const size_t smem = fs.smem;
  const FusedFn fn = fs.fn;
  const int per_sm = fs.per_sm;

  // query chunks bound the centroid-distance scratch (<= 256 Mi floats)
  const int64_t qchunk = std::max<int64_t>(1, std::min<int64_t>(a.nq, (int64_t(1) << 28) / K));
  const int64_t full = (int64_t)sms * per_sm;
  const int64_t grid = std::min<int64_t>(qchunk, full);
  // a batch too small to fill the GPU splits each query's probes over CTAs
  const int split = split_factor(a, std::min(qchunk, a.nq), full, fs);
  // the warp-per-query layout, where it applies: per-warp candidate regions
  // and the redo list ([0] count, [32] the redo launch's work counter, the
  // list from [64])
  const WarpFn wfn = split > 1 ? nullptr : pick_warp(a);
  int64_t wctas = 0;
  if (wfn) RBQ_CHECK(warp_ctas(wfn, &wctas));
  const int capw = warp_capw(a);
  DevBuf candw, redo, wkey, worder, wooff, wsortws;
  if (wfn) {
    RBQ_CHECK(candw.alloc(sizeof(int4) * wctas * (kWarpThreads / 32) * capw, s));
    RBQ_CHECK(redo.alloc(sizeof(int32_t) * (qchunk + 64), s));
    RBQ_CHECK(wkey.alloc(sizeof(int32_t) * qchunk, s));
    RBQ_CHECK(worder.alloc(sizeof(int32_t) * qchunk, s));
    RBQ_CHECK(wooff.alloc(sizeof(int32_t) * (kWorkKeys + 1), s));
    RBQ_CHECK(wsortws.alloc(sizeof(int32_t) * counting_sort_ws_ints(qchunk, kWorkKeys), s));
  }
  DevBuf cd, rq, pid, pdist, cand, err, ubout, scnt, cand2, qn, pnq2;
  if (metric_cos(X)) RBQ_CHECK(qn.alloc(sizeof(float) * qchunk * d, s));
  if (metric_ip(X)) RBQ_CHECK(pnq2.alloc(sizeof(float) * qchunk * nprobe, s));
  RBQ_CHECK(cd.alloc(sizeof(float) * probe_scratch_floats(X, qchunk), s));
  RBQ_CHECK(rq.alloc(sizeof(float) * qchunk * dpad, s));
  RBQ_CHECK(pid.alloc(sizeof(int32_t) * qchunk * nprobe, s));
  RBQ_CHECK(pdist.alloc(sizeof(float) * qchunk * nprobe, s));
  RBQ_CHECK(cand.alloc(sizeof(int4) * std::max<int64_t>(grid, qchunk * split) * a.cand_cap, s));
  RBQ_CHECK(err.alloc(sizeof(int), s));
  if (split > 1) {
    RBQ_CHECK(ubout.alloc(sizeof(uint32_t) * qchunk * split * a.k, s));
    RBQ_CHECK(scnt.alloc(sizeof(int) * qchunk * split * 2, s));
    RBQ_CHECK(cand2.alloc(sizeof(int4) * qchunk * a.cand_cap, s));
    RBQ_CHECK(set_merge_attr());
  }
  // dynamic query scheduling; with per-query probe counts, longest first
  DevBuf nextc, okey, order, ooff;
  RBQ_CHECK(nextc.alloc(sizeof(int), s));
  if (a.pred || a.per_query_nprobe) {
    RBQ_CHECK(okey.alloc(sizeof(int32_t) * qchunk, s));
    RBQ_CHECK(order.alloc(sizeof(int32_t) * qchunk, s));
    RBQ_CHECK(ooff.alloc(sizeof(int32_t) * (nprobe + 2), s));
  }
  DevBuf fid, fdist;  // learned probe counts: the 64 nearest buckets per query
  if (a.pred) {
    RBQ_CHECK(fid.alloc(sizeof(int32_t) * qchunk * kMlpIn, s));
    RBQ_CHECK(fdist.alloc(sizeof(float) * qchunk * kMlpIn, s));
  }
  RBQ_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));

  cudaEvent_t ev[5] = {};
  const bool timing = a.stage_ms != nullptr;
  float acc_ms[4] = {0, 0, 0, 0};
  if (timing)
    for (auto& e : ev) RBQ_CUDA(cudaEventCreate(&e));

  for (int64_t q0 = 0; q0 < a.nq; q0 += qchunk) {
    const int64_t nqc = std::min(qchunk, a.nq - q0);
    if (timing) RBQ_CUDA(cudaEventRecord(ev[0], s));
    const float* Q = nullptr;
    RBQ_CHECK(search_queries(X, a.queries + q0 * d, nqc, qn.as<float>(), &Q, s));
    RBQ_CHECK(centroid_scores(X, Q, nqc, cd.as<float>(), err.as<int>(), s));
    if (timing) RBQ_CUDA(cudaEventRecord(ev[1], s));
    int32_t* probe_ids = a.trace && a.trace->probe_ids ? a.trace->probe_ids + q0 * nprobe
                                                       : pid.as<int32_t>();
    float* probe_dist = a.trace && a.trace->probe_dist ? a.trace->probe_dist + q0 * nprobe
                                                       : pdist.as<float>();
    const int32_t* npq = a.per_query_nprobe ? a.per_query_nprobe + q0 : nullptr;
    // learned counts: the 64 nearest buckets give the features, the network
    // gives each query's count, and the probe list then holds that many (a
    // selection of nprobe_max for every query would cost more: most need few)
    if (a.pred) {
      RBQ_CHECK(predict_chunk(a, Q, cd.as<float>(), nqc, q0, fid.as<int32_t>(),
                              fdist.as<float>(), s));
      npq = a.pred_nprobe + q0;
    }
    RBQ_CHECK(probe_select(X, Q, nqc, cd.as<float>(), nprobe, npq, probe_ids, probe_dist, s,
                           a.pred ? fid.as<int32_t>() : nullptr, fdist.as<float>(),
                           std::min(kMlpIn, K)));
    if (metric_ip(X)) RBQ_CHECK(probe_nq2(X, Q, nqc, nprobe, probe_ids, pnq2.as<float>(), s));
    if (timing) RBQ_CUDA(cudaEventRecord(ev[2], s));
    float* rqp = a.trace && a.trace->rq ? a.trace->rq + q0 * dpad : rq.as<float>();
    if (a.rot_precision == RABITQ_ROT_FP32)
      RBQ_CHECK(gemm_canon(kDot, Q, d, nullptr, nullptr, 0, nullptr, X->P32, dpad, rqp, dpad, nqc,
                           dpad, d, s));
    else
      RBQ_CHECK(rotate_tc(X, Q, nqc, a.rot_precision, rqp, err.as<int>(), s));
    if (timing) RBQ_CUDA(cudaEventRecord(ev[3], s));
    FusedParams P;
    std::memset(&P, 0, sizeof P);
    P.queries = Q;
    P.rq = rqp;
    P.probe_ids = probe_ids;
    P.probe_dist = probe_dist;
    P.probe_nq2 = metric_ip(X) ? pnq2.as<float>() : nullptr;
    P.metric = metric_ip(X);
    P.nprobe_q = npq;
    P.ptc = X->ptc;
    P.codes = X->codes;
    P.factors = X->factors;
    P.data_b = X->data_b;
    P.perm = X->perm;
    P.inv_perm = X->inv_perm;
    P.bucket_off = X->bucket_off;
    P.nq = nqc;
    P.q_offset = q0;
    P.d = d;
    P.dpad = dpad;
    P.W = W;
    P.bq = a.bq;
    P.k = a.k;
    P.nprobe = nprobe;
    P.pch = pch;
    P.m = pilot_m;
    P.cu = cu;
    P.ce = ce;
    P.ct = ct;
    P.scap = fs.scap;
    P.eps0 = a.eps0;
    P.seed = a.seed;
    P.cand_cap = a.cand_cap;
    P.cand = cand.as<int4>();
    P.out_ids = a.out_ids + q0 * a.k;
    P.out_dist = a.out_dist + q0 * a.k;
    P.err = err.as<int>();
    P.next = nextc.as<int>();
    RBQ_CUDA(cudaMemsetAsync(nextc.p, 0, sizeof(int), s));
    if (npq) {
      order_key_kernel<<<(unsigned)((nqc + 255) / 256), 256, 0, s>>>(npq, nqc, nprobe,
                                                                    okey.as<int32_t>());
      if (order_sort_fits(nqc, nprobe + 1))
        RBQ_CHECK(order_sort(okey.as<int32_t>(), nqc, nprobe + 1, order.as<int32_t>(),
                             ooff.as<int32_t>(), nullptr, s));
      else
        RBQ_CHECK(counting_sort(okey.as<int32_t>(), nqc, nprobe + 1, order.as<int32_t>(),
                                ooff.as<int32_t>(), s));
      P.order = order.as<int32_t>();
    }
    if (a.trace) {
      const rabitq_trace& T = *a.trace;
      P.tr = T;
      // per-query trace arrays are offset to this chunk
      P.tr.probe_ids = nullptr;
      P.tr.probe_dist = nullptr;
      P.tr.rq = nullptr;
      if (T.planes) P.tr.planes = T.planes + q0 * nprobe * a.bq * W;
      if (T.sum_qu) P.tr.sum_qu = T.sum_qu + q0 * nprobe;
      if (T.meta) P.tr.meta = T.meta + q0 * nprobe * 4;
      if (T.n_pairs) P.tr.n_pairs = T.n_pairs + q0;
      if (T.pair_id) {
        P.tr.pair_id = T.pair_id + q0 * T.pair_cap;
        P.tr.pair_ip = T.pair_ip + q0 * T.pair_cap;
        P.tr.pair_est = T.pair_est + q0 * T.pair_cap * 3;
      }
      if (T.tau_ub) P.tr.tau_ub = T.tau_ub + q0;
      if (T.tau1) P.tr.tau1 = T.tau1 + q0;
      if (T.tau) P.tr.tau = T.tau + q0;
      if (T.n_surv) P.tr.n_surv = T.n_surv + q0;
      if (T.surv_ids) P.tr.surv_ids = T.surv_ids + q0 * T.surv_cap;
    }
    P.split = split;
    if (split > 1) {
      P.ub_out = ubout.as<uint32_t>();
      P.slice_cnt = scnt.as<int>();
      P.cand2 = cand2.as<int4>();
    }
    if (wfn && warp_batch_ok(a, nqc, wctas)) {
      const WarpScratch ws{candw.as<int4>(), capw, redo.as<int>(), wkey.as<int32_t>(),
                           worder.as<int32_t>(), wooff.as<int32_t>(), wsortws.as<int32_t>()};
      RBQ_CHECK(launch_warp(wfn, wctas, P, ws, fn, (unsigned)grid, smem, s));
    } else {
      const unsigned g = (unsigned)std::min<int64_t>(nqc * split, split > 1 ? full : grid);
      fn<<<g, kThreads, smem, s>>>(P);
      RBQ_CUDA(cudaGetLastError());
      if (split > 1) {
        split_merge_kernel<<<(unsigned)std::min<int64_t>(nqc, full), kThreads, smem, s>>>(P);
        RBQ_CUDA(cudaGetLastError());
      }
    }
    if (timing) {
      RBQ_CUDA(cudaEventRecord(ev[4], s));
      RBQ_CUDA(cudaEventSynchronize(ev[4]));
      for (int i = 0; i < 4; ++i) {
        float t = 0;
        RBQ_CUDA(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
        acc_ms[i] += t;
      }
    }
  }
  int h_err = 0;
  RBQ_CUDA(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaStreamSynchronize(s));
  if (timing) {
    for (int i = 0; i < 4; ++i) a.stage_ms[i] = acc_ms[i];
    for (auto& e : ev) cudaEventDestroy(e);
  }
  if (h_err == 2)
    return fail(RABITQ_ETIMEOUT, "a tensor-core wait expired (probe scores or query rotation)");
  if (h_err)
    return fail(RABITQ_EOVERFLOW,
                "a query's candidate list exceeded max_candidates; raise max_candidates");
  return RABITQ_OK;
}

// ---------------------------------------------- carved (allocation-free) path
// The popcount pipeline with every scratch array carved out of one device
// buffer: no allocation and no host synchronization between the launches, so
// the whole sequence can also be captured in a CUDA graph (search plans).
//
// Layout: [flags (error, work counter) | candidate lists (grid x cap) |
// per-chunk arrays for qchunk queries].
namespace {

struct Carve {
  int64_t grid = 0, cap = 0, qchunk = 0;
  size_t o_ubout = 0, o_scnt = 0, o_cand2 = 0;  // split mode (grid-sized)
  size_t o_cand = 0, o_cd = 0, o_rq = 0, o_pid = 0, o_pdist = 0, o_pnp = 0, o_fid = 0,
         o_fdist = 0, o_okey = 0, o_order = 0, o_ooff = 0, o_sortws = 0, o_qn = 0, o_pnq2 = 0,
         end = 0;
  // warp layout: its kernel (null = not used), resident CTAs, per-warp
  // candidate regions and the redo list
  WarpFn wfn = nullptr;
  int64_t wctas = 0;
  int capw = 0;
  size_t o_candw = 0, o_redo = 0, o_wkey = 0, o_worder = 0, o_wooff = 0, o_wsortws = 0;
};

constexpr size_t kCarveAlign = 256;

// Offsets for the given grid, candidate capacity and query chunk.
Carve carve_layout(const SearchArgs& a, int64_t grid, int64_t cap, int64_t qchunk) {
  const rabitq_index* X = a.X;
  const int K = X->K, nprobe = std::min(a.nprobe, K);
  const bool ordered = a.pred || a.per_query_nprobe;
  const bool own_select = a.pred != nullptr;
  Carve L;
  L.grid = grid;
  L.cap = cap;
  L.qchunk = qchunk;
  size_t o = kCarveAlign;  // the flags
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, kCarveAlign);
    return at;
  };
  L.o_cand = take(sizeof(int4) * grid * cap);
  L.o_cd = take(sizeof(float) * probe_scratch_floats(X, qchunk));
  L.o_rq = take(sizeof(float) * qchunk * X->dpad);
  L.o_pid = take(sizeof(int32_t) * qchunk * nprobe);
  L.o_pdist = take(sizeof(float) * qchunk * nprobe);
  L.o_pnp = take(a.pred ? sizeof(int32_t) * qchunk : 0);
  L.o_fid = take(own_select ? sizeof(int32_t) * qchunk * kMlpIn : 0);
  L.o_fdist = take(own_select ? sizeof(float) * qchunk * kMlpIn : 0);
  L.o_okey = take(ordered ? sizeof(int32_t) * qchunk : 0);
  L.o_order = take(ordered ? sizeof(int32_t) * qchunk : 0);
  L.o_ooff = take(ordered ? sizeof(int32_t) * (nprobe + 2) : 0);
  L.o_sortws = take(ordered ? sizeof(int32_t) * counting_sort_ws_ints(qchunk, nprobe + 1) : 0);
  L.o_qn = take(metric_cos(X) ? sizeof(float) * qchunk * X->d : 0);
  L.o_pnq2 = take(metric_ip(X) ? sizeof(float) * qchunk * nprobe : 0);
  // split mode: at most grid items (slices) and grid / 2 queries
  L.o_ubout = take(a.allow_split ? sizeof(uint32_t) * grid * a.k : 0);
  L.o_scnt = take(a.allow_split ? sizeof(int) * grid * 2 : 0);
  L.o_cand2 = take(a.allow_split ? sizeof(int4) * (grid / 2) * cap : 0);
  L.wfn = pick_warp(a);
  if (L.wfn && warp_ctas(L.wfn, &L.wctas) != RABITQ_OK) L.wfn = nullptr;
  if (L.wfn) {
    L.capw = warp_capw(a);
    L.o_candw = take(sizeof(int4) * L.wctas * (kWarpThreads / 32) * L.capw);
    L.o_redo = take(sizeof(int32_t) * (qchunk + 64));
    L.o_wkey = take(sizeof(int32_t) * qchunk);
    L.o_worder = take(sizeof(int32_t) * qchunk);
    L.o_wooff = take(sizeof(int32_t) * (kWorkKeys + 1));
    L.o_wsortws = take(sizeof(int32_t) * counting_sort_ws_ints(qchunk, kWorkKeys));
  }
  L.end = o;
  return L;
}

}  // namespace

size_t carved_bytes(const SearchArgs& a, int64_t grid, int64_t nq_max) {
  return carve_layout(a, grid, a.cand_cap, std::max<int64_t>(nq_max, 1)).end;
}

int fused_grid(const SearchArgs& a, int* grid_out) {
  FusedShape fs;
  RBQ_CHECK(fused_shape(a, &fs));
  int dev = 0, sms = 0;
  RBQ_CUDA(cudaGetDevice(&dev));
  RBQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  *grid_out = sms * fs.per_sm;
  return RABITQ_OK;
}

// Enqueue the search of a.nq queries (chunks of what fits) on stream s. The
// error flag is the first int of the scratch (1 = candidate overflow,
// 2 = tensor-core wait expired); the caller zeroes it before the first call
// and reads it after the stream has drained. grid: CTAs of the fused kernel
// (0 = one per SM); cap: candidate capacity per CTA.
int search_enqueue_carved(const SearchArgs& a, unsigned char* scratch, size_t scratch_bytes,
                          int64_t grid, int64_t cap, cudaStream_t s) {
  const rabitq_index* X = a.X;
  const int K = X->K, d = X->d, dpad = X->dpad, W = X->W;
  const int nprobe = std::min(a.nprobe, K);
  if (a.nq == 0) return RABITQ_OK;
  if (grid <= 0) {
    int dev = 0, sms = 0;
    RBQ_CUDA(cudaGetDevice(&dev));
    RBQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    grid = sms;
  }
  FusedShape fs;
  RBQ_CHECK(fused_shape(a, &fs));
  const int pch = fs.pch, pilot_m = fs.pilot_m, cu = fs.cu, ce = fs.ce, ct = fs.ct;
  const size_t smem = fs.smem;
  const FusedFn fn = fs.fn;
  if (cap < 4096) return fail(RABITQ_EINVAL, "search scratch too small for the candidate lists");
  int64_t lo = 1, hi = a.nq;
  if (carve_layout(a, grid, cap, 1).end > scratch_bytes)
    return fail(RABITQ_EINVAL,
                "one query's distances to every centroid do not fit in the search scratch "
                "(K too large)");
  while (lo < hi) {  // largest chunk that fits
    const int64_t mid = lo + (hi - lo + 1) / 2;
    if (carve_layout(a, grid, cap, mid).end <= scratch_bytes) lo = mid; else hi = mid - 1;
  }
  const Carve L = carve_layout(a, grid, cap, lo);
  const int64_t qchunk = L.qchunk;
  int* err = reinterpret_cast<int*>(scratch);
  int* next = reinterpret_cast<int*>(scratch + 64);
  int4* cand = reinterpret_cast<int4*>(scratch + L.o_cand);
  float* cd = reinterpret_cast<float*>(scratch + L.o_cd);
  float* rq = reinterpret_cast<float*>(scratch + L.o_rq);
  int32_t* pid = reinterpret_cast<int32_t*>(scratch + L.o_pid);
  float* pdist = reinterpret_cast<float*>(scratch + L.o_pdist);
  int32_t* pnp = reinterpret_cast<int32_t*>(scratch + L.o_pnp);
  int32_t* fid = reinterpret_cast<int32_t*>(scratch + L.o_fid);
  float* fdist = reinterpret_cast<float*>(scratch + L.o_fdist);
  int32_t* okey = reinterpret_cast<int32_t*>(scratch + L.o_okey);
  int32_t* order = reinterpret_cast<int32_t*>(scratch + L.o_order);
  int32_t* ooff = reinterpret_cast<int32_t*>(scratch + L.o_ooff);
  int32_t* sortws = reinterpret_cast<int32_t*>(scratch + L.o_sortws);
  float* qn = reinterpret_cast<float*>(scratch + L.o_qn);
  float* pnq2 = reinterpret_cast<float*>(scratch + L.o_pnq2);
  const int navail = std::min(kMlpIn, K);
  for (int64_t q0 = 0; q0 < a.nq; q0 += qchunk) {
    const int64_t nqc = std::min(qchunk, a.nq - q0);
    const bool ev = a.stage_ev && q0 == 0 && nqc == a.nq;
    if (ev) RBQ_CUDA(cudaEventRecordWithFlags(a.stage_ev[0], s, cudaEventRecordExternal));
    const float* Q = nullptr;
    RBQ_CHECK(search_queries(X, a.queries + q0 * d, nqc, qn, &Q, s));
    RBQ_CHECK(centroid_scores(X, Q, nqc, cd, err, s));
    if (ev) RBQ_CUDA(cudaEventRecordWithFlags(a.stage_ev[1], s, cudaEventRecordExternal));
    const int32_t* npq = a.per_query_nprobe ? a.per_query_nprobe + q0 : nullptr;
    if (a.pred) {  // the 64 nearest give the features, the network each query's count
      RBQ_CHECK(probe_select(X, Q, nqc, cd, navail, nullptr, fid, fdist, s));
      RBQ_CHECK(mlp_infer(a.pred, fdist, navail, nqc, navail, pnp, nullptr, nullptr, s));
      npq = pnp;
    }
    RBQ_CHECK(probe_select(X, Q, nqc, cd, nprobe, npq, pid, pdist, s, a.pred ? fid : nullptr,
                           fdist, navail));
    if (a.pred && a.pred_nprobe)
      RBQ_CUDA(cudaMemcpyAsync(a.pred_nprobe + q0, pnp, sizeof(int32_t) * nqc,
                               cudaMemcpyDeviceToDevice, s));
    if (metric_ip(X)) RBQ_CHECK(probe_nq2(X, Q, nqc, nprobe, pid, pnq2, s));
    if (ev) RBQ_CUDA(cudaEventRecordWithFlags(a.stage_ev[2], s, cudaEventRecordExternal));
    if (a.rot_precision == RABITQ_ROT_FP32)
      RBQ_CHECK(gemm_canon(kDot, Q, d, nullptr, nullptr, 0, nullptr, X->P32, dpad, rq, dpad, nqc,
                           dpad, d, s));
    else
      RBQ_CHECK(rotate_tc(X, Q, nqc, a.rot_precision, rq, err, s));
    if (ev) RBQ_CUDA(cudaEventRecordWithFlags(a.stage_ev[3], s, cudaEventRecordExternal));
    FusedParams P;
    std::memset(&P, 0, sizeof P);
    P.queries = Q;
    P.rq = rq;
    P.probe_ids = pid;
    P.probe_dist = pdist;
    P.probe_nq2 = metric_ip(X) ? pnq2 : nullptr;
    P.metric = metric_ip(X);
    P.nprobe_q = npq;
    P.ptc = X->ptc;
    P.codes = X->codes;
    P.factors = X->factors;
    P.data_b = X->data_b;
    P.perm = X->perm;
    P.inv_perm = X->inv_perm;
    P.bucket_off = X->bucket_off;
    P.nq = nqc;
    P.q_offset = q0;
    P.d = d;
    P.dpad = dpad;
    P.W = W;
    P.bq = a.bq;
    P.k = a.k;
    P.nprobe = nprobe;
    P.pch = pch;
    P.m = pilot_m;
    P.cu = cu;
    P.ce = ce;
    P.ct = ct;
    P.scap = fs.scap;
    P.eps0 = a.eps0;
    P.seed = a.seed;
    P.cand_cap = (int)cap;
    P.cand = cand;
    P.out_ids = a.out_ids + q0 * a.k;
    P.out_dist = a.out_dist + q0 * a.k;
    P.err = err;
    P.next = next;
    RBQ_CUDA(cudaMemsetAsync(next, 0, sizeof(int), s));
    if (npq) {
      order_key_kernel<<<(unsigned)((nqc + 255) / 256), 256, 0, s>>>(npq, nqc, nprobe, okey);
      RBQ_CUDA(cudaGetLastError());
      RBQ_CHECK(order_sort(okey, nqc, nprobe + 1, order, ooff, sortws, s));
      P.order = order;
    }
    const int split = a.allow_split ? split_factor(a, nqc, grid, fs) : 1;
    P.split = split;
    if (split > 1) {
      P.ub_out = reinterpret_cast<uint32_t*>(scratch + L.o_ubout);
      P.slice_cnt = reinterpret_cast<int*>(scratch + L.o_scnt);
      P.cand2 = reinterpret_cast<int4*>(scratch + L.o_cand2);
    }
    if (split == 1 && L.wfn && warp_batch_ok(a, nqc, L.wctas)) {
      const WarpScratch ws{reinterpret_cast<int4*>(scratch + L.o_candw), L.capw,
                           reinterpret_cast<int*>(scratch + L.o_redo),
                           reinterpret_cast<int32_t*>(scratch + L.o_wkey),
                           reinterpret_cast<int32_t*>(scratch + L.o_worder),
                           reinterpret_cast<int32_t*>(scratch + L.o_wooff),
                           reinterpret_cast<int32_t*>(scratch + L.o_wsortws)};
      RBQ_CHECK(launch_warp(L.wfn, L.wctas, P, ws, fn, (unsigned)grid, smem, s));
    } else {
      fn<<<(unsigned)std::min<int64_t>(nqc * split, grid), kThreads, smem, s>>>(P);
      RBQ_CUDA(cudaGetLastError());
      if (split > 1) {
        RBQ_CHECK(set_merge_attr());
        split_merge_kernel<<<(unsigned)std::min<int64_t>(nqc, grid), kThreads, smem, s>>>(P);
        RBQ_CUDA(cudaGetLastError());
      }
    }
    if (ev) RBQ_CUDA(cudaEventRecordWithFlags(a.stage_ev[4], s, cudaEventRecordExternal));
  }
  return RABITQ_OK;
}

int search_dev_prealloc(const SearchArgs& a_in, unsigned char* scratch, size_t scratch_bytes,
                        cudaStream_t s) {
  if (a_in.nq == 0) return RABITQ_OK;
  SearchArgs a = a_in;
  a.allow_split = 0;  // the fixed scratch has no room for the split buffers
  // flags: err[0] = search error (1 = candidate overflow, 2 = expired wait),
  // err[1] = a query value is not finite; both must start at zero (the
  // carved layout keeps the first 256 bytes for flags; the work counter is at
  // byte 64)
  int* err = reinterpret_cast<int*>(scratch);
  RBQ_CUDA(cudaMemsetAsync(err, 0, 2 * sizeof(int), s));
  RBQ_CHECK(finite_flag(a.queries, a.nq * a.X->d, err + 1, s));
  // one CTA per SM; the candidate lists take at most half of the scratch
  int dev = 0, sms = 0;
  RBQ_CUDA(cudaGetDevice(&dev));
  RBQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t cap = std::min<int64_t>(
      a.cand_cap, (int64_t)((scratch_bytes / 2 - kCarveAlign) / (sizeof(int4) * sms)));
  RBQ_CHECK(search_enqueue_carved(a, scratch, scratch_bytes, sms, cap, s));
  int h_err[2] = {0, 0};
  RBQ_CUDA(cudaMemcpyAsync(h_err, err, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaStreamSynchronize(s));
  if (h_err[1])
    return fail(RABITQ_EINVAL, "a query has a non-finite value (outputs undefined)");
  if (h_err[0] == 2) return fail(RABITQ_ETIMEOUT, "a tensor-core wait expired (probe scores or query rotation)");
  if (h_err[0])
    return fail(RABITQ_EOVERFLOW,
                "a query's candidate list exceeded the fixed scratch's capacity");
  return RABITQ_OK;
}


// Search through the bucket-major tensor-core scan (two passes), then the
// per-query end. Same results as search_dev.
int search_dev_tc(const SearchArgs& a, cudaStream_t s) {
  const rabitq_index* X = a.X;
  const int K = X->K, d = X->d, dpad = X->dpad, W = X->W;
  const int nprobe = std::min(a.nprobe, K);
  if (a.nq == 0) return RABITQ_OK;
  int dev = 0, sms = 0;
  RBQ_CUDA(cudaGetDevice(&dev));
  RBQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int cap = a.cand_cap;  // per-query list capacity
  const int pilot_m = 4 * a.k;
  const int ce = pow2_at_least(pilot_m);
  const int ct = std::max(1024, pow2_at_least(a.k + kThreads));
  // passes over probe ranks [0, b1), [b1, b2), [b2, nprobe); tau' is
  // tightened and the lists compacted after each of the first two
  const int b1 = std::min(nprobe, 2), b2 = std::min(nprobe, 8);
  // query chunks: lists <= 4 GiB, centroid distances <= 1 GiB
  int64_t qchunk = std::min<int64_t>(a.nq, (int64_t(1) << 28) / K);
  qchunk = std::max<int64_t>(1, std::min<int64_t>(qchunk, (int64_t(1) << 32) / ((int64_t)cap * 16)));
  const int64_t np = qchunk * nprobe;
  DevBuf cd, rq, pid, pdist, keys, pperm, poff, qub, pmeta, psum, tiles, toffA, lists, lcnt, qtau,
      err, qn, pnq2;
  if (metric_cos(X)) RBQ_CHECK(qn.alloc(sizeof(float) * qchunk * d, s));
  if (metric_ip(X)) RBQ_CHECK(pnq2.alloc(sizeof(float) * np, s));
  RBQ_CHECK(cd.alloc(sizeof(float) * probe_scratch_floats(X, qchunk), s));
  RBQ_CHECK(rq.alloc(sizeof(float) * qchunk * dpad, s));
  RBQ_CHECK(pid.alloc(sizeof(int32_t) * np, s));
  RBQ_CHECK(pdist.alloc(sizeof(float) * np, s));
  RBQ_CHECK(keys.alloc(sizeof(int32_t) * np, s));
  RBQ_CHECK(pperm.alloc(sizeof(int32_t) * np, s));
  RBQ_CHECK(poff.alloc(sizeof(int32_t) * (3 * K + 5), s));
  RBQ_CHECK(qub.alloc(sizeof(__nv_bfloat16) * np * dpad, s));
  RBQ_CHECK(pmeta.alloc(sizeof(float4) * np, s));
  RBQ_CHECK(psum.alloc(sizeof(int32_t) * np, s));
  RBQ_CHECK(tiles.alloc(sizeof(int32_t) * (K + 1), s));
  RBQ_CHECK(toffA.alloc(sizeof(int32_t) * 3 * (K + 1), s));
  RBQ_CHECK(lists.alloc(sizeof(int4) * qchunk * cap, s));
  RBQ_CHECK(lcnt.alloc(sizeof(int32_t) * qchunk, s));
  RBQ_CHECK(qtau.alloc(sizeof(float) * qchunk, s));
  RBQ_CHECK(err.alloc(sizeof(int), s));
  DevBuf fid, fdist;  // learned probe counts: the 64 nearest buckets per query
  if (a.pred) {
    RBQ_CHECK(fid.alloc(sizeof(int32_t) * qchunk * kMlpIn, s));
    RBQ_CHECK(fdist.alloc(sizeof(float) * qchunk * kMlpIn, s));
  }
  RBQ_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  RBQ_CUDA(cudaMemsetAsync(tiles.p, 0, sizeof(int32_t) * (K + 1), s));

  const size_t scan_smem = 64 * 1024;  // 32 KB of operands; caps residency at 3 CTAs/SM
  RBQ_CUDA(cudaFuncSetAttribute(tc_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)scan_smem));
  const size_t tail_smem = fused_smem_bytes(1, a.bq, W, d, 32, ce, ct, kThreads / 32, nullptr);
  RBQ_CUDA(cudaFuncSetAttribute(tc_tail_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tail_smem));
  int tail_per_sm = 1;
  RBQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&tail_per_sm, tc_tail_kernel, kThreads,
                                                         tail_smem));
  tail_per_sm = std::max(tail_per_sm, 1);
  cudaEvent_t ev[5] = {};
  const bool timing = a.stage_ms != nullptr;
  float acc_ms[4] = {0, 0, 0, 0};
  if (timing)
    for (auto& e : ev) RBQ_CUDA(cudaEventCreate(&e));
  for (int64_t q0 = 0; q0 < a.nq; q0 += qchunk) {
    const int64_t nqc = std::min(qchunk, a.nq - q0);
    const int64_t npc = nqc * nprobe;
    if (timing) RBQ_CUDA(cudaEventRecord(ev[0], s));
    const float* Q = nullptr;
    RBQ_CHECK(search_queries(X, a.queries + q0 * d, nqc, qn.as<float>(), &Q, s));
    RBQ_CHECK(centroid_scores(X, Q, nqc, cd.as<float>(), err.as<int>(), s));
    int32_t* probe_ids = a.trace && a.trace->probe_ids ? a.trace->probe_ids + q0 * nprobe
                                                       : pid.as<int32_t>();
    float* probe_dist = a.trace && a.trace->probe_dist ? a.trace->probe_dist + q0 * nprobe
                                                       : pdist.as<float>();
    if (timing) RBQ_CUDA(cudaEventRecord(ev[1], s));
    const int32_t* npq = a.per_query_nprobe ? a.per_query_nprobe + q0 : nullptr;
    if (a.pred) {
      RBQ_CHECK(predict_chunk(a, Q, cd.as<float>(), nqc, q0, fid.as<int32_t>(),
                              fdist.as<float>(), s));
      npq = a.pred_nprobe + q0;
    }
    RBQ_CHECK(probe_select(X, Q, nqc, cd.as<float>(), nprobe, npq, probe_ids, probe_dist, s,
                           a.pred ? fid.as<int32_t>() : nullptr, fdist.as<float>(),
                           std::min(kMlpIn, K)));
    if (metric_ip(X)) RBQ_CHECK(probe_nq2(X, Q, nqc, nprobe, probe_ids, pnq2.as<float>(), s));
    if (timing) RBQ_CUDA(cudaEventRecord(ev[2], s));
    float* rqp = a.trace && a.trace->rq ? a.trace->rq + q0 * dpad : rq.as<float>();
    if (a.rot_precision == RABITQ_ROT_FP32)
      RBQ_CHECK(gemm_canon(kDot, Q, d, nullptr, nullptr, 0, nullptr, X->P32, dpad, rqp, dpad, nqc,
                           dpad, d, s));
    else
      RBQ_CHECK(rotate_tc(X, Q, nqc, a.rot_precision, rqp, err.as<int>(), s));
    if (timing) RBQ_CUDA(cudaEventRecord(ev[3], s));
    // pairs by (pass, bucket)
    pair_keys_kernel<<<(unsigned)((npc + 255) / 256), 256, 0, s>>>(probe_ids, npc, nprobe, b1, b2,
                                                                   K, keys.as<int32_t>());
    RBQ_CHECK(counting_sort(keys.as<int32_t>(), npc, 3 * K + 4, pperm.as<int32_t>(),
                            poff.as<int32_t>(), s));
    quantize_pairs_kernel<<<(unsigned)((npc * 32 + 255) / 256), 256, 0, s>>>(
        rqp, probe_ids, probe_dist, metric_ip(X) ? pnq2.as<float>() : nullptr, X->ptc, npc,
        nprobe, dpad, a.bq, a.eps0, a.seed, q0,
        qub.as<__nv_bfloat16>(), pmeta.as<float4>(), psum.as<int32_t>());
    RBQ_CUDA(cudaGetLastError());
    for (int pass = 0; pass < 3; ++pass) {
      tile_count_kernel<<<(K + 255) / 256, 256, 0, s>>>(X->bucket_off, poff.as<int32_t>(),
                                                        pass * (K + 1), K, tiles.as<int32_t>());
      RBQ_CHECK(exclusive_scan_i32(tiles.as<int32_t>(), toffA.as<int32_t>() + pass * (K + 1),
                                   K + 1, s));
    }
    RBQ_CUDA(cudaMemsetAsync(lcnt.p, 0, sizeof(int32_t) * nqc, s));
    fill_f32_kernel<<<(unsigned)((nqc + 255) / 256), 256, 0, s>>>(qtau.as<float>(), nqc,
                                                                  HUGE_VALF);
    TcScanParams T;
    T.codes = X->codes;
    T.factors = X->factors;
    T.bucket_off = X->bucket_off;
    T.W = W;
    T.dpad = dpad;
    T.K = K;
    T.nprobe = nprobe;
    T.pair_perm = pperm.as<int32_t>();
    T.pair_off = poff.as<int32_t>();
    T.qub = qub.as<__nv_bfloat16>();
    T.pmeta = pmeta.as<float4>();
    T.psum = psum.as<int32_t>();
    T.qtau = qtau.as<float>();
    T.lists = lists.as<int4>();
    T.lcnt = lcnt.as<int32_t>();
    T.cap = cap;
    T.err = err.as<int>();
    for (int pass = 0; pass < 3; ++pass) {
      T.key_base = pass * (K + 1);
      T.tile_off = toffA.as<int32_t>() + pass * (K + 1);
      tc_scan_kernel<<<(unsigned)(2 * sms), kTsThreads, scan_smem, s>>>(T);
      RBQ_CUDA(cudaGetLastError());
      if (pass < 2) {
        list_threshold_kernel<<<(unsigned)std::min<int64_t>(nqc, 4 * sms), kThreads, 0, s>>>(
            lists.as<int4>(), lcnt.as<int32_t>(), cap, nqc, a.k, qtau.as<float>());
        RBQ_CUDA(cudaGetLastError());
      }
    }
    FusedParams P;
    std::memset(&P, 0, sizeof P);
    P.queries = Q;
    P.probe_ids = probe_ids;
    P.nprobe_q = npq;
    P.metric = metric_ip(X);
    P.data_b = X->data_b;
    P.perm = X->perm;
    P.inv_perm = X->inv_perm;
    P.bucket_off = X->bucket_off;
    P.nq = nqc;
    P.q_offset = q0;
    P.d = d;
    P.dpad = dpad;
    P.W = W;
    P.bq = a.bq;
    P.k = a.k;
    P.m = pilot_m;
    P.nprobe = nprobe;
    P.pch = 1;
    P.cu = 32;
    P.ce = ce;
    P.ct = ct;
    P.out_ids = a.out_ids + q0 * a.k;
    P.out_dist = a.out_dist + q0 * a.k;
    P.err = err.as<int>();
    if (a.trace) {
      const rabitq_trace& Tr = *a.trace;
      if (Tr.n_pairs) P.tr.n_pairs = Tr.n_pairs + q0;
      if (Tr.tau_ub) P.tr.tau_ub = Tr.tau_ub + q0;
      if (Tr.tau1) P.tr.tau1 = Tr.tau1 + q0;
      if (Tr.tau) P.tr.tau = Tr.tau + q0;
      if (Tr.n_surv) P.tr.n_surv = Tr.n_surv + q0;
      if (Tr.surv_ids) {
        P.tr.surv_ids = Tr.surv_ids + q0 * Tr.surv_cap;
        P.tr.surv_cap = Tr.surv_cap;
      }
    }
    tc_tail_kernel<<<(unsigned)std::min<int64_t>(nqc, (int64_t)sms * tail_per_sm), kThreads,
                     tail_smem, s>>>(P, lists.as<int4>(), lcnt.as<int32_t>(), cap);
    RBQ_CUDA(cudaGetLastError());
    if (timing) {
      RBQ_CUDA(cudaEventRecord(ev[4], s));
      RBQ_CUDA(cudaEventSynchronize(ev[4]));
      for (int i = 0; i < 4; ++i) {
        float t = 0;
        RBQ_CUDA(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
        acc_ms[i] += t;
      }
    }
  }
  if (timing) {
    for (int i = 0; i < 4; ++i) a.stage_ms[i] = acc_ms[i];
    for (auto& e : ev) cudaEventDestroy(e);
  }
  int h_err = 0;
  RBQ_CUDA(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaStreamSynchronize(s));
  if (h_err == 2) return fail(RABITQ_ETIMEOUT, "a tensor-core wait expired in the scan");
  if (h_err)
    return fail(RABITQ_EOVERFLOW,
                "a query's candidate list exceeded max_candidates; raise max_candidates");
  return RABITQ_OK;
}

// Top-nsel buckets of each query, ascending (distance, id): the canonical
// query-centroid distances of the IVF probe (§4), then the block select.
int select_buckets(const rabitq_index* X, const float* Q, int64_t nq, int nsel, int32_t* ids,
                   float* dist, cudaStream_t s) {
  if (nq <= 0) return RABITQ_OK;
  const int K = X->K, d = X->d;
  nsel = std::min(nsel, K);
  const int64_t qchunk = std::max<int64_t>(1, std::min<int64_t>(nq, (int64_t(1) << 28) / K));
  DevBuf cd;
  RBQ_CHECK(cd.alloc(sizeof(float) * probe_scratch_floats(X, qchunk), s));
  DevBuf err;
  RBQ_CHECK(err.alloc(sizeof(int), s));
  RBQ_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  for (int64_t q0 = 0; q0 < nq; q0 += qchunk) {
    const int64_t m = std::min(qchunk, nq - q0);
    RBQ_CHECK(probe_keys_tc(X, Q + q0 * d, m, cd.as<float>(), err.as<int>(), s));
    RBQ_CHECK(probe_select(X, Q + q0 * d, m, cd.as<float>(), nsel, nullptr, ids + q0 * nsel,
                           dist + q0 * nsel, s));
  }
  int h_err = 0;
  RBQ_CUDA(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaStreamSynchronize(s));
  if (h_err) return fail(RABITQ_ETIMEOUT, "a tensor-core wait expired in the probe scores");
  return RABITQ_OK;
}

// Learned probe counts (and optionally features and network outputs).
int predict_dev(const rabitq_index* X, const rabitq_predictor* pr, const float* Q, int64_t nq,
                int32_t* nprobe_out, float* feat, float* y, cudaStream_t s) {
  if (nq <= 0) return RABITQ_OK;
  const int navail = std::min(kMlpIn, X->K);
  const int64_t chunk = std::min<int64_t>(nq, int64_t(1) << 20);
  DevBuf ids, dist;
  RBQ_CHECK(ids.alloc(sizeof(int32_t) * chunk * navail, s));
  RBQ_CHECK(dist.alloc(sizeof(float) * chunk * navail, s));
  for (int64_t q0 = 0; q0 < nq; q0 += chunk) {
    const int64_t m = std::min(chunk, nq - q0);
    RBQ_CHECK(select_buckets(X, Q + q0 * X->d, m, navail, ids.as<int32_t>(), dist.as<float>(), s));
    RBQ_CHECK(mlp_infer(pr, dist.as<float>(), navail, m, navail, nprobe_out + q0,
                        feat ? feat + q0 * kMlpIn : nullptr, y ? y + q0 : nullptr, s));
  }
  return RABITQ_OK;
}

// Single-code estimates of nq queries against ids (nq x m) into out
// (nq x m x 3), in query chunks that bound the rotated-query scratch. The
// error flag (device int, zeroed by the caller) is set for an id outside
// [-1, n).
int estimate_dev(const rabitq_index* X, const float* Q, int64_t nq, const int64_t* ids, int m,
                 int bq, float eps0, uint64_t seed, int rot_precision, float* out, int* err,
                 cudaStream_t s) {
  if (nq <= 0 || m <= 0) return RABITQ_OK;
  const int d = X->d, dpad = X->dpad;
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(nq, (int64_t(1) << 26) / dpad));
  DevBuf rq, qn;
  RBQ_CHECK(rq.alloc(sizeof(float) * chunk * dpad, s));
  if (metric_cos(X)) RBQ_CHECK(qn.alloc(sizeof(float) * chunk * d, s));
  for (int64_t q0 = 0; q0 < nq; q0 += chunk) {
    const int64_t nqc = std::min(chunk, nq - q0);
    const float* Qc = nullptr;
    RBQ_CHECK(search_queries(X, Q + q0 * d, nqc, qn.as<float>(), &Qc, s));
    if (rot_precision == RABITQ_ROT_FP32)
      RBQ_CHECK(gemm_canon(kDot, Qc, d, nullptr, nullptr, 0, nullptr, X->P32, dpad, rq.as<float>(),
                           dpad, nqc, dpad, d, s));
    else
      RBQ_CHECK(rotate_tc(X, Qc, nqc, rot_precision, rq.as<float>(), err, s));
    EstParams E;
    E.queries = Qc;
    E.rq = rq.as<float>();
    E.ids = ids + q0 * m;
    E.inv_perm = X->inv_perm;
    E.assign = X->assign;
    E.codes = X->codes;
    E.factors = X->factors;
    E.centroids = X->centroids;
    E.ptc = X->ptc;
    E.nq = nqc;
    E.n = X->n;
    E.m = m;
    E.d = d;
    E.dpad = dpad;
    E.bq = bq;
    E.metric = metric_ip(X);
    E.eps0 = eps0;
    E.seed = seed;
    E.out = out + q0 * m * 3;
    E.err = err;
    E.q_offset = q0;  // the quantization stream is the query's index in the call
    const int64_t warps = nqc * m;
    estimate_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(E);
    RBQ_CUDA(cudaGetLastError());
  }
  return RABITQ_OK;
}

}  // namespace rbq
