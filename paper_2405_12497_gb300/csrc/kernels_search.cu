// kernels_search.cu -- query phase (Alg. 2 of the paper with the IVF probing
// and error-bound re-ranking of §4).
//
// Stages per batch of queries:
//   1. canonical squared distances to every centroid (kernels_gemm.cu);
//   2. probe selection: the nprobe nearest centroids by (distance, id);
//   3. query rotation P^{-1}[q_r; 0] (kernels_gemm.cu, FP32 canonical);
//   4. one persistent fused kernel, a CTA per query at a time: randomized
//      B_q-bit quantization of q' per probed cluster (§3.3.1), bucket scan
//      with the bit-plane popcount form of <x_b, q_u> (§3.3.2), the unbiased
//      estimator and its error bound (Theorem 3.2), the k-th smallest upper
//      bound tau, the survivors LB <= tau, their exact distances and the
//      top-k by (distance, id).
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace rbq {
namespace {

constexpr int kThreads = 256;

// ------------------------------------------------------------ selection
// Top-nsel of a row of K non-negative distances by (distance, id): radix
// select of the nsel-th smallest key, collection of everything below it plus
// the lowest ids among its ties, then a bitonic sort of the selection.
__global__ void __launch_bounds__(kThreads) select_kernel(
    const float* __restrict__ CD, int K, int nprobe, const int32_t* __restrict__ nprobe_q,
    int sort_n, int32_t* __restrict__ out_ids, float* __restrict__ out_dist) {
  extern __shared__ unsigned long long sel[];  // sort_n entries
  __shared__ int hist[256];
  __shared__ uint32_t s_prefix, s_mask;
  __shared__ int s_remaining, s_less, s_tie_base;
  const int q = blockIdx.x;
  const float* row = CD + (int64_t)q * K;
  int nsel = nprobe;
  if (nprobe_q) nsel = min(max(nprobe_q[q], 1), nprobe);
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
      const uint32_t key = float_key(row[c]);
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
    const uint32_t key = float_key(row[c]);
    if (key < T) sel[atomicAdd(&s_less, 1)] = ((unsigned long long)key << 32) | (uint32_t)c;
  }
  __syncthreads();
  // ties in ascending id order, chunk by chunk
  __shared__ int warp_cnt[kThreads / 32];
  for (int c0 = 0; c0 < K; c0 += blockDim.x) {
    if (s_tie_base >= need_ties) break;
    const int c = c0 + threadIdx.x;
    const bool tie = (c < K) && float_key(row[c]) == T;
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
    out_ids[(int64_t)q * nprobe + j] = ok ? (int32_t)(sel[j] & 0xffffffffu) : -1;
    out_dist[(int64_t)q * nprobe + j] = ok ? key_float((uint32_t)(sel[j] >> 32))
                                           : __int_as_float(0x7f800000);
  }
}

// ------------------------------------------------------ fused query kernel
// Shared state of the block radix select.
struct SelState {
  int hist[256];
  int bin, rem, tie_taken;
  int warp_cnt[kThreads / 32];
};

struct FusedParams {
  const float* queries;     // nq x d
  const float* rq;          // nq x dpad
  const int32_t* probe_ids; // nq x nprobe
  const float* probe_dist;  // nq x nprobe
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
  int4* cand;               // gridDim.x x cand_cap: {pos, LB, estimate, -}
  int64_t* out_ids;
  float* out_dist;
  int* err;
  rabitq_trace tr;
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
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline size_t fused_smem_bytes(int pch, int bq, int W, int d, int cu, int ce,
                                                   int ct, int nwarps,
                                                   size_t* off /* 9 entries or null */) {
  size_t o = 0, offs[9];
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
  if (off)
    for (int i = 0; i < 9; ++i) off[i] = offs[i];
  return o;
}

// Quantize q' for one probed cluster with one warp (§3.3.1). Lane l holds
// elements k = 128 i + 4 l + r (r = 0..3), so the four u_k of one Philox call
// (counter k/4) belong to one lane.
__device__ __forceinline__ void quantize_probe(const FusedParams& P, const FusedSmem& S, int64_t q,
                                               int j, int jg, int c, float nq2) {
  const int lane = threadIdx.x & 31;
  const int dpad = P.dpad, W = P.W, bq = P.bq;
  const int nblk = (dpad + 127) >> 7;
  const float* rq = P.rq + q * dpad;
  const float* pc = P.ptc + (int64_t)c * dpad;
  // pass 1: v_l = min qd, v_r = max qd with qd = rq - P^T c
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
  const uint64_t gq = (uint64_t)(P.q_offset + q);
  int sum = 0;
  uint64_t* planes = S.planes + (size_t)j * bq * W;
  for (int i = 0; i < nblk; ++i) {
    const int k0 = 128 * i + 4 * lane;
    int qu[4] = {0, 0, 0, 0};
    if (delta > 0.0f && k0 < dpad) {
      float qd[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) qd[r] = (k0 + r < dpad) ? __fsub_rn(rq[k0 + r], pc[k0 + r]) : 0.0f;
      const U4 w = philox4x32_10(P.seed, (uint32_t)(k0 >> 2), (uint32_t)gq, (uint32_t)c, kTagQuant);
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
    // bit-planes: the nibble of lane l sits at bits 4l..4l+3 of the 128-bit block
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
  }
  sum = warp_sum_i(sum);
  if (lane == 0) {
    const float sqd = __fsqrt_rn((float)dpad);
    const float keps = __fdiv_rn(__fmul_rn(2.0f, P.eps0), __fsqrt_rn((float)(dpad - 1)));
    const float n_q = __fsqrt_rn(nq2);
    const float4 m = make_float4(__fdiv_rn(delta, sqd), __fdiv_rn(vl, sqd), __fmul_rn(n_q, keps),
                                 nq2);
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
  const int tid = threadIdx.x, lane = tid & 31;
  K prefix = 0, mask = 0;
  int rem = want;
  for (int shift = NB - 8; shift >= 0; shift -= 8) {
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

// Sort a shared key buffer (padded with the maximum key), keep the `keep`
// smallest; returns the count kept. Whole block; synchronized on return.
__device__ __forceinline__ void sort_keep_u64(unsigned long long* a, int cap, int* cnt, int keep) {
  for (int i = *cnt + threadIdx.x; i < cap; i += blockDim.x) a[i] = ~0ull;
  __syncthreads();
  block_bitonic_sort_u64(a, cap);
  if (threadIdx.x == 0 && *cnt > keep) *cnt = keep;
  __syncthreads();
}

// In-place, order-keeping compaction of the candidate list with predicate f.
template <class F>
__device__ __forceinline__ void compact_cand(int4* cand, int* cnt, int cap, int* scratch, F keep_f) {
  const int n = min(*cnt, cap);
  int out = 0;
  __syncthreads();
  for (int b = 0; b < n; b += blockDim.x) {
    const int i = b + threadIdx.x;
    int4 e = make_int4(0, 0, 0, 0);
    bool keep = false;
    if (i < n) {
      e = cand[i];
      keep = keep_f(e);
    }
    const unsigned bal = __ballot_sync(kFull, keep);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) scratch[wid] = __popc(bal);
    __syncthreads();
    int before = out, tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      if (w < wid) before += scratch[w];
      tot += scratch[w];
    }
    if (keep) cand[before + __popc(bal & ((1u << lane) - 1u))] = e;
    out += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *cnt = out;
  __syncthreads();
}

// Exact squared distances of a list of rows: each lane streams its own row
// with 16-byte loads (eight in flight per lane, a warp has 256 rows' worth of
// loads outstanding) and folds it in ascending dimension order (canonical
// squared distance). Keys (distance, id) go to the top-k buffer.
// SRC 0: the pilot (ids in S.estk); SRC 1: the candidate list (positions).
template <int SRC>
__device__ void rerank_rows(const FusedParams& P, const FusedSmem& S, int64_t q, int count,
                            const int4* cand, int* top_cnt, int* surv_cnt) {
  const int d = P.d;
  const bool vec = (d & 3) == 0;
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
        pos = cand[i].x;
        id = P.perm[pos];
      }
    }
    float acc = 0.0f;
    if (valid) {
      const float* x = P.data_b + (int64_t)pos * d;
      if (vec) {
        const float4* x4 = reinterpret_cast<const float4*>(x);
        const float4* q4 = reinterpret_cast<const float4*>(S.qv);
        int c = 0;
        for (; c + 8 <= (d >> 2); c += 8) {
          float4 v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) v[u] = __ldg(x4 + c + u);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const float4 qq = q4[c + u];
            float t = __fsub_rn(qq.x, v[u].x); acc = __fmaf_rn(t, t, acc);
            t = __fsub_rn(qq.y, v[u].y); acc = __fmaf_rn(t, t, acc);
            t = __fsub_rn(qq.z, v[u].z); acc = __fmaf_rn(t, t, acc);
            t = __fsub_rn(qq.w, v[u].w); acc = __fmaf_rn(t, t, acc);
          }
        }
        for (; c < (d >> 2); ++c) {
          const float4 vv = __ldg(x4 + c), qq = q4[c];
          float t = __fsub_rn(qq.x, vv.x); acc = __fmaf_rn(t, t, acc);
          t = __fsub_rn(qq.y, vv.y); acc = __fmaf_rn(t, t, acc);
          t = __fsub_rn(qq.z, vv.z); acc = __fmaf_rn(t, t, acc);
          t = __fsub_rn(qq.w, vv.w); acc = __fmaf_rn(t, t, acc);
        }
      } else {
        for (int dd = 0; dd < d; ++dd) {
          const float t = __fsub_rn(S.qv[dd], __ldg(x + dd));
          acc = __fmaf_rn(t, t, acc);
        }
      }
    }
    const int slot = warp_reserve(valid, top_cnt);
    if (valid) {
      S.topk[slot] = ((unsigned long long)float_key(acc) << 32) | (uint32_t)id;
      const int si = i + (SRC == 0 ? 0 : *surv_cnt);
      if (P.tr.surv_ids && si < P.tr.surv_cap) P.tr.surv_ids[q * P.tr.surv_cap + si] = id;
    }
    __syncthreads();
    if (*top_cnt > P.ct - (int)blockDim.x) select_keep<unsigned long long>(S.topk, top_cnt, P.k, *S.sel);
  }
  __syncthreads();
  if (threadIdx.x == 0) *surv_cnt += count;
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
  if constexpr (WT > 0) {
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

constexpr int kPPT = 4;  // most pairs per thread per scan round (buffer sizing)

// Pairs per thread per round: as many as the code registers allow.
template <int WT>
__host__ __device__ constexpr int pairs_per_thread() {
  return WT == 0 ? 2 : (WT <= 4 ? 4 : (WT <= 8 ? 2 : 1));
}

template <int WT, int BQT>
__global__ void __launch_bounds__(kThreads, 2) fused_search_kernel(FusedParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_ub_cnt, s_cand_cnt, s_top_cnt, s_surv, s_overflow;
  __shared__ float s_tau;
  __shared__ int s_scratch[kThreads / 32];
  __shared__ SelState s_sel;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarps = blockDim.x >> 5;
  size_t off[9];
  fused_smem_bytes(P.pch, P.bq, P.W, P.d, P.cu, P.ce, P.ct, nwarps, off);
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
  const int W = P.W, bq = P.bq, k = P.k, m = P.m;
  int4* cand = P.cand + (int64_t)blockIdx.x * P.cand_cap;

  for (int64_t q = blockIdx.x; q < P.nq; q += gridDim.x) {
    int np = P.nprobe;
    if (P.nprobe_q) np = min(max(P.nprobe_q[q], 1), P.nprobe);
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
    for (int pc0 = 0; pc0 < np; pc0 += P.pch) {
      const int npc = min(P.pch, np - pc0);
      for (int j = wid; j < npc; j += nwarps) {
        const int jg = pc0 + j;
        const int c = P.probe_ids[q * P.nprobe + jg];
        quantize_probe(P, S, q, j, jg, c, P.probe_dist[q * P.nprobe + jg]);
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
      constexpr int PPT = pairs_per_thread<WT>();
      const int step = PPT * blockDim.x;
      for (int base = 0; base < total; base += step) {
        // issue every load of this thread's PPT pairs first (they are
        // independent), then evaluate; keeps PPT code/factor loads in flight
        int64_t posv[PPT];
        int jv[PPT];
        CodeRegs<WT> cr[PPT];
        float4 fv[PPT];
#pragma unroll
        for (int pp = 0; pp < PPT; ++pp) {
          const int t = base + pp * blockDim.x + tid;
          posv[pp] = -1;
          jv[pp] = 0;
          if (t < total) {
            while (S.pref[j + 1] <= t) ++j;
            posv[pp] = (int64_t)S.pbeg[j] + (t - S.pref[j]);
            jv[pp] = j;
            load_code<WT>(cr[pp], P.codes + posv[pp] * W);
            fv[pp] = __ldg(P.factors + posv[pp]);
          }
        }
        // evaluate the estimator and its bounds for every pair of the round
        float distv[PPT], lbv[PPT], ubv[PPT];
        int ipv[PPT];
        const float tau = s_tau;
#pragma unroll
        for (int pp = 0; pp < PPT; ++pp) {
          distv[pp] = 0.0f;
          lbv[pp] = __int_as_float(0x7f800000);
          ubv[pp] = __int_as_float(0x7f800000);
          ipv[pp] = 0;
          if (posv[pp] >= 0) {
            const int jj = jv[pp];
            const int ip = code_ip<WT, BQT>(cr[pp], P.codes + posv[pp] * W,
                                            S.planes + (size_t)jj * bq * W, W, bq);
            const float4 f = fv[pp];
            const float4 mt = S.pmeta[jj];
            // estimator (§3.3.2 + Theorem 3.2) and its bound, fixed FP32 order
            const float t1 = (float)(2 * ip - S.psum[jj]);
            const float xq = __fadd_rn(__fmul_rn(mt.x, t1), __fmul_rn(mt.y, f.w));
            const float dist = __fsub_rn(__fadd_rn(f.x, mt.w), __fmul_rn(f.y, xq));
            const float e = __fmul_rn(f.z, mt.z);
            distv[pp] = dist;
            lbv[pp] = __fsub_rn(dist, e);
            ubv[pp] = __fadd_rn(dist, e);
            ipv[pp] = ip;
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
                                   __float_as_int(distv[pp]), 0);
            else
              s_overflow = 1;
            ++bc;
          }
          if (P.tr.pair_id) {
            const int64_t tt = pairs_done + base + pp * blockDim.x + tid;
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
        __syncthreads();
        if (s_ub_cnt > P.cu - step) {  // keep the k smallest upper bounds
          const uint32_t T = select_keep<uint32_t>(S.ubk, &s_ub_cnt, k, *S.sel);
          if (tid == 0) s_tau = key_float(T);
          __syncthreads();
        }
        if (s_cand_cnt > P.cand_cap - step) {
          const float tau = s_tau;
          compact_cand(cand, &s_cand_cnt, P.cand_cap, s_scratch,
                       [tau](const int4& e) { return __int_as_float(e.y) <= tau; });
          if (s_cand_cnt > P.cand_cap - step && tid == 0) s_overflow = 1;
          __syncthreads();
        }
        if (s_overflow) break;
      }
      pairs_done += total;
      __syncthreads();
      if (s_overflow) break;
    }
    // tau_ub: k-th smallest upper bound; pilot: the m smallest estimates
    const int n_ub = s_ub_cnt;
    const uint32_t T_ub = (n_ub >= k) ? block_select<uint32_t>(S.ubk, n_ub, k, *S.sel) : 0u;
    const float tau_ub = (n_ub >= k) ? key_float(T_ub) : __int_as_float(0x7f800000);
    // the candidate list (LB <= running tau') shrinks to LB <= tau_ub
    compact_cand(cand, &s_cand_cnt, P.cand_cap, s_scratch,
                 [tau_ub](const int4& e) { return __int_as_float(e.y) <= tau_ub; });
    // pilot: the m smallest (estimate, id) of the list
    const int nl = s_cand_cnt;
    const bool pilot_all = nl <= m;
    uint32_t T_e = 0xffffffffu, T_id = 0xffffffffu;
    if (!pilot_all) {
      T_e = block_select_f<uint32_t>(nl, m, *S.sel,
                                     [cand](int i) { return float_key(__int_as_float(cand[i].z)); });
      const int ties = S.sel->rem;
      // among the list entries whose estimate equals the m-th one, the
      // `ties` smallest ids belong to the pilot
      T_id = block_select_f<uint32_t>(nl, ties, *S.sel, [cand, T_e, &P](int i) {
        const int4 e = cand[i];
        return float_key(__int_as_float(e.z)) == T_e ? (uint32_t)__ldg(P.perm + e.x) : 0xffffffffu;
      });
    }
    // write the pilot's (id, position) pairs to the pilot list
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
        in = pilot_all || ek < T_e ||
             (ek == T_e && (uint32_t)__ldg(P.perm + e.x) <= T_id);
      }
      const int slot = warp_reserve(in, &s_pilot);
      if (in) {
        S.estk[slot] = ((unsigned long long)(uint32_t)__ldg(P.perm + e.x) << 32) | (uint32_t)e.x;
        cand[i].w = 1;
      }
    }
    __syncthreads();
    const int pilot = s_pilot;
    // exact distances of the pilot; tau1 = k-th smallest of them
    rerank_rows<0>(P, S, q, pilot, cand, &s_top_cnt, &s_surv);
    const unsigned long long T1 =
        (pilot >= k) ? block_select<unsigned long long>(S.topk, s_top_cnt, k, *S.sel) : 0ull;
    const float tau1 = (pilot >= k) ? key_float((uint32_t)(T1 >> 32)) : __int_as_float(0x7f800000);
    const float tau = fminf(tau_ub, tau1);
    // the rest of the re-rank set: LB <= tau, outside the pilot
    compact_cand(cand, &s_cand_cnt, P.cand_cap, s_scratch, [tau](const int4& e) {
      return e.w == 0 && __int_as_float(e.y) <= tau;
    });
    rerank_rows<1>(P, S, q, s_cand_cnt, cand, &s_top_cnt, &s_surv);
    sort_keep_u64(S.topk, P.ct, &s_top_cnt, k);
    const int got = min(s_top_cnt, k);
    for (int j2 = tid; j2 < k; j2 += blockDim.x) {
      const bool ok = j2 < got;
      P.out_ids[q * k + j2] = ok ? (int64_t)(S.topk[j2] & 0xffffffffu) : -1;
      P.out_dist[q * k + j2] =
          ok ? key_float((uint32_t)(S.topk[j2] >> 32)) : __int_as_float(0x7f800000);
    }
    if (tid == 0) {
      if (s_overflow) atomicExch(P.err, 1);
      if (P.tr.n_pairs) P.tr.n_pairs[q] = pairs_done;
      if (P.tr.tau_ub) P.tr.tau_ub[q] = tau_ub;
      if (P.tr.tau1) P.tr.tau1[q] = tau1;
      if (P.tr.tau) P.tr.tau[q] = tau;
      if (P.tr.n_surv) P.tr.n_surv[q] = s_surv;
    }
    __syncthreads();
  }
}

typedef void (*FusedFn)(FusedParams);

// Compile-time code lengths of the common shapes (D' = 128, 256, 1024 with
// B_q = 4); everything else runs the generic instance.
FusedFn pick_fused(int W, int bq) {
  if (bq == 4) {
    if (W == 2) return fused_search_kernel<2, 4>;
    if (W == 4) return fused_search_kernel<4, 4>;
    if (W == 16) return fused_search_kernel<16, 4>;
  }
  return fused_search_kernel<0, 0>;
}

int pow2_at_least(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace

int search_dev(const SearchArgs& a, cudaStream_t s) {
  const rabitq_index* X = a.X;
  const int K = X->K, d = X->d, dpad = X->dpad, W = X->W;
  const int nprobe = std::min(a.nprobe, K);
  if (a.nq == 0) return RABITQ_OK;
  int dev = 0, sms = 0;
  RBQ_CUDA(cudaGetDevice(&dev));
  RBQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

  // fused-kernel shape
  const int plane_bytes = a.bq * W * 8;
  int pch = std::max(1, std::min(nprobe, (32 * 1024) / plane_bytes));
  const int pilot_m = 4 * a.k;  // pilot size
  const int cu = std::max(1024, pow2_at_least(a.k + kPPT * kThreads));
  const int ce = pow2_at_least(pilot_m);  // the pilot list
  const int ct = std::max(512, pow2_at_least(a.k + kThreads));
  const size_t smem = fused_smem_bytes(pch, a.bq, W, d, cu, ce, ct, kThreads / 32, nullptr);
  const FusedFn fn = pick_fused(W, a.bq);
  RBQ_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  RBQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem));
  per_sm = std::max(per_sm, 1);

  // query chunks bound the centroid-distance scratch (<= 256 Mi floats)
  const int64_t qchunk = std::max<int64_t>(1, std::min<int64_t>(a.nq, (int64_t(1) << 28) / K));
  const int64_t grid = std::min<int64_t>(qchunk, (int64_t)sms * per_sm);
  DevBuf cd, rq, pid, pdist, cand, err;
  RBQ_CHECK(cd.alloc(sizeof(float) * qchunk * K, s));
  RBQ_CHECK(rq.alloc(sizeof(float) * qchunk * dpad, s));
  RBQ_CHECK(pid.alloc(sizeof(int32_t) * qchunk * nprobe, s));
  RBQ_CHECK(pdist.alloc(sizeof(float) * qchunk * nprobe, s));
  RBQ_CHECK(cand.alloc(sizeof(int4) * grid * a.cand_cap, s));
  RBQ_CHECK(err.alloc(sizeof(int), s));
  RBQ_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));

  cudaEvent_t ev[5] = {};
  const bool timing = a.stage_ms != nullptr;
  float acc_ms[4] = {0, 0, 0, 0};
  if (timing)
    for (auto& e : ev) RBQ_CUDA(cudaEventCreate(&e));

  const int sort_n = pow2_at_least(nprobe);
  const size_t sel_smem = sizeof(unsigned long long) * sort_n;
  RBQ_CUDA(cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sel_smem));
  for (int64_t q0 = 0; q0 < a.nq; q0 += qchunk) {
    const int64_t nqc = std::min(qchunk, a.nq - q0);
    const float* Q = a.queries + q0 * d;
    if (timing) RBQ_CUDA(cudaEventRecord(ev[0], s));
    RBQ_CHECK(gemm_canon(kSqDist, Q, d, nullptr, nullptr, 0, nullptr, X->centroids_t, K,
                         cd.as<float>(), K, nqc, K, d, s));
    if (timing) RBQ_CUDA(cudaEventRecord(ev[1], s));
    int32_t* probe_ids = a.trace && a.trace->probe_ids ? a.trace->probe_ids + q0 * nprobe
                                                       : pid.as<int32_t>();
    float* probe_dist = a.trace && a.trace->probe_dist ? a.trace->probe_dist + q0 * nprobe
                                                       : pdist.as<float>();
    select_kernel<<<(unsigned)nqc, kThreads, sel_smem, s>>>(
        cd.as<float>(), K, nprobe, a.per_query_nprobe ? a.per_query_nprobe + q0 : nullptr,
        sort_n, probe_ids, probe_dist);
    RBQ_CUDA(cudaGetLastError());
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
    P.nprobe_q = a.per_query_nprobe ? a.per_query_nprobe + q0 : nullptr;
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
    P.eps0 = a.eps0;
    P.seed = a.seed;
    P.cand_cap = a.cand_cap;
    P.cand = cand.as<int4>();
    P.out_ids = a.out_ids + q0 * a.k;
    P.out_dist = a.out_dist + q0 * a.k;
    P.err = err.as<int>();
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
    const unsigned g = (unsigned)std::min<int64_t>(nqc, grid);
    fn<<<g, kThreads, smem, s>>>(P);
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
  int h_err = 0;
  RBQ_CUDA(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaStreamSynchronize(s));
  if (timing) {
    for (int i = 0; i < 4; ++i) a.stage_ms[i] = acc_ms[i];
    for (auto& e : ev) cudaEventDestroy(e);
  }
  if (h_err == 2)
    return fail(RABITQ_ETIMEOUT, "a tensor-core wait expired in the query rotation");
  if (h_err)
    return fail(RABITQ_EOVERFLOW,
                "a query's candidate list exceeded max_candidates; raise max_candidates");
  return RABITQ_OK;
}

// The same pipeline as search_dev, with every scratch array carved out of a
// caller-provided device buffer instead of being allocated: query chunks are
// sized to what fits. Used by the entry point that must not allocate.
int search_dev_prealloc(const SearchArgs& a, unsigned char* scratch, size_t scratch_bytes,
                        cudaStream_t s) {
  const rabitq_index* X = a.X;
  const int K = X->K, d = X->d, dpad = X->dpad, W = X->W;
  const int nprobe = std::min(a.nprobe, K);
  if (a.nq == 0) return RABITQ_OK;
  int dev = 0, sms = 0;
  RBQ_CUDA(cudaGetDevice(&dev));
  RBQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int plane_bytes = a.bq * W * 8;
  const int pch = std::max(1, std::min(nprobe, (32 * 1024) / plane_bytes));
  const int pilot_m = 4 * a.k;
  const int cu = std::max(1024, pow2_at_least(a.k + kPPT * kThreads));
  const int ce = pow2_at_least(pilot_m);  // the pilot list
  const int ct = std::max(512, pow2_at_least(a.k + kThreads));
  const size_t smem = fused_smem_bytes(pch, a.bq, W, d, cu, ce, ct, kThreads / 32, nullptr);
  const FusedFn fn = pick_fused(W, a.bq);
  RBQ_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int sort_n = pow2_at_least(nprobe);
  const size_t sel_smem = sizeof(unsigned long long) * sort_n;
  RBQ_CUDA(cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sel_smem));
  // layout: [error flag | candidate lists (one CTA per SM) | per-chunk query arrays]
  const size_t A = 256;
  const int64_t grid = sms;
  size_t off = A;
  const size_t cand_room = scratch_bytes / 2 > off ? scratch_bytes / 2 - off : 0;
  int64_t cap = std::min<int64_t>(a.cand_cap, (int64_t)(cand_room / (sizeof(int4) * grid)));
  if (cap < 1024) return fail(RABITQ_EINVAL, "rabitq_search_noalloc: scratch too small");
  int4* cand = reinterpret_cast<int4*>(scratch + off);
  off = align_up(off + sizeof(int4) * grid * cap, A);
  const size_t per_q = sizeof(float) * K + sizeof(float) * dpad + sizeof(int32_t) * nprobe +
                       sizeof(float) * nprobe;
  const size_t room = scratch_bytes > off + 4 * A ? scratch_bytes - off - 4 * A : 0;
  const int64_t qchunk = std::min<int64_t>(a.nq, (int64_t)(room / per_q));
  if (qchunk < 1)
    return fail(RABITQ_EINVAL,
                "rabitq_search_noalloc: one query's distances to every centroid do not fit in "
                "the fixed scratch (K too large)");
  float* cd = reinterpret_cast<float*>(scratch + off);
  off = align_up(off + sizeof(float) * qchunk * K, A);
  float* rq = reinterpret_cast<float*>(scratch + off);
  off = align_up(off + sizeof(float) * qchunk * dpad, A);
  int32_t* pid = reinterpret_cast<int32_t*>(scratch + off);
  off = align_up(off + sizeof(int32_t) * qchunk * nprobe, A);
  float* pdist = reinterpret_cast<float*>(scratch + off);
  off = align_up(off + sizeof(float) * qchunk * nprobe, A);
  if (off > scratch_bytes) return fail(RABITQ_EINVAL, "rabitq_search_noalloc: layout overflow");
  int* err = reinterpret_cast<int*>(scratch);
  RBQ_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));  // the flag must start at zero
  for (int64_t q0 = 0; q0 < a.nq; q0 += qchunk) {
    const int64_t nqc = std::min(qchunk, a.nq - q0);
    const float* Q = a.queries + q0 * d;
    RBQ_CHECK(gemm_canon(kSqDist, Q, d, nullptr, nullptr, 0, nullptr, X->centroids_t, K, cd, K,
                         nqc, K, d, s));
    select_kernel<<<(unsigned)nqc, kThreads, sel_smem, s>>>(
        cd, K, nprobe, a.per_query_nprobe ? a.per_query_nprobe + q0 : nullptr, sort_n, pid,
        pdist);
    RBQ_CUDA(cudaGetLastError());
    RBQ_CHECK(gemm_canon(kDot, Q, d, nullptr, nullptr, 0, nullptr, X->P32, dpad, rq, dpad, nqc,
                         dpad, d, s));
    FusedParams P;
    std::memset(&P, 0, sizeof P);
    P.queries = Q;
    P.rq = rq;
    P.probe_ids = pid;
    P.probe_dist = pdist;
    P.nprobe_q = a.per_query_nprobe ? a.per_query_nprobe + q0 : nullptr;
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
    P.eps0 = a.eps0;
    P.seed = a.seed;
    P.cand_cap = (int)cap;
    P.cand = cand;
    P.out_ids = a.out_ids + q0 * a.k;
    P.out_dist = a.out_dist + q0 * a.k;
    P.err = err;
    fn<<<(unsigned)std::min<int64_t>(nqc, grid), kThreads, smem, s>>>(P);
    RBQ_CUDA(cudaGetLastError());
  }
  int h_err = 0;
  RBQ_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  RBQ_CUDA(cudaStreamSynchronize(s));
  if (h_err)
    return fail(RABITQ_EOVERFLOW,
                "a query's candidate list exceeded the fixed scratch's capacity");
  return RABITQ_OK;
}


}  // namespace rbq
