/*
 * rabitq_oracle.c -- plain, slow, scalar CPU oracle for the RaBitQ IVF query
 * path (Gao & Long, "RaBitQ: Quantizing High-Dimensional Vectors with a
 * Theoretical Error Bound for Approximate Nearest Neighbor Search", SIGMOD'24).
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs may load this file's library. It shares no
 * code, header or table with the CUDA library, and never reads anything the
 * CUDA library produced as an expected value.
 *
 * Every function follows the paper's steps in the paper's order; where the
 * paper is silent (summation order, tie breaks, the source of the random
 * numbers), the reading used here is stated at the function and in the
 * numerics contract of the design notes:
 *
 *   - canonical FP32 dot:      s = 0; for i ascending: s = fmaf(a_i, b_i, s)
 *   - canonical FP32 sq. dist: s = 0; for i ascending: t = a_i - b_i;
 *                              s = fmaf(t, t, s)
 *   - canonical FP64 dot:      the same with fma() in double.
 *   - ties: (value, id) lexicographic everywhere.
 *   - random numbers: Philox4x32-10 (Salmon et al., SC'11), keyed by the
 *     64-bit seed, counter words listed at each use.
 *
 * Compiled with -O2 -ffp-contract=off and without -ffast-math so that every
 * float operation written here is one IEEE-754 round-to-nearest operation.
 *
 * Parity status: every function is pinned by the tests in
 * tests/test_oracle_pins.py (the inner-product / cosine metric and the
 * single-code estimator in tests/test_oracle_ip_pins.py). k-means, whose
 * variant the paper does not fix, is pinned by Lloyd iterates worked out by
 * hand (ties to the lower centroid id, an empty cluster keeping its value,
 * the FP32 mean in id order) besides its invariants.
 *
 * Metrics: squared Euclidean distance (the paper's setting) and the inner
 * product of the paper's closing footnote (§6), which also gives the cosine
 * similarity on unit vectors. Internally an inner-product search ranks by
 * the score -<o_r, q_r> (smaller is better), so the bounds, thresholds and
 * re-ranking rule are those of the distance search.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))

/* Rows [0, n) split evenly over `threads` POSIX threads; each row's
 * arithmetic is the same whatever the split. */
typedef void (*orc_rows_fn)(void* ctx, int64_t r0, int64_t r1);
typedef struct { orc_rows_fn fn; void* ctx; int64_t r0, r1; } orc_rows_job;
static void* orc_rows_run(void* a) {
  orc_rows_job* j = (orc_rows_job*)a;
  j->fn(j->ctx, j->r0, j->r1);
  return NULL;
}
static void parallel_rows(int64_t n, int32_t threads, orc_rows_fn fn, void* ctx) {
  if (threads < 1) threads = 1;
  if (threads > n) threads = (int32_t)(n > 0 ? n : 1);
  if (threads == 1) { fn(ctx, 0, n); return; }
  pthread_t th[256];
  orc_rows_job jobs[256];
  if (threads > 256) threads = 256;
  for (int32_t t = 0; t < threads; ++t) {
    jobs[t].fn = fn; jobs[t].ctx = ctx;
    jobs[t].r0 = n * t / threads; jobs[t].r1 = n * (t + 1) / threads;
    pthread_create(&th[t], NULL, orc_rows_run, &jobs[t]);
  }
  for (int32_t t = 0; t < threads; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11). Ten rounds; the key is bumped by the Weyl       */
/* constants between rounds.                                                */
/* ------------------------------------------------------------------------ */
enum {
  ORC_TAG_KINIT = 1,   /* k-means initial centroid ids            */
  ORC_TAG_GAUSS = 2,   /* Gaussian matrix that is orthonormalized */
  ORC_TAG_QUANT = 3,   /* u_i of the randomized query rounding    */
  ORC_TAG_SAMPLE = 4,  /* k-means training sample                 */
};

ORC_API void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                               uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox(uint64_t seed, uint32_t a, uint32_t b, uint32_t c, uint32_t d,
                   uint32_t out[4]) {
  uint32_t ctr[4] = {a, b, c, d};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Natural logarithm from the mathematics, written with basic IEEE ops only  */
/* so that it is reproducible to the bit: x = m * 2^e with m in             */
/* [sqrt(1/2), sqrt(2)); log m = 2 atanh(y), y = (m-1)/(m+1),               */
/* atanh(y) = sum_j y^(2j+1)/(2j+1) (12 terms: |y| <= 0.1716 so the tail is  */
/* below 2e-20 relative).                                                   */
/* ------------------------------------------------------------------------ */
ORC_API double orc_log(double x) {
  const double SQRT2 = 1.4142135623730951;
  const double LN2 = 0.6931471805599453;
  uint64_t bits;
  memcpy(&bits, &x, sizeof bits);
  int64_t e = (int64_t)((bits >> 52) & 0x7ffu) - 1023;
  uint64_t mb = (bits & 0x000fffffffffffffull) | 0x3ff0000000000000ull;
  double m;
  memcpy(&m, &mb, sizeof m);
  if (m > SQRT2) {
    m = m * 0.5;
    e = e + 1;
  }
  double num = m - 1.0;
  double den = m + 1.0;
  double y = num / den;
  double z = y * y;
  double p = 1.0 / 23.0;
  for (int j = 10; j >= 0; --j) {
    double coef = 1.0 / (double)(2 * j + 1);
    p = p * z;
    p = p + coef;
  }
  double t1 = (double)e * LN2;
  double t2 = (2.0 * y) * p;
  return t1 + t2;
}

/* ------------------------------------------------------------------------ */
/* Random orthogonal matrix P (paper §3.1.2; construction of App. B.3: a    */
/* D'xD' matrix of standard Gaussians orthonormalized row by row with       */
/* Gram-Schmidt).                                                           */
/* ------------------------------------------------------------------------ */

/* Standard Gaussians by the Marsaglia polar method (Marsaglia & Bray 1964).
 * Entry e = i*dpad + k belongs to pair m = e/2. Attempt t of pair m draws
 * Philox(seed; m, t, 0, TAG_GAUSS): u1 = (w0 << 21 | w1 >> 11) * 2^-53,
 * u2 = (w2 << 21 | w3 >> 11) * 2^-53, v = 2u - 1, s = v1^2 + v2^2; the first
 * attempt with 0 < s < 1 gives (v1 f, v2 f), f = sqrt(-2 log(s) / s). */
ORC_API void orc_gaussian_matrix(uint64_t seed, int32_t dpad, double* G) {
  const int64_t total = (int64_t)dpad * dpad;
  for (int64_t m = 0; m < total / 2; ++m) {
    double g0 = 0.0, g1 = 0.0;
    for (uint32_t t = 0; t < 64; ++t) {
      uint32_t w[4];
      philox(seed, (uint32_t)m, t, 0u, ORC_TAG_GAUSS, w);
      uint64_t a = ((uint64_t)w[0] << 21) | (uint64_t)(w[1] >> 11);
      uint64_t b = ((uint64_t)w[2] << 21) | (uint64_t)(w[3] >> 11);
      double u1 = (double)a * 0x1.0p-53;
      double u2 = (double)b * 0x1.0p-53;
      double v1 = 2.0 * u1 - 1.0;
      double v2 = 2.0 * u2 - 1.0;
      double s1 = v1 * v1;
      double s2 = v2 * v2;
      double s = s1 + s2;
      if (s > 0.0 && s < 1.0) {
        double lg = orc_log(s);
        double q = (-2.0 * lg) / s;
        double f = sqrt(q);
        g0 = v1 * f;
        g1 = v2 * f;
        break;
      }
    }
    G[2 * m] = g0;
    G[2 * m + 1] = g1;
  }
}

static double dot64(const double* a, const double* b, int32_t n) {
  double s = 0.0;
  for (int32_t k = 0; k < n; ++k) s = fma(a[k], b[k], s);
  return s;
}

/* Row-wise Gram-Schmidt of App. B.3: p_i = (g - sum_{j<i} <g,p_j> p_j) / norm.
 * The projection step is applied twice ("twice is enough", Giraud et al.
 * 2005) so that P^T P = I to ~1e-15; the second pass changes the result only
 * by rounding. All projection coefficients of one pass are taken from the
 * same vector (classical form). Sums: canonical FP64 (fma, ascending index). */
ORC_API void orc_orthonormalize_rows(int32_t dpad, const double* G, double* P) {
  double* v = (double*)malloc(sizeof(double) * (size_t)dpad);
  double* c = (double*)malloc(sizeof(double) * (size_t)dpad);
  for (int32_t i = 0; i < dpad; ++i) {
    memcpy(v, G + (int64_t)i * dpad, sizeof(double) * (size_t)dpad);
    for (int pass = 0; pass < 2; ++pass) {
      for (int32_t j = 0; j < i; ++j) c[j] = dot64(v, P + (int64_t)j * dpad, dpad);
      for (int32_t k = 0; k < dpad; ++k) {
        double t = 0.0;
        for (int32_t j = 0; j < i; ++j) t = fma(c[j], P[(int64_t)j * dpad + k], t);
        v[k] = v[k] - t;
      }
    }
    double nrm = sqrt(dot64(v, v, dpad));
    for (int32_t k = 0; k < dpad; ++k) P[(int64_t)i * dpad + k] = v[k] / nrm;
  }
  free(v);
  free(c);
}

ORC_API void orc_sample_rotation(uint64_t seed, int32_t dpad, double* P) {
  double* G = (double*)malloc(sizeof(double) * (size_t)dpad * (size_t)dpad);
  orc_gaussian_matrix(seed, dpad, G);
  orc_orthonormalize_rows(dpad, G, P);
  free(G);
}

/* ------------------------------------------------------------------------ */
/* Canonical FP32 kernels of the numerics contract.                          */
/* ------------------------------------------------------------------------ */
enum { ORC_METRIC_L2 = 0, ORC_METRIC_IP = 1 };

static float sqdist32(const float* a, const float* b, int32_t d) {
  float s = 0.0f;
  for (int32_t i = 0; i < d; ++i) {
    float t = a[i] - b[i];
    s = fmaf(t, t, s);
  }
  return s;
}

static float dot32(const float* a, const float* b, int32_t d) {
  float s = 0.0f;
  for (int32_t i = 0; i < d; ++i) s = fmaf(a[i], b[i], s);
  return s;
}

/* Unit vectors for the cosine similarity (footnote of §6: the cosine of two
 * vectors equals the inner product of their unit vectors):
 * out_r = x_r / ||x_r||, ||x_r|| = sqrt(canonical dot(x_r, x_r)); a zero row
 * stays zero. */
ORC_API void orc_normalize_rows(const float* x, int64_t n, int32_t d, float* out) {
  for (int64_t r = 0; r < n; ++r) {
    const float* xr = x + r * d;
    float nrm = sqrtf(dot32(xr, xr, d));
    for (int32_t i = 0; i < d; ++i) out[r * d + i] = (nrm > 0.0f) ? xr[i] / nrm : xr[i];
  }
}

/* out[r*nb + c] = canonical squared distance between a_r and b_c. */
ORC_API void orc_sqdist_matrix(const float* a, int64_t na, const float* b, int64_t nb,
                               int32_t d, float* out) {
  for (int64_t r = 0; r < na; ++r)
    for (int64_t c = 0; c < nb; ++c)
      out[r * nb + c] = sqdist32(a + r * d, b + c * d, d);
}

/* Inverse rotation P^{-1} x = P^T [x; 0] (paper §3.1.3 and §3.3): the input
 * is zero-padded from d to dpad dimensions, so only the first d rows of the
 * row-major P take part: out[k] = sum_{i<d} x_i P[i][k], canonical order. */
ORC_API void orc_rotate(const float* x, int64_t n, int32_t d, const float* P32,
                        int32_t dpad, float* out) {
  for (int64_t r = 0; r < n; ++r) {
    const float* xr = x + r * d;
    for (int32_t k = 0; k < dpad; ++k) {
      float s = 0.0f;
      for (int32_t i = 0; i < d; ++i) s = fmaf(xr[i], P32[(int64_t)i * dpad + k], s);
      out[r * dpad + k] = s;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* IVF k-means (paper §4: "clusters them with the KMeans algorithm").         */
/* The paper fixes no k-means variant. Reading: training                    */
/* set = all points, or the ids whose Philox(seed; id, 0, 0, TAG_SAMPLE) w0   */
/* lies below floor(2^32 * sample / n) when 0 < sample < n; init = K distinct */
/* training points chosen by Floyd's algorithm (Philox(seed; t, 0, 0,        */
/* TAG_KINIT) w0, r = (w0 * (j+1)) >> 32); Lloyd iterations: assign to the    */
/* argmin canonical distance (ties to the lower centroid id), update to the   */
/* mean (FP32 sum over members in ascending id order, divided by the count), */
/* an empty cluster keeps its centroid; finally every point is assigned with */
/* the final centroids.                                                      */
/* ------------------------------------------------------------------------ */
ORC_API int64_t orc_kmeans_sample(int64_t n, int64_t sample, uint64_t seed, int32_t* ids) {
  if (sample <= 0 || sample >= n) {
    for (int64_t i = 0; i < n; ++i) ids[i] = (int32_t)i;
    return n;
  }
  uint32_t thr = (uint32_t)(((uint64_t)sample << 32) / (uint64_t)n);
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i) {
    uint32_t w[4];
    philox(seed, (uint32_t)i, 0u, 0u, ORC_TAG_SAMPLE, w);
    if (w[0] < thr) ids[m++] = (int32_t)i;
  }
  return m;
}

/* Floyd's sampling of K distinct indices of [0, n), in the order chosen. */
ORC_API void orc_kmeans_init_ids(int64_t n, int32_t K, uint64_t seed, int32_t* out) {
  uint8_t* taken = (uint8_t*)calloc((size_t)n, 1);
  for (int32_t t = 0; t < K; ++t) {
    uint64_t j = (uint64_t)(n - K + t);
    uint32_t w[4];
    philox(seed, (uint32_t)t, 0u, 0u, ORC_TAG_KINIT, w);
    uint64_t r = ((uint64_t)w[0] * (j + 1)) >> 32;
    uint64_t pick = taken[r] ? j : r;
    taken[pick] = 1;
    out[t] = (int32_t)pick;
  }
  free(taken);
}

typedef struct {
  const float* data; const int32_t* rows; int32_t d; const float* cent; int32_t K;
  int32_t* assign; float* adist;
} assign_ctx;

static void assign_rows(void* vc, int64_t r0, int64_t r1) {
  assign_ctx* a = (assign_ctx*)vc;
  for (int64_t r = r0; r < r1; ++r) {
    const float* x = a->data + (int64_t)(a->rows ? a->rows[r] : r) * a->d;
    int32_t best = 0;
    float bd = sqdist32(x, a->cent, a->d);
    for (int32_t c = 1; c < a->K; ++c) {
      float dc = sqdist32(x, a->cent + (int64_t)c * a->d, a->d);
      if (dc < bd) { bd = dc; best = c; }
    }
    a->assign[r] = best;
    if (a->adist) a->adist[r] = bd;
  }
}

static void assign_all(const float* data, int64_t n, const int32_t* rows, int32_t d,
                       const float* cent, int32_t K, int32_t* assign, float* adist,
                       int32_t threads) {
  assign_ctx a = {data, rows, d, cent, K, assign, adist};
  parallel_rows(n, threads, assign_rows, &a);
}

ORC_API void orc_kmeans(const float* data, int64_t n, int32_t d, int32_t K, int32_t iters,
                        int64_t sample, uint64_t seed, float* centroids, int32_t* assign,
                        float* assign_dist, int32_t threads) {
  int32_t* rows = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int64_t m = orc_kmeans_sample(n, sample, seed, rows);
  if (m < K) m = orc_kmeans_sample(n, 0, seed, rows); /* too small a sample: use all */
  int32_t* init = (int32_t*)malloc(sizeof(int32_t) * (size_t)K);
  orc_kmeans_init_ids(m, K, seed, init);
  for (int32_t c = 0; c < K; ++c)
    memcpy(centroids + (int64_t)c * d, data + (int64_t)rows[init[c]] * d, sizeof(float) * (size_t)d);
  int32_t* a = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  float* sum = (float*)malloc(sizeof(float) * (size_t)d);
  for (int32_t it = 0; it < iters; ++it) {
    assign_all(data, m, rows, d, centroids, K, a, NULL, threads);
    for (int32_t c = 0; c < K; ++c) {
      int64_t cnt = 0;
      for (int32_t i = 0; i < d; ++i) sum[i] = 0.0f;
      for (int64_t r = 0; r < m; ++r) {  /* rows[] is ascending in id */
        if (a[r] != c) continue;
        const float* x = data + (int64_t)rows[r] * d;
        for (int32_t i = 0; i < d; ++i) sum[i] = sum[i] + x[i];
        ++cnt;
      }
      if (cnt == 0) continue;
      float fc = (float)cnt;
      for (int32_t i = 0; i < d; ++i) centroids[(int64_t)c * d + i] = sum[i] / fc;
    }
  }
  assign_all(data, n, NULL, d, centroids, K, assign, assign_dist, threads);
  free(rows); free(init); free(a); free(sum);
}

/* ------------------------------------------------------------------------ */
/* Index phase, Alg. 1 (normalize, codes, pre-computed factors).            */
/* ------------------------------------------------------------------------ */

/* For data vector o_r in cluster c (paper §3.1.1, §3.1.3, Alg. 1):
 *   res   = o_r - c                      (FP32, d entries; zero-padded)
 *   r     = P^{-1} res = P^T [res; 0]    (canonical dot, dpad entries)
 *   bit_k = (r_k >= 0)                   (sign code; -0 and +0 give 1)
 *   F1    = ||o_r - c||^2                (canonical squared distance)
 *   n_o   = sqrt(F1)
 *   a_o   = <o_bar, o> = ||r||_1 / (sqrt(dpad) n_o), at most 1; n_o = 0 -> 1
 *           (App. B.1: <o_bar,o> = ||P^{-1} o||_1 / sqrt(D))
 *   F2    = 2 n_o / a_o                  (coefficient of the estimator term)
 *   F3    = n_o sqrt(1 - a_o^2) / a_o    (coefficient of the error bound)
 *   G     = 2 popcount(bits) - dpad      (as float)
 * Codes are dpad/64 words per vector, bit k in word k>>6 at position k&63.
 * factors[4*n + {0,1,2,3}] = {F1, F2, F3, G}.
 *
 * Inner-product metric (footnote of §6): <o_r, q_r> = ||o_r - c|| ||q_r - c||
 * <o, q> + <o_r - c, c> + <q_r, c>, so the score -<o_r, q_r> takes the form
 * (F1 + add) - F2 xq of the distance estimator with
 *   F1 = -<o_r - c, c>  (canonical dot of the FP32 residual and c)
 *   F2 = n_o / a_o      (half the distance coefficient: exact scaling)
 *   F3 = n_o sqrt(1 - a_o^2) / (2 a_o)   (half: the score's bound is half
 *                                          the distance's)
 * and add = -<q_r, c> per (query, cluster).                                */
typedef struct {
  const float* data; int32_t d; const float* centroids; const int32_t* assign;
  const float* P32; int32_t dpad; uint64_t* codes; float* factors; int32_t metric;
} encode_ctx;

static void encode_rows(void* vc, int64_t v0, int64_t v1) {
  encode_ctx* E = (encode_ctx*)vc;
  const float* data = E->data; const int32_t d = E->d; const float* centroids = E->centroids;
  const int32_t* assign = E->assign; const float* P32 = E->P32; const int32_t dpad = E->dpad;
  uint64_t* codes = E->codes; float* factors = E->factors;
  const int32_t W = dpad / 64;
  const float sqrt_dpad = sqrtf((float)dpad);
  float* res = (float*)malloc(sizeof(float) * (size_t)d);
  float* r = (float*)malloc(sizeof(float) * (size_t)dpad);
  for (int64_t v = v0; v < v1; ++v) {
    const float* o = data + v * d;
    const float* c = centroids + (int64_t)assign[v] * d;
    for (int32_t i = 0; i < d; ++i) res[i] = o[i] - c[i];
    float F1 = sqdist32(o, c, d);
    orc_rotate(res, 1, d, P32, dpad, r);
    uint64_t* code = codes + v * W;
    for (int32_t w = 0; w < W; ++w) code[w] = 0;
    int32_t pc = 0;
    float l1 = 0.0f;
    for (int32_t k = 0; k < dpad; ++k) {
      if (r[k] >= 0.0f) {
        code[k >> 6] |= (uint64_t)1 << (k & 63);
        ++pc;
      }
      l1 = l1 + fabsf(r[k]);
    }
    float n_o = sqrtf(F1);
    float a_o = 1.0f;
    if (n_o > 0.0f) {
      float den = sqrt_dpad * n_o;
      a_o = l1 / den;
      if (a_o > 1.0f) a_o = 1.0f;
    }
    float two_no = 2.0f * n_o;
    float F2 = two_no / a_o;
    float a2 = a_o * a_o;
    float om = 1.0f - a2;
    float sq = sqrtf(om);
    float num = n_o * sq;
    float F3 = num / a_o;
    if (E->metric == ORC_METRIC_IP) {
      float oc = dot32(res, c, d);
      F1 = -oc;
      F2 = 0.5f * F2;
      F3 = 0.5f * F3;
    }
    factors[4 * v + 0] = F1;
    factors[4 * v + 1] = F2;
    factors[4 * v + 2] = F3;
    factors[4 * v + 3] = (float)(2 * pc - dpad);
  }
  free(res);
  free(r);
}

ORC_API void orc_encode_metric(const float* data, int64_t n, int32_t d, const float* centroids,
                               const int32_t* assign, const float* P32, int32_t dpad,
                               uint64_t* codes, float* factors, int32_t metric,
                               int32_t threads) {
  encode_ctx E = {data, d, centroids, assign, P32, dpad, codes, factors, metric};
  parallel_rows(n, threads, encode_rows, &E);
}

ORC_API void orc_encode(const float* data, int64_t n, int32_t d, const float* centroids,
                        const int32_t* assign, const float* P32, int32_t dpad,
                        uint64_t* codes, float* factors, int32_t threads) {
  orc_encode_metric(data, n, d, centroids, assign, P32, dpad, codes, factors, ORC_METRIC_L2,
                    threads);
}

/* ------------------------------------------------------------------------ */
/* Query phase, Alg. 2.                                                      */
/* ------------------------------------------------------------------------ */

/* Randomized uniform scalar quantization of the rotated query residual
 * (paper §3.3.1). Reading: the un-normalized qd = P^T(q_r - c) is quantized
 * (the quantizer is affine-equivariant, so the codes equal those of the unit
 * q' = qd / ||q_r - c||), with qd = rq - ptc where rq = P^T[q_r;0] and
 * ptc = P^T[c;0] (linearity). Steps:
 *   v_l = min qd, v_r = max qd, Delta = (v_r - v_l) / (2^Bq - 1)
 *   qu_k = floor((qd_k - v_l)/Delta + u_k), clamped to 2^Bq - 1; Delta = 0 -> 0
 *   u_k = (w >> 8) 2^-24 from Philox(seed; k/4, qid, cid, TAG_QUANT), word k%4
 * Outputs: qu (dpad ints, may be NULL), the Bq bit-planes (plane j: dpad/64
 * words of bit j of qu, paper §3.3.2 Eq. efficient-computation), sum(qu) and
 * the per-(query, cluster) constants of the estimator:
 *   meta[0] = A = Delta / sqrt(dpad), meta[1] = B = v_l / sqrt(dpad),
 *   meta[2] = E = sqrt(nq2) * 2 eps0 / sqrt(dpad - 1), meta[3] = nq2,
 *   meta[4] = v_l, meta[5] = Delta.                                         */
ORC_API void orc_quantize(const float* rq, const float* ptc, int32_t dpad, int32_t bq,
                          uint64_t seed, int32_t qid, int32_t cid, float nq2, float eps0,
                          int32_t* qu_out, uint64_t* planes, int32_t* sum_qu, float* meta) {
  const int32_t W = dpad / 64;
  const int32_t qmax = (1 << bq) - 1;
  float* qd = (float*)malloc(sizeof(float) * (size_t)dpad);
  int32_t* qu = (int32_t*)malloc(sizeof(int32_t) * (size_t)dpad);
  for (int32_t k = 0; k < dpad; ++k) qd[k] = rq[k] - ptc[k];
  float vl = qd[0], vr = qd[0];
  for (int32_t k = 1; k < dpad; ++k) {
    if (qd[k] < vl) vl = qd[k];
    if (qd[k] > vr) vr = qd[k];
  }
  float range = vr - vl;
  float delta = range / (float)qmax;
  int32_t s = 0;
  for (int32_t k = 0; k < dpad; ++k) {
    int32_t q = 0;
    if (delta > 0.0f) {
      uint32_t w[4];
      philox(seed, (uint32_t)(k >> 2), (uint32_t)qid, (uint32_t)cid, ORC_TAG_QUANT, w);
      float u = (float)(w[k & 3] >> 8) * 0x1.0p-24f;
      float x = (qd[k] - vl) / delta;
      float y = x + u;
      q = (int32_t)floorf(y);
      if (q > qmax) q = qmax;
    }
    qu[k] = q;
    s += q;
  }
  for (int32_t j = 0; j < bq; ++j)
    for (int32_t w = 0; w < W; ++w) planes[j * W + w] = 0;
  for (int32_t k = 0; k < dpad; ++k)
    for (int32_t j = 0; j < bq; ++j)
      if ((qu[k] >> j) & 1) planes[j * W + (k >> 6)] |= (uint64_t)1 << (k & 63);
  if (qu_out) memcpy(qu_out, qu, sizeof(int32_t) * (size_t)dpad);
  *sum_qu = s;
  const float sqrt_dpad = sqrtf((float)dpad);
  const float keps = (2.0f * eps0) / sqrtf((float)(dpad - 1));
  const float n_q = sqrtf(nq2);
  meta[0] = delta / sqrt_dpad;
  meta[1] = vl / sqrt_dpad;
  meta[2] = n_q * keps;
  meta[3] = nq2;
  meta[4] = vl;
  meta[5] = delta;
  free(qd);
  free(qu);
}

/* <x_b, qu> by the bit-plane decomposition (paper §3.3.2):
 * sum_j 2^j popcount(x_b AND qu^(j)). */
ORC_API int32_t orc_bitplane_ip(const uint64_t* code, const uint64_t* planes, int32_t W,
                                int32_t bq) {
  int32_t ip = 0;
  for (int32_t j = 0; j < bq; ++j) {
    int32_t pj = 0;
    for (int32_t w = 0; w < W; ++w) pj += __builtin_popcountll(code[w] & planes[j * W + w]);
    ip += pj << j;
  }
  return ip;
}

/* Estimated squared distance and its bounds for one (query, code) pair.
 * <x_bar, q_bar> (un-normalized, paper §3.3.2 Eq. compute-inner-product):
 *   xq = (Delta (2 ip - sum qu) + v_l (2 pc - D')) / sqrt(D') = A t1 + B t2
 * estimator (Theorem 3.2) in the distance identity of §3.1.1:
 *   dist = ||o_r-c||^2 + ||q_r-c||^2 - 2 ||o_r-c|| ||q_r-c|| <o_bar,q>/<o_bar,o>
 *        = (F1 + nq2) - F2 xq
 * error bound (Theorem 3.2) times 2 ||o_r-c|| ||q_r-c||:
 *   e = F3 E,  LB = dist - e,  UB = dist + e.
 * Fixed FP32 order, no contraction. out = {dist, LB, UB}.                   */
ORC_API void orc_estimate(int32_t ip, int32_t sum_qu, const float* fac, const float* meta,
                          float* out) {
  float t1 = (float)(2 * ip - sum_qu);
  float t2 = fac[3];
  float p1 = meta[0] * t1;
  float p2 = meta[1] * t2;
  float xq = p1 + p2;
  float u1 = fac[0] + meta[3];
  float u2 = fac[1] * xq;
  float dist = u1 - u2;
  float e = fac[2] * meta[2];
  out[0] = dist;
  out[1] = dist - e;
  out[2] = dist + e;
}

/* ------------------------------------------------------------------------ */
/* IVF search (paper §4): probe the nprobe nearest centroids, estimate the   */
/* distances of every code in the probed buckets, drop by the error bound,   */
/* re-rank the rest by exact distance.                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
  /* index */
  const float* data;        /* n x d, original id order              */
  const float* centroids;   /* K x d                                 */
  const float* ptc;         /* K x dpad: P^T [c; 0]                  */
  const float* P32;         /* dpad x dpad, row-major (rows >= d unused) */
  const uint64_t* codes;    /* n x dpad/64, original id order        */
  const float* factors;     /* n x 4, original id order              */
  const int32_t* bucket_off;/* K+1                                   */
  const int32_t* bucket_ids;/* n: ids of bucket c in ascending order */
  int64_t n;
  int32_t d, dpad, K;
  const int32_t* assign;    /* n: cluster of each id                 */
  int32_t metric;           /* ORC_METRIC_L2 or ORC_METRIC_IP        */
} orc_index;

typedef struct {
  int32_t k, nprobe, bq, mode; /* mode 0: order-independent re-rank set; 1: sequential */
  float eps0;
  uint64_t seed;
} orc_params;

typedef struct {
  /* optional per-query trace outputs (NULL to skip) */
  int32_t* probe_ids;   /* nprobe            */
  float* probe_dist;    /* nprobe            */
  float* rq;            /* dpad              */
  uint64_t* planes;     /* nprobe x bq x W   */
  int32_t* sum_qu;      /* nprobe            */
  float* meta;          /* nprobe x 6        */
  int32_t* pair_id;     /* cap_pairs         */
  int32_t* pair_ip;     /* cap_pairs         */
  float* pair_est;      /* cap_pairs x 3     */
  int32_t cap_pairs;
  int32_t n_pairs;      /* out */
  float tau;            /* out (mode 0)      */
  int32_t* surv_ids;    /* cap_surv: the re-rank set, ascending id */
  int32_t cap_surv;
  int32_t n_surv;       /* out */
  float tau_ub, tau1;   /* out (mode 0) */
} orc_trace;

static int cmp_pair(float da, int32_t ia, float db, int32_t ib) {
  if (da < db) return -1;
  if (da > db) return 1;
  return (ia < ib) ? -1 : (ia > ib);
}

/* insertion of (dist, id) into an ascending top-k list of size *cnt <= k */
static void topk_insert(float* td, int32_t* ti, int32_t* cnt, int32_t k, float d, int32_t id) {
  int32_t c = *cnt;
  if (c == k && cmp_pair(d, id, td[k - 1], ti[k - 1]) >= 0) return;
  int32_t pos = (c < k) ? c : k - 1;
  while (pos > 0 && cmp_pair(d, id, td[pos - 1], ti[pos - 1]) < 0) {
    td[pos] = td[pos - 1];
    ti[pos] = ti[pos - 1];
    --pos;
  }
  td[pos] = d;
  ti[pos] = id;
  if (c < k) *cnt = c + 1;
}

static int cmp_float(const void* a, const void* b) {
  float x = *(const float*)a, y = *(const float*)b;
  return (x < y) ? -1 : (x > y);
}

static int cmp_int(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x < y) ? -1 : (x > y);
}

/* Select the nsel smallest of dist[0..K) by (dist, id), ascending. */
ORC_API void orc_select(const float* dist, int64_t nrows, int32_t K, int32_t nsel,
                        int32_t* ids, float* sel_dist) {
  float* td = (float*)malloc(sizeof(float) * (size_t)nsel);
  int32_t* ti = (int32_t*)malloc(sizeof(int32_t) * (size_t)nsel);
  for (int64_t r = 0; r < nrows; ++r) {
    int32_t cnt = 0;
    for (int32_t c = 0; c < K; ++c) topk_insert(td, ti, &cnt, nsel, dist[r * K + c], c);
    for (int32_t j = 0; j < nsel; ++j) {
      ids[r * nsel + j] = (j < cnt) ? ti[j] : -1;
      if (sel_dist) sel_dist[r * nsel + j] = (j < cnt) ? td[j] : INFINITY;
    }
  }
  free(td);
  free(ti);
}

/* Exact score of (q, id): the canonical squared distance, or -<q, o> for
 * the inner-product metric. */
static float exact_score(const orc_index* X, const float* q, int32_t id) {
  const float* o = X->data + (int64_t)id * X->d;
  return X->metric == ORC_METRIC_IP ? -dot32(q, o, X->d) : sqdist32(q, o, X->d);
}

/* Centroid score: ||q - c||^2, or -<q, c> (probe the largest inner products). */
static float centroid_score(const orc_index* X, const float* q, int32_t c) {
  const float* cc = X->centroids + (int64_t)c * X->d;
  return X->metric == ORC_METRIC_IP ? -dot32(q, cc, X->d) : sqdist32(q, cc, X->d);
}

static void search_one(const orc_index* X, const orc_params* p, const float* q, int32_t qid,
                       int64_t* out_ids, float* out_dist, orc_trace* tr, float* scratch_cd,
                       int32_t* scratch_ids, float* scratch_pd) {
  const int32_t d = X->d, dpad = X->dpad, K = X->K, W = dpad / 64;
  const int32_t nprobe = p->nprobe < K ? p->nprobe : K;
  /* centroid distances and the nprobe nearest (paper §4) */
  for (int32_t c = 0; c < K; ++c) scratch_cd[c] = centroid_score(X, q, c);
  orc_select(scratch_cd, 1, K, nprobe, scratch_ids, scratch_pd);
  /* inverse rotation of the raw query (Alg. 2 step 1, by linearity) */
  float* rq = (float*)malloc(sizeof(float) * (size_t)dpad);
  orc_rotate(q, 1, d, X->P32, dpad, rq);
  if (tr) {
    memcpy(tr->probe_ids, scratch_ids, sizeof(int32_t) * (size_t)nprobe);
    memcpy(tr->probe_dist, scratch_pd, sizeof(float) * (size_t)nprobe);
    if (tr->rq) memcpy(tr->rq, rq, sizeof(float) * (size_t)dpad);
  }
  /* total number of pairs */
  int64_t total = 0;
  for (int32_t j = 0; j < nprobe; ++j) {
    int32_t c = scratch_ids[j];
    total += X->bucket_off[c + 1] - X->bucket_off[c];
  }
  int32_t* pid = (int32_t*)malloc(sizeof(int32_t) * (size_t)(total + 1));
  float* pest = (float*)malloc(sizeof(float) * 3 * (size_t)(total + 1));
  uint64_t* planes = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)p->bq * W);
  float meta[6];
  int64_t t = 0;
  int32_t k = p->k;
  float* td = (float*)malloc(sizeof(float) * (size_t)k);
  int32_t* ti = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
  int32_t cnt = 0;
  for (int32_t j = 0; j < nprobe; ++j) {
    int32_t c = scratch_ids[j];
    int32_t sq;
    /* ||q_r - c||^2 scales the bound; the estimator's additive constant
     * (meta[3]) is the centroid score: ||q_r - c||^2, or -<q_r, c> */
    float nq2 = (X->metric == ORC_METRIC_IP)
                    ? sqdist32(q, X->centroids + (int64_t)c * d, d) : scratch_pd[j];
    orc_quantize(rq, X->ptc + (int64_t)c * dpad, dpad, p->bq, p->seed, qid, c, nq2,
                 p->eps0, NULL, planes, &sq, meta);
    meta[3] = scratch_pd[j];
    if (tr) {
      memcpy(tr->planes + (int64_t)j * p->bq * W, planes, sizeof(uint64_t) * (size_t)p->bq * W);
      tr->sum_qu[j] = sq;
      memcpy(tr->meta + 6 * j, meta, sizeof meta);
    }
    for (int32_t b = X->bucket_off[c]; b < X->bucket_off[c + 1]; ++b) {
      int32_t id = X->bucket_ids[b];
      int32_t ip = orc_bitplane_ip(X->codes + (int64_t)id * W, planes, W, p->bq);
      float est[3];
      orc_estimate(ip, sq, X->factors + 4 * (int64_t)id, meta, est);
      if (tr && t < tr->cap_pairs) {
        tr->pair_id[t] = id;
        tr->pair_ip[t] = ip;
        tr->pair_est[3 * t + 0] = est[0];
        tr->pair_est[3 * t + 1] = est[1];
        tr->pair_est[3 * t + 2] = est[2];
      }
      pid[t] = id;
      pest[3 * t + 0] = est[0];
      pest[3 * t + 1] = est[1];
      pest[3 * t + 2] = est[2];
      if (p->mode == 1) {
        /* paper-literal: drop o if its lower bound exceeds the exact
         * distance of the current k-th nearest neighbour (§4) */
        float kth = (cnt == k) ? td[k - 1] : INFINITY;
        if (!(est[1] > kth)) {
          float ex = exact_score(X, q, id);
          topk_insert(td, ti, &cnt, k, ex, id);
        }
      }
      ++t;
    }
  }
  if (tr) tr->n_pairs = (int32_t)t;
  if (p->mode == 0) {
    /* Order-independent reading of the re-ranking rule of §4 for k >= 1:
     *  tau_ub = k-th smallest upper bound over all estimated codes;
     *  pilot  = the 4k codes with the smallest estimated distance (by
     *           (estimate, id)) among those with LB <= tau_ub, re-ranked
     *           first;
     *  tau1   = k-th smallest exact distance within the pilot;
     *  tau    = min(tau_ub, tau1) (each is at least the k-th nearest exact
     *           distance, w.h.p. for tau_ub, always for tau1);
     *  re-rank set = pilot + every code whose lower bound is <= tau. */
    float tau_ub = INFINITY, tau1 = INFINITY;
    if (t >= k) {
      float* ubs = (float*)malloc(sizeof(float) * (size_t)t);
      for (int64_t i = 0; i < t; ++i) ubs[i] = pest[3 * i + 2];
      qsort(ubs, (size_t)t, sizeof(float), cmp_float);
      tau_ub = ubs[k - 1];
      free(ubs);
    }
    const int64_t m = 4 * (int64_t)k;
    uint8_t* in_set = (uint8_t*)calloc((size_t)(t + 1), 1);
    /* pilot: m smallest (estimate, id) with LB <= tau_ub, by selection into a
     * sorted list */
    float* pd = (float*)malloc(sizeof(float) * (size_t)(m + 1));
    int32_t* pi = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
    int32_t* pix = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
    int32_t pc = 0;
    for (int64_t i = 0; i < t; ++i) {
      if (!(pest[3 * i + 1] <= tau_ub)) continue;
      float e = pest[3 * i + 0];
      int32_t id = pid[i];
      if (pc == m && cmp_pair(e, id, pd[m - 1], pi[m - 1]) >= 0) continue;
      int32_t pos = (pc < m) ? pc : (int32_t)m - 1;
      while (pos > 0 && cmp_pair(e, id, pd[pos - 1], pi[pos - 1]) < 0) {
        pd[pos] = pd[pos - 1]; pi[pos] = pi[pos - 1]; pix[pos] = pix[pos - 1];
        --pos;
      }
      pd[pos] = e; pi[pos] = id; pix[pos] = (int32_t)i;
      if (pc < m) ++pc;
    }
    float* pex = (float*)malloc(sizeof(float) * (size_t)(m + 1));
    for (int32_t j = 0; j < pc; ++j) {
      in_set[pix[j]] = 1;
      pex[j] = exact_score(X, q, pi[j]);
    }
    if (pc >= k) {
      qsort(pex, (size_t)pc, sizeof(float), cmp_float);
      tau1 = pex[k - 1];
    }
    float tau = tau_ub < tau1 ? tau_ub : tau1;
    for (int64_t i = 0; i < t; ++i)
      if (pest[3 * i + 1] <= tau) in_set[i] = 1;
    int32_t ns = 0;
    int32_t* surv = (int32_t*)malloc(sizeof(int32_t) * (size_t)(t + 1));
    for (int64_t i = 0; i < t; ++i)
      if (in_set[i]) surv[ns++] = pid[i];
    qsort(surv, (size_t)ns, sizeof(int32_t), cmp_int);
    for (int32_t i = 0; i < ns; ++i) {
      float ex = exact_score(X, q, surv[i]);
      topk_insert(td, ti, &cnt, k, ex, surv[i]);
    }
    if (tr) {
      tr->tau = tau;
      tr->tau_ub = tau_ub;
      tr->tau1 = tau1;
      tr->n_surv = ns;
      if (tr->surv_ids) {
        int32_t mm = ns < tr->cap_surv ? ns : tr->cap_surv;
        memcpy(tr->surv_ids, surv, sizeof(int32_t) * (size_t)mm);
      }
    }
    free(surv); free(in_set); free(pd); free(pi); free(pix); free(pex);
  }
  /* inner products are returned as <o_r, q_r> (descending), -inf pads */
  const int neg = X->metric == ORC_METRIC_IP;
  for (int32_t j = 0; j < k; ++j) {
    out_ids[j] = (j < cnt) ? ti[j] : -1;
    float v = (j < cnt) ? td[j] : INFINITY;
    out_dist[j] = neg ? -v : v;
  }
  free(rq); free(pid); free(pest); free(planes); free(td); free(ti);
}

/* Trace search of one query (for staged parity tests). */
ORC_API void orc_search_trace(const orc_index* X, const orc_params* p, const float* q,
                              int32_t qid, int64_t* out_ids, float* out_dist, orc_trace* tr) {
  float* cd = (float*)malloc(sizeof(float) * (size_t)X->K);
  int32_t* ids = (int32_t*)malloc(sizeof(int32_t) * (size_t)X->K);
  float* pd = (float*)malloc(sizeof(float) * (size_t)X->K);
  search_one(X, p, q, qid, out_ids, out_dist, tr, cd, ids, pd);
  free(cd); free(ids); free(pd);
}

typedef struct {
  const orc_index* X;
  const orc_params* p;
  const float* Q;
  const int32_t* npq;  /* per-query probe counts or NULL */
  int64_t q0, q1;
  int64_t* ids;
  float* dist;
} orc_job;

static void* search_range(void* arg) {
  orc_job* J = (orc_job*)arg;
  float* cd = (float*)malloc(sizeof(float) * (size_t)J->X->K);
  int32_t* ids = (int32_t*)malloc(sizeof(int32_t) * (size_t)J->X->K);
  float* pd = (float*)malloc(sizeof(float) * (size_t)J->X->K);
  for (int64_t i = J->q0; i < J->q1; ++i) {
    orc_params pi = *J->p;
    if (J->npq) {  /* this query's own count, within [1, nprobe] */
      int32_t v = J->npq[i];
      pi.nprobe = v < 1 ? 1 : (v > J->p->nprobe ? J->p->nprobe : v);
    }
    search_one(J->X, &pi, J->Q + i * J->X->d, (int32_t)i, J->ids + i * J->p->k,
               J->dist + i * J->p->k, NULL, cd, ids, pd);
  }
  free(cd); free(ids); free(pd);
  return NULL;
}

/* Search nq queries, split evenly over `threads` POSIX threads (query i uses
 * qid = i for its quantization stream). npq (NULL = every query probes
 * p->nprobe buckets): query i probes its npq[i] nearest buckets, clamped to
 * [1, p->nprobe] -- the search of a per-query (learned) probe count. */
ORC_API void orc_search_pq(const orc_index* X, const orc_params* p, const float* Q, int64_t nq,
                           const int32_t* npq, int32_t threads, int64_t* out_ids,
                           float* out_dist) {
  if (threads < 1) threads = 1;
  if (threads > nq) threads = (int32_t)(nq > 0 ? nq : 1);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
  orc_job* jobs = (orc_job*)malloc(sizeof(orc_job) * (size_t)threads);
  for (int32_t t = 0; t < threads; ++t) {
    jobs[t].X = X; jobs[t].p = p; jobs[t].Q = Q; jobs[t].npq = npq;
    jobs[t].q0 = nq * t / threads;
    jobs[t].q1 = nq * (t + 1) / threads;
    jobs[t].ids = out_ids; jobs[t].dist = out_dist;
  }
  if (threads == 1) {
    search_range(&jobs[0]);
  } else {
    for (int32_t t = 0; t < threads; ++t) pthread_create(&th[t], NULL, search_range, &jobs[t]);
    for (int32_t t = 0; t < threads; ++t) pthread_join(th[t], NULL);
  }
  free(th);
  free(jobs);
}

/* Search nq queries, every one probing p->nprobe buckets. */
ORC_API void orc_search(const orc_index* X, const orc_params* p, const float* Q, int64_t nq,
                        int32_t threads, int64_t* out_ids, float* out_dist) {
  orc_search_pq(X, p, Q, nq, NULL, threads, out_ids, out_dist);
}

typedef struct {
  const float* data; int64_t n; int32_t d; const float* Q; int32_t k; const uint8_t* allowed;
  int64_t* out_ids; float* out_dist; int32_t metric;
} bf_ctx;

static void bf_rows(void* vc, int64_t q0, int64_t q1) {
  bf_ctx* B = (bf_ctx*)vc;
  const int32_t k = B->k, d = B->d;
  float* td = (float*)malloc(sizeof(float) * (size_t)k);
  int32_t* ti = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
  for (int64_t i = q0; i < q1; ++i) {
    int32_t cnt = 0;
    const uint8_t* al = B->allowed ? B->allowed + i * B->n : NULL;
    for (int64_t v = 0; v < B->n; ++v) {
      if (al && !al[v]) continue;
      float sc = (B->metric == ORC_METRIC_IP) ? -dot32(B->Q + i * d, B->data + v * d, d)
                                              : sqdist32(B->Q + i * d, B->data + v * d, d);
      topk_insert(td, ti, &cnt, k, sc, (int32_t)v);
    }
    for (int32_t j = 0; j < k; ++j) {
      B->out_ids[i * k + j] = (j < cnt) ? ti[j] : -1;
      float v = (j < cnt) ? td[j] : INFINITY;
      B->out_dist[i * k + j] = (B->metric == ORC_METRIC_IP) ? -v : v;
    }
  }
  free(td);
  free(ti);
}

/* Exact k nearest neighbours by brute force (canonical FP32 distance,
 * ties by id), restricted to `allowed` ids when allowed != NULL. */
ORC_API void orc_bruteforce_knn(const float* data, int64_t n, int32_t d, const float* Q,
                                int64_t nq, int32_t k, const uint8_t* allowed,
                                int64_t* out_ids, float* out_dist, int32_t threads) {
  bf_ctx B = {data, n, d, Q, k, allowed, out_ids, out_dist, ORC_METRIC_L2};
  parallel_rows(nq, threads, bf_rows, &B);
}

/* Exact k largest inner products (canonical FP32 dot, ranked by the score
 * -<q, o> with ties by id); out_ip holds <q, o>, -inf pads. */
ORC_API void orc_bruteforce_ip(const float* data, int64_t n, int32_t d, const float* Q,
                               int64_t nq, int32_t k, int64_t* out_ids, float* out_ip,
                               int32_t threads) {
  bf_ctx B = {data, n, d, Q, k, NULL, out_ids, out_ip, ORC_METRIC_IP};
  parallel_rows(nq, threads, bf_rows, &B);
}

/* ------------------------------------------------------------------------ */
/* Single-code estimator (§3.3.2, the first case: one query and one code at */
/* a time, as a graph index would visit them).                              */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_index* X; const orc_params* p; const float* Q; const int64_t* ids; int32_t m;
  float* out;
} est_ctx;

static void est_rows(void* vc, int64_t i0, int64_t i1) {
  est_ctx* E = (est_ctx*)vc;
  const orc_index* X = E->X;
  const orc_params* p = E->p;
  const int32_t d = X->d, dpad = X->dpad, W = dpad / 64;
  float* rq = (float*)malloc(sizeof(float) * (size_t)dpad);
  uint64_t* planes = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)p->bq * W);
  for (int64_t i = i0; i < i1; ++i) {
    const float* q = E->Q + i * d;
    orc_rotate(q, 1, d, X->P32, dpad, rq);
    for (int32_t j = 0; j < E->m; ++j) {
      float* o = E->out + 3 * (i * E->m + j);
      int64_t id = E->ids[i * E->m + j];
      if (id < 0) {
        o[0] = o[1] = o[2] = NAN;
        continue;
      }
      int32_t c = X->assign[id];
      float nq2 = sqdist32(q, X->centroids + (int64_t)c * d, d);
      float meta[6];
      int32_t sq;
      orc_quantize(rq, X->ptc + (int64_t)c * dpad, dpad, p->bq, p->seed, (int32_t)i, c, nq2,
                   p->eps0, NULL, planes, &sq, meta);
      meta[3] = centroid_score(X, q, c);
      int32_t ip = orc_bitplane_ip(X->codes + id * W, planes, W, p->bq);
      float est[3];
      orc_estimate(ip, sq, X->factors + 4 * id, meta, est);
      if (X->metric == ORC_METRIC_IP) {
        o[0] = -est[0];
        o[1] = -est[2];
        o[2] = -est[1];
      } else {
        o[0] = est[0];
        o[1] = est[1];
        o[2] = est[2];
      }
    }
  }
  free(rq);
  free(planes);
}

/* For query i (quantization stream qid = i) and code ids[i m + j]: quantize
 * the rotated query against the code's own cluster c (cid = c) and evaluate
 * the estimator with its bound. out[3 (i m + j) + {0, 1, 2}] = {estimate,
 * lower bound, upper bound} of the squared distance, or of <o_r, q_r> for the
 * inner-product metric; an id of -1 gives three NaNs. */
ORC_API void orc_estimate_codes(const orc_index* X, const orc_params* p, const float* Q,
                                int64_t nq, const int64_t* ids, int32_t m, float* out,
                                int32_t threads) {
  est_ctx E = {X, p, Q, ids, m, out};
  parallel_rows(nq, threads, est_rows, &E);
}

/* ------------------------------------------------------------------------ */
/* FP64 references for the statistical pins (no quantization of q').        */
/* ------------------------------------------------------------------------ */

/* Given unit o and q (dimension dim) and an orthogonal P (dim x dim,
 * row-major), return {<o_bar,o>, <o_bar,q>, estimate <o_bar,q>/<o_bar,o>,
 * <o_bar, e1>} in FP64 with o_bar = P x_bar, x_bar = sign(P^T o)/sqrt(dim)
 * (paper §3.1.3, Lemma 3.1, Theorem 3.2). */
ORC_API void orc_estimator_fp64(const double* P, int32_t dim, const double* o, const double* q,
                                double* out) {
  double* r = (double*)malloc(sizeof(double) * (size_t)dim);
  double* x = (double*)malloc(sizeof(double) * (size_t)dim);
  double* ob = (double*)malloc(sizeof(double) * (size_t)dim);
  double* e1 = (double*)malloc(sizeof(double) * (size_t)dim);
  double inv = 1.0 / sqrt((double)dim);
  for (int32_t k = 0; k < dim; ++k) {
    double s = 0.0;
    for (int32_t i = 0; i < dim; ++i) s = fma(P[(int64_t)i * dim + k], o[i], s);
    r[k] = s;
    x[k] = (s >= 0.0) ? inv : -inv;
  }
  for (int32_t i = 0; i < dim; ++i) {
    double s = 0.0;
    for (int32_t k = 0; k < dim; ++k) s = fma(P[(int64_t)i * dim + k], x[k], s);
    ob[i] = s;
  }
  double oo = dot64(ob, o, dim);
  double oq = dot64(ob, q, dim);
  double qo = dot64(q, o, dim);
  double nrm = 0.0;
  for (int32_t i = 0; i < dim; ++i) {
    e1[i] = q[i] - qo * o[i];
    nrm = fma(e1[i], e1[i], nrm);
  }
  nrm = sqrt(nrm);
  double oe = 0.0;
  if (nrm > 0.0)
    for (int32_t i = 0; i < dim; ++i) oe = fma(ob[i], e1[i] / nrm, oe);
  out[0] = oo;
  out[1] = oq;
  out[2] = oq / oo;
  out[3] = oe;
  free(r); free(x); free(ob); free(e1);
}
