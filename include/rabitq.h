/*
 * rabitq.h -- C-ABI of the GB300 (sm_103a) RaBitQ IVF library.
 *
 * RaBitQ (Gao & Long, SIGMOD 2024) quantizes each data vector to a D'-bit
 * sign code of its inverse-rotated residual and estimates squared distances
 * with an unbiased estimator whose error bound decides which candidates are
 * re-ranked with exact distances. This library builds the IVF index (Alg. 1
 * and §4 of the paper) and answers k-nearest-neighbour queries (Alg. 2 and
 * §4) entirely in its own CUDA kernels.
 *
 * Conventions for every call:
 *  - Return value: RABITQ_OK (0) or a negative rabitq_status; the message of
 *    the last failure on the calling thread is rabitq_last_error().
 *  - Inputs are caller-owned and read-only; the library copies what it keeps.
 *  - Outputs are caller-allocated; on error their contents are undefined.
 *  - Host pointers unless the options say a pointer is device memory.
 *  - Matrices are row-major, float32 unless stated.
 *  - An index is owned by the library from rabitq_build/rabitq_index_load
 *    until rabitq_free. Searches on one const index may run concurrently
 *    from several host threads on distinct streams.
 */
#ifndef RABITQ_H
#define RABITQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rabitq_index rabitq_index;
typedef struct rabitq_predictor rabitq_predictor;
typedef struct rabitq_plan rabitq_plan;

typedef enum {
  RABITQ_OK = 0,
  RABITQ_EINVAL = -1,       /* invalid argument (sizes, ranges, null pointer)  */
  RABITQ_ENOMEM = -2,       /* device or host allocation failed               */
  RABITQ_ECUDA = -3,        /* a CUDA runtime call or kernel failed            */
  RABITQ_ETIMEOUT = -4,     /* a bounded device wait expired                  */
  RABITQ_EIO = -5,          /* file missing, truncated or corrupt             */
  RABITQ_EUNSUPPORTED = -6, /* option not supported on this device/build      */
  RABITQ_EOVERFLOW = -7,    /* a query's candidate list exceeded its capacity */
  RABITQ_EBUSY = -8         /* a server refused a request: budget exhausted   */
} rabitq_status;

/* Precision of the query rotation P^{-1} q (§3.3 of the paper). FP32 is the
 * canonical, bit-reproducible path; TF32 and BF16 run on tensor cores with
 * FP32 accumulation. */
enum { RABITQ_ROT_FP32 = 0, RABITQ_ROT_TF32 = 1, RABITQ_ROT_BF16 = 2 };

/* Similarity of an index (fixed at build). L2: squared Euclidean distance,
 * the paper's setting. IP: inner product, by the decomposition of the
 * paper's closing footnote (§6): <o_r, q_r> = ||o_r - c|| ||q_r - c|| <o, q>
 * + <o_r - c, c> + <q_r, c>, where <o, q> of the unit residuals is estimated
 * exactly as for distances (same code, same bound, halved). COSINE: the
 * inner product of unit vectors (data normalized at build, queries at
 * search). IP and COSINE probe the clusters with the largest <q_r, c>. */
enum { RABITQ_METRIC_L2 = 0, RABITQ_METRIC_IP = 1, RABITQ_METRIC_COSINE = 2 };

/* Bucket-scan implementation of <x_b, q_u> (§3.3.2): bit-plane popcount or
 * an exact integer product on tensor cores; AUTO picks per shape. */
enum { RABITQ_SCAN_AUTO = 0, RABITQ_SCAN_POPC = 1, RABITQ_SCAN_TC = 2 };

/* Work layout of the popcount scan: one CTA (8 warps) per query, or one warp
 * per query (no block barriers; D' of 128 or 256, B_q = 4, k <= 128 and
 * batches large enough to fill the GPU; other searches use the CTA layout).
 * AUTO follows rabitq_autotune's choice, else the warp layout where it
 * applies. Results are identical in every layout. */
enum { RABITQ_LAYOUT_AUTO = 0, RABITQ_LAYOUT_CTA = 1, RABITQ_LAYOUT_WARP = 2 };

/* Staging of the CTA layout's scan rounds (D' of 128 or 256, B_q = 4): each
 * round's codes and factors are copied into shared memory by the bulk-copy
 * (TMA) engine while the block evaluates the round before (BULK), or loaded
 * by every thread on its own (OFF). AUTO follows rabitq_autotune_tiles'
 * choice, else OFF (the faster of the two on the shapes measured). Results
 * are identical either way. */
enum { RABITQ_STAGING_AUTO = 0, RABITQ_STAGING_OFF = 1, RABITQ_STAGING_BULK = 2 };

typedef struct {
  int32_t kmeans_iters;     /* Lloyd iterations (default 10)                    */
  int64_t kmeans_sample;    /* train k-means on about this many points, 0 = all */
  int32_t code_bits;        /* D' (multiple of 64, >= d); 0 = ceil(d/64)*64     */
  int32_t data_on_device;   /* `data` is a device pointer                       */
  void* stream;             /* cudaStream_t to run on; NULL = the legacy stream */
  const float* centroids;   /* optional K x d centroids (host or device, as
                               `data`); when given, k-means is skipped          */
  int32_t metric;           /* RABITQ_METRIC_* (default L2)                     */
} rabitq_build_opts;

typedef struct {
  int32_t rot_precision;    /* RABITQ_ROT_*                                      */
  int32_t scan_path;        /* RABITQ_SCAN_*                                     */
  uint64_t quant_seed;      /* seed of the randomized query rounding (default 3) */
  int32_t io_on_device;     /* queries and outputs are device pointers           */
  void* stream;             /* cudaStream_t; NULL = the legacy default stream    */
  const int32_t* per_query_nprobe; /* optional nq probe counts (same memory kind
                               as the queries), each clamped to [1, nprobe]      */
  int32_t max_candidates;   /* per-query capacity of the candidate list that
                               survives the error bound, 4096..2^26 (0 = 65536) */
  int32_t collect_stats;    /* record per-stage device times (rabitq_last_stats) */
  int32_t scan_layout;      /* RABITQ_LAYOUT_* of the popcount scan (default AUTO) */
  int32_t lane_pairs;       /* codes per lane per step in the warp layout: 1 or 2;
                               0 = the tuned or default value                    */
  int32_t scan_staging;     /* RABITQ_STAGING_* of the CTA layout (default AUTO) */
} rabitq_search_opts;

/* Fill the option structs with their defaults. */
void rabitq_build_opts_default(rabitq_build_opts* opts);
void rabitq_search_opts_default(rabitq_search_opts* opts);

/*
 * rabitq_build -- index phase (Alg. 1 of the paper with the IVF of §4).
 *   data        n x d float32 raw vectors o_r
 *   n, d        n >= 1, 1 <= d <= 4096
 *   n_clusters  K, 1 <= K <= n, K <= 65536: IVF k-means clusters; each
 *               vector is normalized by its own centroid c (§3.1.1)
 *   seed        seeds the k-means initialization and the random orthogonal
 *               matrix P (§3.1.2); the whole build is deterministic
 *   opts        NULL = defaults
 *   out         receives the new index
 * Produces the centroids, P (D' x D', FP64, row-major; the code of o is the
 * sign vector of P^{-1}(o_r - c), §3.1.3), the packed D'-bit codes and the
 * factors ||o_r - c|| and <o_bar, o> (Alg. 1 line 4).
 * Errors: EINVAL on bad sizes or a non-finite input; ENOMEM; ECUDA.
 */
int rabitq_build(const float* data, int64_t n, int32_t d, int32_t n_clusters, uint64_t seed,
                 const rabitq_build_opts* opts, rabitq_index** out);

/*
 * rabitq_search -- query phase (Alg. 2 with the IVF probing and error-bound
 * re-ranking of §4).
 *   queries   nq x d float32 raw query vectors q_r
 *   nq        >= 0 (0 is a no-op)
 *   k         1..1024 neighbours per query
 *   nprobe    1..min(K, 16384) buckets probed per query (the nearest centroids)
 *   bq        1..8 bits of the randomized query quantization (§3.3.1)
 *   eps0      >= 0, confidence parameter of the error bound (Theorem 3.2)
 *   out_ids   nq x k int64 ids, ascending by (distance, id); -1 pads
 *   out_dist  nq x k float32 exact squared distances; +inf pads. For the
 *             IP / COSINE metrics: exact inner products (cosines), ids
 *             descending by (value, then ascending id); -inf pads. The
 *             search ranks by the score -<o_r, q_r> with the same bounds
 *             and re-ranking rule.
 * Re-ranking (§4, order-independent form): tau_ub is the k-th smallest upper
 * bound over all estimated codes; among the codes whose distance lower bound
 * is at most tau_ub, the 4k with the smallest estimated distances (the pilot,
 * ties by id) get exact distances first; tau1 is the k-th smallest of those;
 * every other code is re-ranked iff its lower bound is at most
 * min(tau_ub, tau1).
 * Errors: EINVAL (also for a non-finite query value, found during the search:
 * the outputs are then undefined; and when the current device is not the one
 * the index lives on); ENOMEM; ECUDA; EOVERFLOW when more than max_candidates
 * codes of one query pass the bound (raise max_candidates).
 */
int rabitq_search(const rabitq_index* idx, const float* queries, int64_t nq, int32_t k,
                  int32_t nprobe, int32_t bq, float eps0, int64_t* out_ids, float* out_dist,
                  const rabitq_search_opts* opts);

/*
 * rabitq_search_trace -- rabitq_search that also writes the intermediates of
 * every stage, for staged verification. All pointers are DEVICE memory (the
 * queries and outputs too); any trace pointer may be NULL to skip it.
 *   probe_ids, probe_dist  nq x nprobe: probed clusters by (score, id)
 *                          and the score ||q_r - c||^2 (IP / COSINE:
 *                          -<q_r, c>)
 *   rq                     nq x D': P^{-1} [q_r; 0]
 *   planes                 nq x nprobe x bq x (D'/64) bit-planes of q_u
 *   sum_qu                 nq x nprobe: sum of q_u
 *   meta                   nq x nprobe x 4: Delta/sqrt(D'), v_l/sqrt(D'),
 *                          ||q_r-c|| 2 eps0/sqrt(D'-1), and the estimator's
 *                          additive term ||q_r-c||^2 (IP / COSINE: -<q_r, c>)
 *   pair_cap               per-query capacity of the pair arrays
 *   n_pairs                nq: codes estimated per query
 *   pair_id, pair_ip       nq x pair_cap: id and <x_b, q_u> per pair, in
 *                          probe order then bucket order (ascending id)
 *   pair_est               nq x pair_cap x 3: estimated distance, LB, UB
 *                          (IP / COSINE: of the score -<o_r, q_r>)
 *   tau_ub                 nq: k-th smallest UB (+inf if fewer than k codes)
 *   tau1                   nq: k-th smallest exact distance among the pilot,
 *                          the 4k codes with the smallest estimates among
 *                          those with LB <= tau_ub (+inf if fewer than k)
 *   tau                    nq: min(tau_ub, tau1), the drop threshold
 *   surv_cap, n_surv, surv_ids  the re-rank set (pilot plus every code with
 *                          LB <= tau), in no particular order
 */
typedef struct {
  int32_t* probe_ids;
  float* probe_dist;
  float* rq;
  uint64_t* planes;
  int32_t* sum_qu;
  float* meta;
  int32_t pair_cap;
  int32_t* n_pairs;
  int32_t* pair_id;
  int32_t* pair_ip;
  float* pair_est;
  float* tau_ub;
  float* tau1;
  float* tau;
  int32_t surv_cap;
  int32_t* n_surv;
  int32_t* surv_ids;
} rabitq_trace;

int rabitq_search_trace(const rabitq_index* idx, const float* queries, int64_t nq, int32_t k,
                        int32_t nprobe, int32_t bq, float eps0, int64_t* out_ids,
                        float* out_dist, const rabitq_search_opts* opts,
                        const rabitq_trace* trace);

/*
 * rabitq_search_noalloc -- rabitq_search that allocates no memory, for callers
 * that cannot allocate when they search: a serving process whose own allocator
 * already holds the GPU's free memory, a latency-critical path that must not
 * pay an allocation, a host that forbids allocation after start-up. The paper
 * has no counterpart; this is a library convenience.
 * Arguments and results are those of rabitq_search, except that queries,
 * out_ids, out_dist and opts->per_query_nprobe must be DEVICE pointers
 * (io_on_device is implied), no trace or stats are produced, and only the
 * FP32 rotation and popcount scan are available.
 * Scratch: one fixed 64 MiB device array inside the library (every GPU that
 * loads the library holds it until exit); queries are processed in chunks
 * that fit it. The candidate capacity is min(max_candidates, what fits); a
 * query whose candidates do not fit returns EOVERFLOW. The first call on a
 * device looks up the array's device address with that device current; make
 * that first call before any stream capture. All calls share the array:
 * calls that overlap on the GPU race. Errors: those of rabitq_search
 * (including EINVAL for a non-finite query value, read with the call's own
 * completion wait, and for a current device other than the index's), plus
 * EINVAL for host pointers or for a K so large that one query's centroid
 * distances do not fit in the scratch.
 */
int rabitq_search_noalloc(const rabitq_index* idx, const float* queries, int64_t nq, int32_t k,
                          int32_t nprobe, int32_t bq, float eps0, int64_t* out_ids,
                          float* out_dist, const rabitq_search_opts* opts);

/*
 * ---- Learned probe count (an extension; the paper uses one fixed nprobe) --
 *
 * A small MLP predicts, per query, how many of the nearest buckets to probe
 * (§4 probes a fixed number). Input: 64 features of the query's 64 smallest
 * query-centroid squared distances d_0 <= ... <= d_63 (ties by bucket id;
 * when K < 64 the last one repeats):
 *     x_0 = d_0 / (d_0 + s0)        (s0 = mean d_0 over the training queries)
 *     x_j = d_0 / d_j  (j >= 1)     (1 when d_j = 0)
 * Network: 64 -> 256 -> ReLU -> 256 -> ReLU -> 1 (y = predicted log2 of the
 * probe count). Weights and biases hold BF16 values; products accumulate in
 * FP32. Probe count of a query: clamp(ceil(mult * 2^y), 1, nprobe_max).
 * Parameters are packed into one vector of RABITQ_MLP_PARAMS floats:
 *   W1 (64 x 256, row-major: z1[n] = sum_j x_j W1[j][n] + b1[n]), b1 (256),
 *   W2 (256 x 256), b2 (256), w3 (256), b3 (1).
 *
 * Labels (the exact method decides them): for a training query with true
 * neighbours g_1..g_k, let r_j be the rank (0-based, buckets ordered by
 * (distance, id)) of the bucket holding g_j, censored at nprobe_max; the
 * label is the probe count R = 1 + the need-th smallest r_j (need =
 * ceil(target_recall * k)), at most nprobe_max, so probing R buckets covers
 * at least `need` of the k neighbours; the regression target is log2 R.
 * Training minimises the mean squared error with Adam (beta1 0.9, beta2
 * 0.999, eps 1e-8, all as FP32 values) on an FP32 master copy that is
 * rounded to BF16 values after every step; mult is then the smallest value on the grid
 * 2^((i - 128)/32), i = 0..511, whose mean coverage over the validation
 * queries (fraction of their k neighbours inside the predicted buckets) is
 * at least target_recall.
 */
enum {
  RABITQ_MLP_IN = 64,
  RABITQ_MLP_HIDDEN = 256,
  RABITQ_MLP_PARAMS = 64 * 256 + 256 + 256 * 256 + 256 + 256 + 1
};

typedef struct {
  int32_t k;              /* neighbours per training query (default 100)       */
  float target_recall;    /* mean recall the multiplier is calibrated for
                             (default 0.95)                                     */
  int32_t nprobe_max;     /* largest predicted probe count; also the probe count
                             of the label search when gt_ids is NULL
                             (0 = min(K, 512))                                   */
  int32_t epochs;         /* passes over the training split (default 30)       */
  int32_t batch;          /* rows per Adam step (default 1024)                 */
  float lr;               /* Adam step size (default 1e-3)                     */
  float val_fraction;     /* the last fraction of the queries is the validation
                             split (default 0.1; at least one query each side)  */
  uint64_t seed;          /* weight initialisation and batch order (default 5) */
  const int64_t* gt_ids;  /* optional nt x k true neighbour ids (-1 = none);
                             NULL = rabitq_search with nprobe_max buckets, Bq 4,
                             eps0 1.9 finds them                               */
  int32_t io_on_device;   /* train_q and gt_ids are device pointers            */
  void* stream;           /* cudaStream_t; NULL = the legacy default stream    */
} rabitq_predictor_opts;

typedef struct {
  int32_t n_clusters, k, nprobe_max;
  float target_recall, s0, mult;
  float train_loss, val_loss;   /* mean squared error of log2 R               */
  float val_recall;             /* mean coverage of the validation split at mult */
  float val_mean_nprobe;        /* mean predicted probe count there            */
  int64_t n_train, n_val;
} rabitq_predictor_info;

void rabitq_predictor_opts_default(rabitq_predictor_opts* opts);

/*
 * rabitq_predictor_train -- labels, training and calibration on the GPU.
 *   idx        the index the predictor serves (its K and centroids)
 *   train_q    nt x d training queries (nt >= 2)
 *   out        receives the new predictor (library-owned until
 *              rabitq_predictor_free)
 * Errors: EINVAL (sizes, k > 1024, target outside (0, 1], non-finite
 * queries); ENOMEM; ECUDA; EOVERFLOW from the label search; EUNSUPPORTED
 * for an IP / COSINE index (the features are sorted centroid distances:
 * learned probe counts, labels, learned searches and plans with a
 * predictor need a RABITQ_METRIC_L2 index).
 */
int rabitq_predictor_train(const rabitq_index* idx, const float* train_q, int64_t nt,
                           const rabitq_predictor_opts* opts, rabitq_predictor** out);

/* A predictor from given parameters (host, RABITQ_MLP_PARAMS floats, each
 * rounded to BF16), feature scale s0 > 0, multiplier mult > 0, for an index
 * of n_clusters buckets. */
int rabitq_predictor_create(const float* params, float s0, float mult, int32_t nprobe_max,
                            int32_t n_clusters, rabitq_predictor** out);
int rabitq_predictor_get_info(const rabitq_predictor* pr, rabitq_predictor_info* out);
/* Copy the parameters (BF16 values as float) to a HOST buffer. */
int rabitq_predictor_get_params(const rabitq_predictor* pr, float* out /* RABITQ_MLP_PARAMS */);
/* Replace the multiplier (e.g. for a recall/speed sweep), mult > 0. */
int rabitq_predictor_set_mult(rabitq_predictor* pr, float mult);
void rabitq_predictor_free(rabitq_predictor* pr);

/*
 * rabitq_predict_nprobe -- per-query probe counts (and optionally the
 * features, nq x 64, and the network outputs y, nq) of nq queries. Memory
 * kind of queries and outputs per opts->io_on_device; opts->stream used.
 */
int rabitq_predict_nprobe(const rabitq_index* idx, const rabitq_predictor* pr,
                          const float* queries, int64_t nq, int32_t* out_nprobe,
                          float* out_features, float* out_y, const rabitq_search_opts* opts);

/*
 * rabitq_search_learned -- rabitq_search with each query's probe count from
 * the predictor (computed inside the search from the same query-centroid
 * distances). The result equals rabitq_search with nprobe = nprobe_max and
 * per_query_nprobe = rabitq_predict_nprobe's output. opts->per_query_nprobe
 * must be NULL. Errors: those of rabitq_search; EINVAL when the predictor
 * was made for another K.
 */
int rabitq_search_learned(const rabitq_index* idx, const rabitq_predictor* pr,
                          const float* queries, int64_t nq, int32_t k, int32_t bq, float eps0,
                          int64_t* out_ids, float* out_dist, const rabitq_search_opts* opts);

/*
 * rabitq_compute_labels -- the labels above for nq queries with given true
 * neighbours (host buffers): ranks (nq x k, r_j censored at nprobe_max, in
 * the order of gt_ids) and label_r (nq, the probe count R).
 */
int rabitq_compute_labels(const rabitq_index* idx, const float* queries, int64_t nq,
                          const int64_t* gt_ids, int32_t k, float target_recall,
                          int32_t nprobe_max, int32_t* ranks, int32_t* label_r);

/*
 * rabitq_mlp_grad -- one forward and backward pass of the network on the
 * GPU, host buffers: params (RABITQ_MLP_PARAMS), X (B x 64), t (B). Writes
 * y (B, may be NULL), the gradient of mean((y - t)^2) with respect to every
 * parameter (grads, packed like params, may be NULL) and that loss (may be
 * NULL). For gradient checks and for inspecting a trained network.
 */
int rabitq_mlp_grad(const float* params, const float* X, const float* t, int64_t B, float* y,
                    float* grads, float* loss);

/*
 * rabitq_mlp_adam -- one Adam step (step >= 1) of the training update on the
 * GPU, host buffers of RABITQ_MLP_PARAMS floats: master, m1, m2 are updated
 * in place; work receives the master rounded to BF16 values.
 */
int rabitq_mlp_adam(float* master, float* m1, float* m2, const float* grads, int32_t step,
                    float lr, float* work);

/*
 * rabitq_autotune -- time the popcount scan (RABITQ_SCAN_POPC) and the
 * tensor-core scan (RABITQ_SCAN_TC) on a sample of queries at the given
 * search parameters, best of `reps` (>= 1) runs each after one warm-up run,
 * and make the faster one the path RABITQ_SCAN_AUTO takes on this index from
 * then on (both give identical results). A tensor-core run that overflows
 * its candidate lists counts as infinitely slow. opts as for rabitq_search
 * (scan_path is ignored). chosen (may be NULL) receives the path; times_ms
 * (may be NULL, 2 entries) the best times {popcount, tensor-core}, -1 for a
 * path that failed. Not thread-safe against searches on the same index.
 */
int rabitq_autotune(rabitq_index* idx, const float* queries, int64_t nq, int32_t k,
                    int32_t nprobe, int32_t bq, float eps0, int32_t reps,
                    const rabitq_search_opts* opts, int32_t* chosen, float* times_ms);

/*
 * rabitq_autotune_tiles -- the batched scheduler's tile autotuner: time every
 * work decomposition of the scan on a sample of queries at the given search
 * parameters and cache the fastest for this index and shape, where the AUTO
 * options (scan_path, scan_layout, lane_pairs) of later searches and plans
 * with a k and nprobe in the same class find it (classes: k <= 16, <= 64,
 * <= 128, larger; nprobe <= 16, <= 64, <= 256, larger). The candidates:
 *   {POPC, CTA, OFF | BULK}  one CTA (8 warps) per query, pairs in rounds
 *                            with a block-wide running threshold; each
 *                            round's codes loaded by the threads (rounds of
 *                            512) or staged by bulk copies (rounds of 256;
 *                            D' of 128 or 256, B_q = 4)
 *   {POPC, WARP, 1 or 2}     one warp per query (four queries per CTA), 1 or
 *                            2 codes per lane per step (where the warp layout
 *                            applies: D' of 128 or 256, B_q = 4, k <= 128)
 *   {TC}                     bucket-major tensor-core products (an overflow
 *                            of its lists rules it out)
 * Every candidate returns identical results. AUTO searches take the fastest
 * tile; plans, which run the popcount scan, take the fastest popcount tile.
 * best receives the chosen tile
 * (time_ms its best time); all (may be NULL) receives up to cap candidates,
 * *n_all their count (time_ms -1 for one that could not run). reps >= 1
 * timed runs each after a warm-up run. Not thread-safe against searches on
 * the same index. Errors: those of rabitq_search.
 */
typedef struct {
  int32_t scan_path;   /* RABITQ_SCAN_POPC or RABITQ_SCAN_TC             */
  int32_t scan_layout; /* RABITQ_LAYOUT_CTA or _WARP (popcount path)      */
  int32_t lane_pairs;  /* codes per lane per step (warp layout), else 0   */
  int32_t staging;     /* RABITQ_STAGING_OFF or _BULK (CTA layout)        */
  float time_ms;       /* best measured time of one search of the sample  */
} rabitq_tile;

int rabitq_autotune_tiles(rabitq_index* idx, const float* queries, int64_t nq, int32_t k,
                          int32_t nprobe, int32_t bq, float eps0, int32_t reps,
                          const rabitq_search_opts* opts, rabitq_tile* best, rabitq_tile* all,
                          int32_t cap, int32_t* n_all);

/*
 * ---- Search plans (CUDA-graph replay of a whole search) -------------------
 *
 * rabitq_plan_create -- a search of up to nq_max queries at fixed k, nprobe,
 * bq, eps0 and options (rot_precision, quant_seed, max_candidates; the scan
 * is the popcount path; per_query_nprobe is not supported), optionally with
 * learned probe counts (pr != NULL: nprobe is then pr's nprobe_max). All
 * device memory is allocated here: the plan's query buffer (nq_max x d), its
 * result buffers (nq_max x k ids and distances) and the scratch. The first
 * run of each batch size nq captures the launch sequence of rabitq_search
 * into a CUDA graph; later runs replay it. Results equal rabitq_search's
 * with scan_path RABITQ_SCAN_POPC. The index and predictor must outlive the
 * plan. Errors: those of rabitq_search's arguments; EUNSUPPORTED; ENOMEM.
 */
int rabitq_plan_create(const rabitq_index* idx, const rabitq_predictor* pr, int64_t nq_max,
                       int32_t k, int32_t nprobe, int32_t bq, float eps0,
                       const rabitq_search_opts* opts, rabitq_plan** out);

/* Device pointers of the plan's buffers (owned by the plan; any may be NULL):
 * queries nq_max x d (the input of rabitq_plan_run), ids / dist nq_max x k
 * (its output), nprobe nq_max (the learned probe counts of the last run, or
 * NULL without a predictor). */
int rabitq_plan_buffers(const rabitq_plan* plan, float** queries, int64_t** ids, float** dist,
                        int32_t** nprobe);

/* Search the first nq (0..nq_max) rows of the plan's query buffer into its
 * result buffers: one graph launch on `stream` (a cudaStream_t; NULL = the
 * legacy stream), asynchronous. Runs on one plan must not overlap (they share
 * the scratch): issue them on one stream. Errors of the device work are
 * reported by rabitq_plan_sync. */
int rabitq_plan_run(rabitq_plan* plan, int64_t nq, void* stream);

/* Wait for `stream`; return OK, or the first device error (EOVERFLOW,
 * ETIMEOUT) of the runs since the last rabitq_plan_sync, and clear it. */
int rabitq_plan_sync(rabitq_plan* plan, void* stream);

/* Copy nq queries (host or device memory) into the plan, run it, copy the
 * results out (host or device memory) and sync: the whole round trip on
 * `stream`. With pinned host buffers every copy is asynchronous. */
int rabitq_plan_search(rabitq_plan* plan, const float* queries, int64_t nq, int64_t* out_ids,
                       float* out_dist, void* stream);

/* With opts->collect_stats set at creation, the device times (ms) of the
 * last run's stages: 0 centroid distances, 1 probe selection (+ learned
 * counts), 2 query rotation, 3 order + fused quantize/scan/prune/re-rank --
 * recorded by event nodes inside the graph. Waits for the last run. Returns
 * the number of entries written (0 without collect_stats). */
int rabitq_plan_stats(rabitq_plan* plan, float* ms, int32_t cap);

/* The tile a plan runs (its AUTO options resolved when the plan was made:
 * the index's tuned tile for its shape, else the defaults); time_ms is 0. */
int rabitq_plan_tile(const rabitq_plan* plan, rabitq_tile* out);

/* Release a plan (NULL is a no-op). */
void rabitq_plan_free(rabitq_plan* plan);

/* Per-stage device times (milliseconds) of the last search on this thread
 * with collect_stats set. Stages: 0 centroid distances, 1 probe selection,
 * 2 query rotation, 3 quantize + scan + prune + re-rank, 4 total (including
 * host<->device copies). Returns the number of stages written (<= cap). */
int rabitq_last_stats(float* ms, int32_t cap);

/* The index's RABITQ_METRIC_*. */
int rabitq_index_metric(const rabitq_index* idx, int32_t* metric);

/*
 * rabitq_estimate -- the single-code estimator (§3.3.2, the first case: one
 * query against one code at a time, as a graph index visits its
 * neighbours). For query i and code ids[i m + j] the query is quantized
 * against the code's own cluster c (random stream of query i and cluster c,
 * as in the bucket scan, so the values equal the scan's for the same batch)
 * and the estimator of Theorem 3.2 is evaluated with its bound.
 *   queries  nq x d float32
 *   ids      nq x m int64 data ids; -1 marks an empty slot
 *   bq, eps0 as for rabitq_search; opts: rot_precision, quant_seed,
 *            io_on_device, stream (other fields ignored)
 *   out      nq x m x 3 float32: {estimate, lower bound, upper bound} of the
 *            squared distance, or of <o_r, q_r> for IP / COSINE; an empty
 *            slot gets three NaNs
 * Errors: EINVAL (sizes; an id outside [-1, n) is reported after the call
 * and its slot gets NaNs); ENOMEM; ECUDA.
 */
int rabitq_estimate(const rabitq_index* idx, const float* queries, int64_t nq,
                    const int64_t* ids, int32_t m, int32_t bq, float eps0, float* out,
                    const rabitq_search_opts* opts);

/*
 * ---- Bucket sharding (the IVF's clusters split over GPUs or index pieces) --
 *
 * rabitq_shard_clusters -- assign the K clusters (sizes: points per cluster,
 * e.g. the bucket offsets' differences) to S shards balanced by points:
 * largest cluster first, each to the shard with the fewest points so far
 * (ties to the lower id). shard_of: K shard numbers out; shard_points (may
 * be NULL): S totals out. Host memory. A shard's index is then built from
 * its clusters' points with the global centroids (rabitq_build_opts.
 * centroids) and the build seed: its codes, factors, probe lists and
 * quantization streams are those of the unsharded index (§4's buckets,
 * Alg. 1), and each shard's search keeps every code of the shard that the
 * unsharded search would keep (its tau_ub, the k-th smallest upper bound of
 * fewer codes, is at least the global one). Errors: EINVAL.
 */
int rabitq_shard_clusters(const int32_t* sizes, int32_t K, int32_t S, int32_t* shard_of,
                          int64_t* shard_points);

/*
 * rabitq_merge_topk -- the k-way merge of per-shard results: for each of nq
 * queries, the k best of n_lists lists of k_in (id, value) entries by
 * (distance, id) -- for the IP / COSINE metrics by (-inner product, id),
 * returned largest first -- into nq x k outputs (ids -1 and +inf / -inf pad).
 * All pointers are DEVICE memory: dist and ids are n_lists x nq x k_in,
 * list-major (each list as a search returns it; id -1 = padding); labels
 * (may be NULL, or hold NULL entries) is a device array of n_lists device
 * pointers mapping each list's ids to global ids (ids[...] indexes
 * labels[list]); global ids must be below 2^32 - 1. n_lists * k_in <= 8192,
 * k <= 1024, nq <= 2^31 - 1. Asynchronous on `stream` (no synchronization).
 * Errors: EINVAL; ECUDA.
 */
int rabitq_merge_topk(const float* dist, const int64_t* ids, int32_t n_lists, int64_t nq,
                      int32_t k_in, int32_t k, const int64_t* const* labels, int32_t metric,
                      int64_t* out_ids, float* out_dist, void* stream);

/*
 * ---- Serving runtime (not in the paper: §5 measures one query at a time) --
 *
 * A server holds resident indices and answers requests -- a batch of nq
 * queries for one index and one k -- submitted from any host thread. A
 * worker thread runs the queued requests of one (index, k) together as one
 * search-plan replay of up to max_batch queries (the oldest request first,
 * then every queued request of the same index and k that still fits, in
 * arrival order), and copies each request's results to its host buffers
 * before completing it. Admission is by device memory: a request's queries
 * are copied into a staging pool of mem_budget bytes when it is submitted
 * and stay there until its batch has run; a request that does not fit the
 * free pool is refused with RABITQ_EBUSY (retry or drop it). The indices and
 * predictors must outlive the server; add every index before submitting.
 *   max_batch        queries per batch and per request (default 256)
 *   mem_budget       staging pool bytes (default 64 MiB)
 *   batch_window_us  how long a lone queued request may wait for company
 *                    before it runs (default 0: it runs at once)
 * rabitq_server_add_index: nprobe (1..min(K, 16384)) for a fixed probe count, or a
 *   predictor for learned counts (nprobe then ignored); slot receives the
 *   index's number for rabitq_server_submit.
 * rabitq_server_submit: queries (host, nq x d) are copied before it returns
 *   the ticket; out_ids / out_dist (host, nq x k) must stay valid until the
 *   request completes. Errors: EINVAL, EBUSY, ECUDA.
 * rabitq_server_wait: blocks until the request completes or timeout_s
 *   passes (ETIMEOUT); latency_us (may be NULL) receives the time from
 *   submission to results on the host. A completed ticket is released.
 *   The request's search errors (EOVERFLOW, ETIMEOUT, ...) are returned here.
 * rabitq_server_free: finishes the queued requests, then frees everything.
 */
typedef struct rabitq_server rabitq_server;
typedef struct {
  int32_t max_batch;
  int64_t mem_budget;
  float batch_window_us;
} rabitq_server_opts;
typedef struct {
  int64_t admitted, refused;          /* requests                           */
  int64_t batches;                    /* plan replays run                   */
  int64_t batched_requests, batched_queries;
  int64_t in_flight_bytes, peak_in_flight_bytes;  /* staging pool use     */
} rabitq_server_stats;

void rabitq_server_opts_default(rabitq_server_opts* opts);
int rabitq_server_create(const rabitq_server_opts* opts, rabitq_server** out);
int rabitq_server_add_index(rabitq_server* server, const rabitq_index* idx,
                            const rabitq_predictor* predictor, int32_t nprobe, int32_t bq,
                            float eps0, int32_t* slot);
int rabitq_server_submit(rabitq_server* server, int32_t slot, const float* queries, int64_t nq,
                         int32_t k, int64_t* out_ids, float* out_dist, int64_t* ticket);
int rabitq_server_wait(rabitq_server* server, int64_t ticket, double timeout_s,
                       double* latency_us);
int rabitq_server_get_stats(rabitq_server* server, rabitq_server_stats* out);
void rabitq_server_free(rabitq_server* server);

/* Sizes of an index: n, d, D' (code bits), K. Any pointer may be NULL. */
int rabitq_index_info(const rabitq_index* idx, int64_t* n, int32_t* d, int32_t* d_pad,
                      int32_t* n_clusters);

/* Accessors: copy to caller-owned HOST buffers, original id order. */
int rabitq_get_centroids(const rabitq_index* idx, float* out /* K x d */);
int rabitq_get_rotation(const rabitq_index* idx, double* out /* D' x D', P row-major */);
int rabitq_get_codes(const rabitq_index* idx, uint64_t* out /* n x D'/64; bit i of the
                     code is word i>>6, bit i&63 */);
/* factors: n x 4 = {||o_r-c||^2, 2||o_r-c||/<o_bar,o>,
 * ||o_r-c|| sqrt(1-<o_bar,o>^2)/<o_bar,o>, 2 popcount(code) - D'}; for the
 * IP / COSINE metrics {-<o_r-c, c>, ||o_r-c||/<o_bar,o>,
 * ||o_r-c|| sqrt(1-<o_bar,o>^2)/(2<o_bar,o>), 2 popcount(code) - D'} */
int rabitq_get_factors(const rabitq_index* idx, float* out /* n x 4 */);
int rabitq_get_assign(const rabitq_index* idx, int32_t* cluster /* n */);
/* Bucket layout: offsets (K+1) and the ids of each bucket, ascending. */
int rabitq_get_buckets(const rabitq_index* idx, int32_t* offsets /* K+1 */,
                       int32_t* ids /* n */);

/*
 * rabitq_sample_rotation -- the random orthogonal P of §3.1.2 on its own:
 * a D' x D' matrix of standard Gaussians (Philox4x32-10 keyed by seed,
 * Marsaglia polar method) orthonormalized row by row by Gram-Schmidt
 * (App. B.3), in FP64 on the device. out: D' x D' HOST buffer, row-major.
 */
int rabitq_sample_rotation(uint64_t seed, int32_t d_pad, double* out);

/* Save / load an index (versioned binary with a CRC-32 of the payload).
 * Errors: EIO on a missing, truncated or corrupt file. */
int rabitq_index_save(const rabitq_index* idx, const char* path);
int rabitq_index_load(const char* path, const rabitq_build_opts* opts, rabitq_index** out);

/* Release an index (NULL is a no-op). */
void rabitq_free(rabitq_index* idx);

/* Message of the last failure on the calling thread ("" if none). */
const char* rabitq_last_error(void);

/*
 * rabitq_selftest_wait -- checks, on the current device, the bounded waits
 * that every mbarrier wait of the library's tensor-core kernels uses (a
 * library safeguard; the paper has no counterpart). One small kernel waits
 * `polls` times on an mbarrier that nothing completes and must give up,
 * then waits again while another warp raises the CTA's failure flag and
 * must give up on the flag; the kernel then exits normally, so the context
 * stays usable. Returns OK when both waits gave up; EIO when one did not;
 * EINVAL for polls == 0; ECUDA on a launch or copy failure.
 */
int rabitq_selftest_wait(uint32_t polls);

#ifdef __cplusplus
}
#endif

#endif /* RABITQ_H */
