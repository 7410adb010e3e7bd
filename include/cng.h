/*
 * cng.h -- C ABI of libcng.so: the alpha-convergent neighbourhood graph (alpha-CNG) of
 * arXiv 2510.05975 ("Fast-Convergent Proximity Graphs for Approximate Nearest Neighbor
 * Search"), built and searched on one GB300 GPU (sm_103a).
 *
 * Conventions for every call
 *   - Pointers named *_dev must be device memory of the current CUDA device; pointers named
 *     "host or device" may be either (the library detects which and copies host data itself).
 *   - Arrays are dense, row-major, with the stated element type; ids are int32 point indices.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are asynchronous on
 *     `stream` unless stated; calls that return statistics synchronise `stream` first.
 *   - Every call returns a cng_status.  On failure, cng_last_error() holds a message for the
 *     calling thread.  Invalid arguments are rejected before any kernel is launched.
 *   - Device-side waits are bounded; a wait that runs out reports CNG_E_TIMEOUT instead of
 *     hanging the GPU.
 *   - Distances are Euclidean (L2, Sec. 2.1 metric space).  The canonical distance used for
 *     every exact decision is D(x,y) = sqrt(sum_i (x_i - y_i)^2) in IEEE double, summed in
 *     index order; FP32 decisions closer than a relative band `tie_band` are re-decided with
 *     that canonical distance on the GPU.  Near-ties are counted in the statistics.
 */
#ifndef CNG_H_
#define CNG_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CNG_OK = 0,
  CNG_E_INVAL = -1,       /* bad argument; nothing launched */
  CNG_E_NOMEM = -2,       /* device or host allocation failed */
  CNG_E_CUDA = -3,        /* CUDA runtime / launch error */
  CNG_E_TIMEOUT = -4,     /* a bounded device wait ran out; results are not valid */
  CNG_E_UNSUPPORTED = -5, /* valid input outside this build's limits (message says which) */
  CNG_E_INTERNAL = -6     /* a device-side consistency check failed */
} cng_status;

typedef enum { CNG_L2 = 0, CNG_IP_AS_L2 = 1, CNG_IP = 2 } cng_metric;
typedef enum { CNG_F32 = 0, CNG_F16 = 1 } cng_dtype;
typedef enum {
  CNG_SCREEN_FP32 = 0,  /* FP32 CUDA-core candidate screen (direct differences) */
  CNG_SCREEN_TC = 1,    /* tensor-core screen: FP16 operands fp16(s x), s a power of two (1 for
                           integer data up to 2048 and for f16 input), FP32 accumulate */
  CNG_SCREEN_TC_BF16 = 2 /* tensor-core screen with BF16 operands bf16(x) (f32 input; f16 input
                            stays FP16), FP32 accumulate: 8x coarser rounding, same rate */
} cng_screen;

/*
 * Build parameters.  Paper names in brackets (Alg. 3 inputs):
 *   alpha   [alpha]  pruning parameter of Def. 2 / Eq. 1, > 0
 *   tau     [tau]    pruning parameter of Def. 2 / Eq. 1, >= 0, raw distance units
 *   R       [M]      out-degree bound, 1 <= R <= L, R <= 64
 *   L       [C]      candidate-list size: the exact L nearest points of P \ {p}, L < n, L <= 256
 *   metric           CNG_IP_AS_L2 requires unit-norm rows (|‖x‖ - 1| <= 1e-3) and then uses L2.
 *                    CNG_IP: maximum inner product for rows of any norm, by building the L2
 *                    graph of the augmented rows x' = [x, sqrt(M^2 - |x|^2)] (M^2 = max |x|^2,
 *                    each |x|^2 summed in FP64 in coordinate order, the extra coordinate the
 *                    correctly rounded FP64 root rounded to FP32; d <= 4095).  Searches (and
 *                    traces, stop training) take d-dimensional queries and use q' = [q, 0], so
 *                    |q' - x'|^2 = |q|^2 + M^2 - 2 <q, x>: ids come in decreasing <q, x> and the
 *                    returned distances are |q' - x'|.  The Euclidean graph is the paper's
 *                    (Sec. 2.1); the augmentation is this library's addition.
 *   screen           cng_screen
 *   tie_band         relative band for FP64 re-decision, >= 5e-6 (default 1e-5)
 *   margin           screened list size is L + margin (default 32; clipped to n - 1)
 *   keep_lists       1: keep candidate and phase-2 lists for cng_lists()
 *   connect_L        beam width of the phase-4 connectivity searches (0 = 32; < 0 skips
 *                    phase 4, leaving points of separated clusters unreachable)
 *   input_order      0 (default): the tensor-core screen sweeps the points in a k-d locality
 *                    order, which makes it faster; 1: in input order.  The results are the
 *                    same either way (an engineering option, not in the paper).
 *   adaptive         1: adaptive-pruning (Alg. 4, Sec. 4.2) in phases 2 and 3 instead of the
 *                    fixed alpha: alpha_i = alpha0 + i * dalpha for i = 0, 1, ..,
 *                    round((alpha_max - alpha0) / dalpha); each point keeps the first R points
 *                    of the first S_i with |S_i| >= R / 2 (else of the last S_i).  alpha is then
 *                    unused.  The paper's setting (Sec. 4.4): alpha0 0.9, dalpha 0.05,
 *                    alpha_max 1.6.
 *   alpha0, alpha_max, dalpha   [alpha_0, alpha_max, Delta alpha] of Alg. 4 (adaptive only)
 *   candidates       CNG_CAND_EXACT (0, default): the exact L nearest points of P \ {p};
 *                    CNG_CAND_BEAM (1): the paper's route (Alg. 3 phase 2, Sec. 4.1): the L
 *                    closest points other than p among those visited by a beam search (Alg. 1)
 *                    for p on a K-NN graph G0 from the navigating node, with queue beam_L
 *                    (0 = L + 1; L + 1 <= beam_L <= 256, so L <= 255).  Phases 3 and 4 follow
 *                    as with exact candidates.
 *   knn_K            [K] degree of G0 (0 = 200); L <= knn_K <= 256 and knn_K < n
 *   beam_L           queue of the candidate searches (see candidates)
 *   knn_graph        G0 as device int32 [n][knn_K] (each row's neighbours, -1 padded at its
 *                    end; the paper builds an approximate K-NN graph), or NULL for the exact
 *                    knn_K-NN graph computed by the library's candidate screen
 *   repair_slots     adjacency slots per row for phase-4 edges (0 = 8, at most 64); the row
 *                    stride of the final graph is R + repair_slots
 *   screen_variant   0 (default): the tensor-core screen's pipeline variant (operand stages,
 *                    row-buffer capacity, checkpoint lag) is chosen by the library's
 *                    autotuner, which times the variants on a sample of row blocks the first
 *                    time a problem shape is built in the process; v >= 1 forces variant v - 1
 *                    (fewer than 8 variants; results never depend on the variant)
 */
typedef struct {
  double alpha;
  double tau;
  int32_t R;
  int32_t L;
  int32_t metric;
  int32_t screen;
  double tie_band;
  int32_t margin;
  int32_t keep_lists;
  int32_t connect_L;
  int32_t input_order;
  int32_t adaptive;
  double alpha0;
  double alpha_max;
  double dalpha;
  int32_t candidates;
  int32_t knn_K;
  int32_t beam_L;
  const int32_t *knn_graph;
  int32_t repair_slots;
  int32_t screen_variant;
} cng_build_params;

enum { CNG_CAND_EXACT = 0, CNG_CAND_BEAM = 1 };

/* Per-phase times (device events, milliseconds) and near-tie / certification counts. */
typedef struct {
  double ms_total, ms_prep, ms_entry, ms_screen, ms_rerank, ms_prune, ms_merge, ms_connect;
  int64_t n_edges;            /* edges of the final graph */
  int64_t cert_fail_rows;     /* rows whose screened list could not be certified, rescanned */
  int64_t order_ties;         /* candidate-order near-ties re-decided in FP64 */
  int64_t rule_ties;          /* pruning comparisons re-decided in FP64 */
  int64_t merge_repruned;     /* nodes whose merged list exceeded R and was pruned again */
  int64_t merge_max_list;     /* largest merged candidate set */
  int64_t repair_edges;       /* edges added by phase 4 (connectivity) */
  int32_t repair_rounds;      /* phase-4 rounds */
  int32_t screen_used;        /* cng_screen actually used */
  int32_t entry;              /* navigating node s */
  int32_t exact_int;          /* 1 when every FP32 squared distance is an exact integer */
  double screen_err_max;      /* largest |screened - rerank| seen on kept candidates */
  double ms_order;            /* locality order of the screen's operands (part of ms_total) */
  double alpha_mean;          /* mean alpha of the phase-2 lists (alpha when not adaptive) */
  double ms_cand_search;      /* CNG_CAND_BEAM: the candidate searches on G0 (ms_screen and
                                 ms_rerank then time G0's exact K-NN, when the library builds it) */
  int32_t screen_variant;     /* tensor-core screen: the pipeline variant used, its operand */
  int32_t screen_stages;      /* stages, row-buffer capacity (entries per row) and checkpoint */
  int32_t screen_cap;         /* lag (windows of 256 column tiles); -1 for the FP32 screen */
  int32_t screen_sync;
  int32_t prune_path;         /* phase-2b sweep: 0 float rows (SIMT), 1 8-bit rows (dp4a SIMT),
                                 2 8-bit rows, candidate-pair Gram tile on the tensor cores,
                                 3 FP16 rows, Gram tile with certified decision windows,
                                 4 float rows, all-pairs Gram blocks on CUDA cores */
} cng_build_stats;

typedef struct cng_index cng_index;

/*
 * cng_build -- Alg. 3 (Sec. 4.1, 4.3):
 *   navigating node s = point nearest the centroid (phase 1);
 *   for each p: its L candidates -- the exact L nearest points of P \ {p} by (D, id), or with
 *   CNG_CAND_BEAM the L closest points visited by a beam search for p on G0 -- then Alg. 2
 *   with the rule of Def. 2 (Eq. 1) and the out-degree cut at R (phase 2);
 *   reverse edges from the phase-2 snapshot, each node's merged set pruned once if it
 *   exceeds R, else kept in (D, id) order (phase 3, lazy pruning of Sec. 4.3);
 *   connectivity (phase 4): in rounds, every point p not reachable from s is searched for from
 *   s (Alg. 1, beam connect_L, all connect_L results); its first result r whose row has a free
 *   slot names p.  Points without in-edges get the edge r -> p, a row taking them in ascending
 *   order while it has free slots; in a round where none of them can be linked, each named r
 *   gets an edge to the smallest point naming it.  Rows hold up to R pruned edges plus up to
 *   repair_slots (default 8) such edges.
 * points: host or device, n x d of `dtype`, borrowed for the call only (the index keeps its own
 * device copy).  *out receives a new index owned by the caller (free with cng_free).
 * stats may be NULL.  Synchronises `stream` before returning.
 */
cng_status cng_build(const void *points, int32_t dtype, int64_t n, int32_t d,
                     const cng_build_params *params, void *stream, cng_index **out,
                     cng_build_stats *stats);

/*
 * cng_entry_noalloc -- the navigating node of cng_build (the point nearest the centroid, ties
 * to the smaller id) without allocating any memory, for callers that cannot allocate device
 * memory when they need it: processes whose device memory is owned by another allocator (a
 * framework's caching allocator, a fixed arena) or budgeted at start-up, and latency-bound
 * loops that cannot afford an allocation's implicit synchronisation.  The paper has no
 * counterpart to this call; it is an engineering addition.  The id equals cng_build's entry
 * for CNG_L2 and CNG_IP_AS_L2 builds of the same points; a CNG_IP build takes its entry on the
 * augmented rows [x, sqrt(M^2 - |x|^2)], which this call does not form.
 * points_dev: device, n x d of `dtype`, row-major without padding; entry_dev: device int32
 * receiving the id.  Asynchronous on `stream`; calls no allocator.  Scratch is a fixed 4 MiB
 * device array held by every GPU that loads the library until exit: a call needs
 * ceil(n / 4096) * d + d + 2 doubles of it, at most 524,288 (n <= 16.7 million at d = 128);
 * larger inputs are rejected with CNG_E_INVAL.  The first call on a device looks up the
 * array's address, so make it before any stream capture.  All calls share the array: calls
 * that overlap on the GPU race.
 */
cng_status cng_entry_noalloc(const void *points_dev, int32_t dtype, int64_t n, int32_t d,
                             int32_t *entry_dev, void *stream);

/* Release an index and its device memory.  NULL-safe.  Waits for the index's last search to
 * finish; its search scratch (host staging, deferred-query list) is kept in a small per-process
 * cache (at most 8 buffers) for the next index on the same device. */
void cng_free(cng_index *index);

/* Thread-local message describing the last failure of this thread (never NULL). */
const char *cng_last_error(void);

/*
 * cng_graph -- borrow the final graph: adj_dev [n][stride] int32 (-1 padded, each row in the
 * order the construction produced: phase-3 edges, then phase-4 edges), deg_dev [n] int32,
 * `R` receives the row stride (degree bound + 8), plus the entry point and n.  The pointers
 * stay valid until cng_free.  Any output pointer may be NULL.
 */
cng_status cng_graph(const cng_index *index, const int32_t **adj_dev, const int32_t **deg_dev,
                     int32_t *R, int32_t *entry, int64_t *n);

/*
 * cng_lists -- borrow the intermediate lists kept when keep_lists = 1:
 *   cand_dev  [n][L] int32  exact candidate lists in (D, id) order
 *   cdist_dev [n][L] float  their FP32 distances
 *   fwd_dev   [n][R] int32  phase-2 out-lists (-1 padded), fdeg_dev [n] int32
 * plus L and the degree bound R.  Returns CNG_E_INVAL if the index was built without
 * keep_lists.
 */
cng_status cng_lists(const cng_index *index, const int32_t **cand_dev, const float **cdist_dev,
                     int32_t *L, const int32_t **fwd_dev, const int32_t **fdeg_dev, int32_t *R);

/* ---------------------------------------------------------------------------------------
 * Search (Alg. 1), batched: one persistent launch serves every query.
 * ------------------------------------------------------------------------------------- */

typedef struct cng_stop_model cng_stop_model;

typedef enum { CNG_SEARCH_FIXED = 0, CNG_SEARCH_LEARNED = 1 } cng_search_mode;

/*
 * mode         CNG_SEARCH_FIXED: Alg. 1 exactly (stop when every queue entry is explored);
 *              CNG_SEARCH_LEARNED: additionally stop when the stop model's probability reaches
 *              `threshold` at a check (every `check_every` hops); Alg. 1's own rule remains.
 * min_stable   learned mode: a check consults the model only when the first min(k, |Q|) ids
 *              have not changed for at least this many hops (0 = at every check); the gate is
 *              free, so the network runs only where a stop is plausible
 * model        required for CNG_SEARCH_LEARNED, ignored otherwise
 * max_hops     0 = unbounded; otherwise queries stop after this many hop vertices (flagged)
 * use_graph    1: launch through a CUDA graph cached per index for this exact call: the
 *              query and output pointers, nq, k, L, mode, launch shape and stream all form
 *              its key, so repeated calls on the same buffers replay one graph; at most 16
 *              are kept per index (the oldest is destroyed first)
 * warps_per_block  queries per CTA (one warp each, <= 8); 0 = autotuned: the first search
 *              of an (L, mode) shape on an index of a given shape (device, dtype, padded d,
 *              adjacency row stride) times every launch shape (1, 2, 4, 8 warps per block x
 *              visited filters of 512, 1024, 2048 slots) on up to 16,384 of its queries
 *              (best of two runs) and keeps the fastest for the rest of the process; results
 *              do not depend on it
 */
typedef struct {
  int32_t mode;
  const cng_stop_model *model;
  float threshold;
  int32_t check_every;
  int32_t max_hops;
  int32_t use_graph;
  int32_t warps_per_block;
  int32_t min_stable;
} cng_search_params;

typedef struct {
  double ms;                /* device time of the search launch */
  int64_t ndc_total;        /* distance computations summed over queries */
  int64_t hops_total;       /* hop vertices summed over queries */
  int64_t fp64_decisions;   /* queue-order near-ties re-decided in FP64 */
  int64_t stopped_early;    /* queries stopped by the learned rule */
  int32_t warps_per_block;  /* launch shape used */
  int32_t hash_slots;       /* visited-filter slots per query used */
} cng_search_stats;

/*
 * cng_search -- beam-search(G, q, s, L, k) of Alg. 1 for each of nq queries (f32, n x d,
 * host or device).  Outputs (host or device; ndc/hops/flags may be NULL):
 *   ids [nq][k] int32, dists [nq][k] float (FP32 distances), ndc [nq], hops [nq] int32,
 *   flags [nq] int32 (bit 0: a queue decision was re-decided in FP64; bit 1: max_hops hit;
 *   bit 2: stopped by the learned rule).
 * Requires 1 <= k <= L <= 256.  Ties in the queue order by (D, id).  Returns identical ids to the
 * FP64 definition for fixed-L mode.  stats may be NULL; when given, `stream` is synchronised.
 * The outputs must all be host memory or all device memory (CNG_E_INVAL otherwise).  Calls on
 * one index share its search scratch, so the library orders them on the GPU: a call on a
 * stream other than the previous call's first waits (cudaStreamWaitEvent) for that call.
 */
cng_status cng_search(const cng_index *index, const float *queries, int64_t nq, int32_t k,
                      int32_t L, const cng_search_params *params, int32_t *ids, float *dists,
                      int32_t *ndc, int32_t *hops, int32_t *flags, void *stream,
                      cng_search_stats *stats);

/* ---------------------------------------------------------------------------------------
 * Grid search of tau on held-out queries (Sec. 4.4, parameter configuration: tau = 0 against
 * the coarse values 10, 1, 0.1, 0.01, 0.001, then a finer search around the best).  Every
 * trial builds the graph of `points` with `params` (its tau replaced) and scores it on the
 * nq queries: the smallest beam width L in search_Ls[0 .. n_Ls) (ascending, each >= k) whose
 * mean Recall@k against gt_ids [nq][k] (host, the exact k nearest ids, e.g. from cng_knn)
 * reaches `target`, and the mean number of hop vertices at that width -- a device-independent
 * cost (the paper compares query speed; hops count the search work and do not depend on the
 * machine).  Fine step: with the best coarse value t > 0, t / 2 and 2 t; with t = 0, 0.0005.
 * The best trial has the fewest mean hops among those reaching the target (ties: smaller
 * tau); *best_tau = 0 when none reaches it.  trials [max_trials] receives each trial in the
 * order run (up to 8), *n_trials their count.  Synchronises; the indexes are freed.
 * ------------------------------------------------------------------------------------- */
typedef struct {
  double tau;
  int32_t L;         /* smallest width reaching the target, 0 if none */
  double recall;     /* mean Recall@k at L (at the largest width if none reaches the target) */
  double hops_mean;  /* mean hop vertices per query at that width */
} cng_tau_trial;

cng_status cng_tune_tau(const void *points, int32_t dtype, int64_t n, int32_t d,
                        const cng_build_params *params, const float *queries, int64_t nq,
                        int32_t k, const int32_t *gt_ids, const int32_t *search_Ls, int32_t n_Ls,
                        double target, void *stream, double *best_tau, cng_tau_trial *trials,
                        int32_t max_trials, int32_t *n_trials);

/* ---------------------------------------------------------------------------------------
 * Learned early stop.  Not part of the paper (its search stops only by Alg. 1's rule): a
 * 16 -> 64 -> 64 -> 1 ReLU network reads the state of a search after a hop and predicts whether
 * the top-k result list is already final; the learned search mode stops when the predicted
 * probability reaches a threshold.  Features after hop t (lg = natural log, floored at 1e-30;
 * D0 = entry distance; D1, Dk, DL = distances of the 1st, min(k,|Q|)-th and last queue entry;
 * Du = the hop vertex's distance; Dk_h[j] = Dk after hop j, Dk_h[0] = D0; tlc = last hop at
 * which the first min(k, |Q|) ids changed; U = unexplored entries; ins = this hop's points left
 * in Q; stride = adjacency row stride):
 *   f0 lg D0, f1 ln(1+t), f2 lg D1 - lg D0, f3 lg Dk - lg D0, f4 lg DL - lg D0, f5 lg Du - lg Dk,
 *   f6..f11 lg Dk_h[max(t-j,0)] - lg Dk for j = 1,2,4,8,16,32, f12 ln(1 + t - tlc), f13 U/L,
 *   f14 |Q|/L, f15 ins/stride.
 * Training samples: every hop t <= max_trace of the plain search of each training query, label
 * 1 iff t >= that query's final tlc.  Parameters (flat FP32, CNG_STOP_NPARAMS):
 *   W1[64][16] b1[64] W2[64][64] b2[64] w3[64] b3[1];  inputs standardised by mu[16], sigma[16].
 * Inference runs on the tensor cores with BF16-rounded weights: each activation (standardised
 * input, hidden layer 1) enters as a pair of BF16 values hi + lo (about 16 significant bits),
 * products are exact and sums are FP32, so the logit is the FP64 network's on the rounded
 * weights to within ~1e-5 relative.
 * ------------------------------------------------------------------------------------- */

#define CNG_STOP_NPARAMS 5313

typedef struct {
  int32_t k;          /* result size the model is trained for */
  int32_t L;          /* beam width of the traced searches (and of the learned searches) */
  int32_t max_trace;  /* hops recorded per training query (0 = 256) */
  int32_t epochs;     /* passes over the samples (0 = 4) */
  int32_t batch;      /* minibatch rows (0 = 4096) */
  float lr;           /* Adam learning rate (0 = 1e-3) */
  uint64_t seed;      /* weight initialisation and minibatch draws (counter-based hash) */
} cng_train_params;

typedef struct {
  double ms_trace, ms_train;  /* device time of the traced search and of the training */
  int64_t samples, positives, steps;
  float loss_first, loss_last;  /* mean loss of the first and last minibatch */
} cng_train_stats;

/*
 * cng_stop_train -- trace the plain search of nq training queries (f32 [nq][d], host or
 * device) on `index`, then train the stop network on the GPU (forward, backward and Adam
 * kernels).  *out receives a model owned by the caller (cng_stop_free).  Synchronises.
 */
cng_status cng_stop_train(const cng_index *index, const float *train_queries, int64_t nq,
                          const cng_train_params *params, void *stream, cng_stop_model **out,
                          cng_train_stats *stats);
void cng_stop_free(cng_stop_model *model);
/* Copy the FP32 master parameters [CNG_STOP_NPARAMS] and mu[16], sigma[16] to host memory
 * (any pointer may be NULL).  bf16_params, if not NULL, receives the BF16-rounded parameter
 * values inference uses (as floats, same layout). */
cng_status cng_stop_export(const cng_stop_model *model, float *params, float *mu, float *sigma,
                           float *bf16_params);
/* A model from given host parameters (layout above); for tests and reloading. */
cng_status cng_stop_import(const float *params, const float *mu, const float *sigma,
                           cng_stop_model **out);
/*
 * cng_trace -- the plain search (Alg. 1) of nq device queries recording, for every hop
 * t <= max_trace, the 16 features into feats_dev [nq][max_trace][16] (entries past a query's
 * last hop are left untouched), plus hops_dev [nq], tlc_dev [nq] and ids_dev [nq][k].
 */
cng_status cng_trace(const cng_index *index, const float *queries_dev, int64_t nq, int32_t k,
                     int32_t L, int32_t max_trace, float *feats_dev, int32_t *hops_dev,
                     int32_t *tlc_dev, int32_t *ids_dev, void *stream);
/* Mean loss and its gradient over B standardised rows x_dev [B][16] with labels y_dev [B]
 * (the training kernels, exposed for gradient checks).  Synchronises. */
cng_status cng_mlp_grad(const float *params_dev, const float *x_dev, const float *y_dev,
                        int64_t B, float *grad_dev, float *loss_dev, void *stream);
/* One Adam step (t >= 1) on device arrays of CNG_STOP_NPARAMS floats. */
cng_status cng_mlp_adam(float *params_dev, float *m_dev, float *v_dev, const float *grad_dev,
                        int64_t t, float lr, void *stream);

/* ---------------------------------------------------------------------------------------
 * Exact k-NN (the candidate step of cng_build, exposed for ground truth and tests).
 * ------------------------------------------------------------------------------------- */

/*
 * cng_knn -- for each of m rows, the exact `k` nearest base points by (D, id) (Alg. 3's
 * candidate lists in exact form).  base: n x d f32 device; rows: m x d f32 device, or NULL
 * for rows = base with each row's own id excluded.  ids_dev [m][k] int32, dists_dev [m][k]
 * float.  k <= 256, k <= n (k < n when rows is NULL).  screen: cng_screen.  Synchronises.
 */
cng_status cng_knn(const float *base_dev, int64_t n, const float *rows_dev, int64_t m, int32_t d,
                   int32_t k, int32_t screen, double tie_band, int32_t *ids_dev,
                   float *dists_dev, void *stream, cng_build_stats *stats);

#ifdef __cplusplus
}
#endif
#endif /* CNG_H_ */
