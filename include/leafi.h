/*
 * leafi.h — C ABI of the B300-native LeaFi search path.
 *
 * LeaFi (Wang, Ileana, Palpanas, SIGMOD 2025) adds learned filters to the
 * leaves of a tree-based data-series index (DSTree or iSAX).  Per query the
 * path computes the index's summarisation lower bounds, runs every leaf's MLP
 * filter in one batch, shifts the predictions by the conformal offset for the
 * query's recall target, prunes, and scans the surviving leaves with squared
 * Euclidean distance while keeping the k best-so-far.  The same scan produces
 * the filters' training targets at build time.
 *
 * Conventions shared by every entry point:
 *   - Array arguments may be host or device pointers (classified with
 *     cudaPointerGetAttributes).  Host arrays are staged through the library;
 *     device arrays are used in place on the index's stream.
 *   - The caller owns every buffer passed in; the library owns the index and
 *     everything reachable from it until leafi_free().
 *   - Series and queries are float32, row-major, length m, z-normalised by
 *     the caller (the paper's data is z-normalised; the library does not
 *     re-normalise).
 *   - Distances returned are Euclidean: sqrtf of the canonical squared
 *     distance  acc = 0; for i < m: t = q_i - x_i; acc = fmaf(t, t, acc).
 *     Results are ordered by (distance, original id) ascending; ties go to
 *     the lowest id; missing entries (k > n) are id -1 / +inf.
 *   - On any error nothing is written to the outputs, the status is returned
 *     and leafi_last_error() describes it.  The one exception: a search that
 *     returns LEAFI_ETIMEOUT may already have written some result rows, whose
 *     contents are then unspecified.  No entry point aborts the process.
 *   - Calls on one index are serialised by an internal mutex.
 */
#ifndef LEAFI_H
#define LEAFI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct leafi_index leafi_index;

typedef enum {
  LEAFI_OK = 0,
  LEAFI_EINVAL = 1,      /* bad argument (size, pointer, parameter) */
  LEAFI_ENOMEM = 2,      /* host or device allocation failed */
  LEAFI_ECUDA = 3,       /* a CUDA call failed */
  LEAFI_ETIMEOUT = 4,    /* a bounded device wait gave up */
  LEAFI_ENOTTRAINED = 5, /* filters / auto-tuners needed but absent */
  LEAFI_EINTERNAL = 6,   /* internal consistency check failed */
  LEAFI_EAGAIN = 7       /* serving: admission refused for now (memory budget); retry later */
} leafi_status;

enum { LEAFI_DSTREE = 0, LEAFI_ISAX = 1 };

enum { LEAFI_MAX_K = 128, LEAFI_MAX_KCLASSES = 4 };
/* Filter models: the MLP of Sec. 5.1 (default) and the CNN of the model-type
 * study in Sec. 5.2 (see leafi_set_cnn_filters). */
enum { LEAFI_FILTER_MLP = 0, LEAFI_FILTER_CNN = 1 };
/* Query-time offsets from the auto-tuner tables (Sec. 4.4.2): the certified
 * STEP position (default) or the paper's spline through the table (Steffen's
 * monotone interpolation), see leafi_set_calibration_mode. */
enum { LEAFI_CALIB_STEP = 0, LEAFI_CALIB_STEFFEN = 1 };

/* ------------------------------------------------------------------ */
/* Index building (Sec. 3 "Tree-based indexes"; Alg. 1 input I)        */
/* ------------------------------------------------------------------ */

typedef struct {
  int32_t index_type;           /* LEAFI_DSTREE or LEAFI_ISAX */
  int32_t leaf_capacity;        /* a leaf splits when it holds more series (paper: 10k) */
  int32_t dstree_init_segments; /* DSTree root segmentation: equal segments (4) */
  int32_t isax_segments;        /* iSAX PAA segments w (16); m % w == 0 */
  int32_t isax_card_bits;       /* iSAX full cardinality 2^bits (8) */
  int32_t wave;                 /* leaves taken per query per search wave (1..65536); the
                                   auto-tuner calibrates this same schedule */
  int32_t device;               /* CUDA device ordinal (-1: host-only tree) */
  int32_t scan_path;            /* 0: tensor-core scan (float16 dot products on tcgen05
                                   with a proven error band and a canonical float32
                                   re-check); 1: CUDA-core scan (canonical float32 for
                                   every pair); 2: tensor-core scan on float8 e4m3
                                   operands with a power-of-two scale per series and
                                   per query (kind::f8f6f4; its band is about 140 times
                                   wider than float16's, so far more pairs are
                                   re-checked; m <= 256).  All give identical results. */
  int32_t host_build;           /* 0: the tree is built level by level on the GPU (the
                                   series in id order are copied to the device once);
                                   1: sequential insertion on the host.  Both give the
                                   same tree.  Host-only indexes (device -1) are always
                                   built on the host. */
} leafi_build_params;

/* Build an index over n series of length m.  Copies `series` into
 * leaf-contiguous device storage (16-byte aligned rows) owned by the index.
 * device = -1 builds the tree alone on the host (inspection only: leaf
 * sizes, leaf_of, info); every device entry point then returns LEAFI_EINVAL.
 * Returns LEAFI_EINVAL for n < 1, m < 1, m > 512, bad parameters. */
leafi_status leafi_build(const float* series, int64_t n, int32_t m, const leafi_build_params* p,
                         leafi_index** out);

/* Release everything owned by the index (NULL is accepted). */
void leafi_free(leafi_index* index);

/* Thread-local description of the last error on this thread. */
const char* leafi_last_error(void);

/* Kernels this library has launched in this process (all indexes); a
 * diagnostic for counting device work between two points. */
int64_t leafi_launch_count(void);

/* Diagnostics for failure-detection tests (no counterpart in the paper).
 * leafi_debug_set_lock_tries: attempts a tensor-core scan work item makes at a
 * query's result-list lock before it gives up, sets the error word and lets the
 * call return LEAFI_ETIMEOUT (the kernel still leaves through its normal exits
 * and the index stays usable); 0 exhausts the budget at the first merge that
 * needs the lock, -1 restores the default (65,536 attempts with back-off).
 * Used by k > 1 searches.
 * leafi_debug_fail_allocations: the `after`-th allocation from now (0 = the
 * next one) of a device buffer, or of a host step that gates on it (host tree
 * builds), fails as if memory were exhausted: the call returns LEAFI_ENOMEM
 * without writing its outputs.  -1 disarms; a fired injection disarms itself. */
leafi_status leafi_debug_set_lock_tries(leafi_index* index, int32_t tries);
leafi_status leafi_debug_fail_allocations(int64_t after);

/* Launch all later work of this index on `cuda_stream` (a cudaStream_t);
 * NULL selects the legacy default stream. */
leafi_status leafi_set_stream(leafi_index* index, void* cuda_stream);

typedef struct {
  int64_t n;             /* series */
  int32_t m;             /* length */
  int32_t index_type;
  int32_t n_leaves;
  int32_t n_nodes;
  int32_t wave;
  int32_t n_filters;     /* 0 until filters are set */
  int32_t filters_trained;
  int32_t n_calib;       /* calibration queries behind the auto-tuners (0 = none) */
  int32_t n_kclasses;
  int32_t kclasses[LEAFI_MAX_KCLASSES];
  int64_t device_bytes;  /* device memory held by the index */
  int32_t tensor_scan;   /* 1 if leaf scans run on the tensor cores */
  int32_t scan_row_bytes;/* bytes the leaf scan streams per series (fp16 row or fp32 row) */
  double calib_confidence;/* see leafi_set_calibration_confidence */
  int32_t filter_model;  /* LEAFI_FILTER_MLP or LEAFI_FILTER_CNN */
  int32_t filter_width;  /* MLP hidden width h, or CNN channels C */
  int32_t wave_exact;    /* wave width of calls without filtered queries (`wave`: with) */
  int32_t items_per_sm;  /* leaf-scan work items per SM a round aims at (leafi_set_scan_part) */
} leafi_index_info;

leafi_status leafi_get_info(const leafi_index* index, leafi_index_info* info);

/* Per-kernel device time, measured with CUDA events on the index's stream
 * around each launch while profiling is on (off by default; switching it
 * resets the totals).  Kinds: 0 leaf scan, 1 candidate merge, 2 bounds and
 * routes, 3 (reserved), 4 filter forward, 5 wave select.  `level`: 0 off,
 * 1 leaf-scan launches only (the cheapest, for timing a run), 2 every kind
 * plus the tensor-core scan's phase counters. */
enum { LEAFI_KERNEL_KINDS = 6 };
leafi_status leafi_set_profiling(leafi_index* index, int32_t level);
leafi_status leafi_get_kernel_times(leafi_index* index, double* ms /* [6] */,
                                    int64_t* launches /* [6] */);
/* Tensor-core scan phase cycles summed over blocks while profiling is on: 0 item set-up, 1 wait for an accumulator, 2 epilogue, 3 flush
 * and emit (epilogue warp 0, lane 0); 4 wait for a free stage, 11 TMA issue
 * (the TMA thread); 5 wait for the query tile, 6 wait for a TMA load, 7 wait
 * for a free accumulator, 14 MMA issue, 8 commits (the MMA thread); 12 wait for a free
 * query tile, 13 gather (the query loader); 9 work items, 10 chunks read by
 * epilogue warp 0; 15 epilogue warp 0's cycles from kernel entry to exit;
 * then the launch timeline in ns of the global timer, summed over launches:
 * 16 first block start to last block end, 17 first to last block start, 18
 * first to last block end, 19 launches (20 doubles in all). */
leafi_status leafi_get_scan_phases(leafi_index* index, double* cycles);
/* Series per leaf (host array of n_leaves). Leaves are numbered depth-first,
 * left child first. */
leafi_status leafi_leaf_sizes(const leafi_index* index, int64_t* sizes);
/* Leaf of every series, by original id (host array of n). */
leafi_status leafi_leaf_of(const leafi_index* index, int32_t* leaf_of);

/* ------------------------------------------------------------------ */
/* Lower bounds and routing (Sec. 3; Alg. 2's bound test)             */
/* ------------------------------------------------------------------ */

/* Squared leaf lower bounds LB^2 (nq x n_leaves, row-major, float64 arrays
 * holding float32 values): DSTree: max over the root-to-leaf path of
 * sum_r l_r (gap(mu_q,r)^2 + gap(sigma_q,r)^2) against each node's mean /
 * sigma ranges; iSAX: MINDIST^2 of the leaf's word.  Segment statistics and
 * PAA values come from float64 prefix sums; the gaps, products and sums are
 * float32, each statistic taken as the two floats around it and each range
 * end and breakpoint rounded outward, so a gap never exceeds its float64
 * value. */
leafi_status leafi_leaf_lower_bounds(leafi_index* index, const float* queries, int64_t nq,
                                     double* lb2);
/* Leaf that each query's own summary routes to (int32, nq). */
leafi_status leafi_route(leafi_index* index, const float* queries, int64_t nq, int32_t* leaf);

/* Same bounds as leafi_leaf_lower_bounds, computed without allocating any
 * device memory.  The paper has no counterpart: this is a library facility for
 * callers that cannot call cudaMalloc -- a program whose GPU memory is reserved
 * up front by another allocator (a framework's caching pool that owns the
 * device), or a latency-critical loop that cannot take cudaMalloc's implicit
 * device-wide synchronisation.  queries [nq][m] float32 and lb2 [nq][n_leaves]
 * float64 must be device (or managed) arrays on the index's GPU; anything else
 * is LEAFI_EINVAL before any launch.  The shapes cannot be checked here: the
 * caller guarantees them.  The work is queued on the index's stream and the
 * call returns without synchronising.  Scratch is one static device array of
 * 16 MiB per GPU, held until the process exits; requests that need more
 * (roughly nq*(2m+2) + nq*(4*intervals + nodes) doubles for a DSTree,
 * nq*(2m+2) + nq*2w for iSAX) are rejected with LEAFI_EINVAL naming the
 * largest nq that fits.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress), so
 * make it before any stream capture.  Every call shares the array and keeps
 * nothing from the previous one (each scratch word read is written earlier in
 * the same call): calls that overlap on the GPU race. */
leafi_status leafi_leaf_lower_bounds_noalloc(leafi_index* index, const float* queries,
                                             int64_t nq, double* lb2);

/* ------------------------------------------------------------------ */
/* Learned filters (Sec. 4 intro; Sec. 5.1: MLP m -> h -> 1, ReLU)      */
/* ------------------------------------------------------------------ */

/* Filtered leaves = the n_filters largest leaves (ties: lower leaf id), the
 * greedy selection of Alg. 3 with threshold th = 0 (out: int32 [n_filters]). */
leafi_status leafi_select_leaves(const leafi_index* index, int32_t n_filters,
                                 int32_t* filter_leaf);
/* Leaf selection of Alg. 3 with this device's costs: t^F = time of one
 * (query, filter) prediction in the batched forward, t^S = time of one
 * (query, series) distance in the batched leaf scan, both measured here on
 * probe batches of 256 of the index's own series (probe filters of hidden
 * width `hidden`, 0 = m, with zero weights); threshold th = a t^F / t^S; w =
 * device bytes of one filter (weights, the tensor-core forward's tf32
 * planes, one auto-tuner column of 300 offsets).  Leaves by non-increasing
 * size (ties: lower id) are taken while size >= th and w^M + w <= mem_cap.
 * filter_leaf (host) needs room for n_leaves entries; report (nullable)
 * returns the measured costs, th, w and the count.  Does not change the
 * index's filters. */
typedef struct {
  double a;         /* 1 / p^F, the expected filter pruning ratio's inverse (2 in the paper) */
  int64_t mem_cap;  /* c^M: device bytes available to filters */
  int32_t hidden;   /* hidden width (MLP) or channels (CNN) of the filters to come (0 = m) */
  int32_t model;    /* LEAFI_FILTER_MLP or LEAFI_FILTER_CNN: whose forward t^F times */
} leafi_select_params;
typedef struct {
  double t_filter_s;     /* t^F */
  double t_series_s;     /* t^S */
  double threshold;      /* th = a t^F / t^S (series) */
  double filter_bytes;   /* w */
  int32_t n_selected;
} leafi_select_report;
leafi_status leafi_select_leaves_auto(leafi_index* index, const leafi_select_params* params,
                                      int32_t* filter_leaf, leafi_select_report* report);

/* Install F filters on the given leaves with weights W1 [F][h][m], b1 [F][h],
 * w2 [F][h], b2 [F] (float32; h = hidden width).  Clears the auto-tuners. */
leafi_status leafi_set_filters(leafi_index* index, const int32_t* filter_leaf, int32_t F,
                               int32_t h, const float* W1, const float* b1, const float* w2,
                               const float* b2);
/* CNN filters (Sec. 5.2, model-type study: two convolutional layers, kernel
 * size 3, latent channels C = m).  Readings of what the paper leaves open: one
 * input channel; stride 1 and zero padding 1, so every layer keeps length m;
 * bias and ReLU after both convolutions; each channel averaged over the m
 * positions, then a linear layer C -> 1 without activation predicting the
 * Euclidean d^L.  Parameters of one filter, flat float32, P =
 * leafi_cnn_params(C) = 3C^2 + 6C + 1 values: w1 [C][3], b1 [C], w2 [C][C][3]
 * (output channel, input channel, tap; tap t meets position i + t - 1), b2
 * [C], wo [C], bo.  theta [F][P], host or device.  LEAFI_EINVAL when the
 * activations of one query (3 planes of C x (m + 2) floats for training) do
 * not fit the device's shared memory (C = m up to about 128).  Installing
 * clears the auto-tuners. */
int64_t leafi_cnn_params(int32_t C);
leafi_status leafi_set_cnn_filters(leafi_index* index, const int32_t* filter_leaf, int32_t F,
                                   int32_t C, const float* theta);
/* Copy the CNN parameters out (theta [F][P]); LEAFI_EINVAL for MLP filters. */
leafi_status leafi_get_cnn_filters(leafi_index* index, float* theta);
/* Initial CNN parameters of F filters of C channels (Philox draws, U(-a, a)
 * with a = 1/sqrt(fan in): 3 for w1/b1, 3C for w2/b2, C for wo/bo). */
leafi_status leafi_initial_cnn_weights(leafi_index* index, int32_t F, int32_t C, uint64_t seed,
                                       float* theta);
/* The filtered leaves, filter by filter (int32 [n_filters], host). */
leafi_status leafi_get_filter_leaves(const leafi_index* index, int32_t* filter_leaf);
/* Copy the current MLP filter weights out (same layouts as leafi_set_filters;
 * LEAFI_EINVAL for CNN filters). */
leafi_status leafi_get_filters(leafi_index* index, float* W1, float* b1, float* w2, float* b2);
/* d^f(q, M_f) for every query and filter (float32, nq x F), either model. */
leafi_status leafi_filter_predict(leafi_index* index, const float* queries, int64_t nq,
                                  float* out);

/* ------------------------------------------------------------------ */
/* Training data: node-wise nearest-neighbour distances (Sec. 3 d^L;    */
/* Alg. 1 SearchGlobalQueries / SearchLocalQueries)                    */
/* ------------------------------------------------------------------ */

/* For every query i and every j < nl: the k best (d^2, id) inside leaf
 * leaves[i*nl+j] (-1 = skip), written to d2/ids [nq][nl][k] (squared
 * canonical distances, float32; ids int64; padding +inf / -1). */
leafi_status leafi_leaf_knn(leafi_index* index, const float* queries, int64_t nq,
                            const int32_t* leaves, int32_t nl, int32_t k, float* d2,
                            int64_t* ids);
/* Training targets d^L (Euclidean float32): Tg [ng][F] for global queries
 * against every filtered leaf, Tl [F][nl] for the nl local queries of each
 * filter (Ql [F][nl][m]) against its own leaf. */
leafi_status leafi_train_targets(leafi_index* index, const float* Qg, int64_t ng,
                                 const float* Ql, int64_t nl, float* Tg, float* Tl);

/* LeaFi-enhanced index building, Alg. 1 end to end: select the
 * filtered leaves (Alg. 3), generate the global and local training queries,
 * compute their targets d^L, train every filter by SGD and fit the auto-tuners
 * on the calibration set.  Every random draw (which series a query comes from,
 * its noise, the initial weights, the epoch shuffles) is taken from the
 * library's counter-based generator (Philox4x32-10) under `seed`, so a build is
 * reproducible bit for bit on the same device. */
typedef struct {
  int32_t n_filters;        /* > 0: the n_filters largest leaves (Alg. 3 with th = 0);
                               -1: Alg. 3 with this device's measured t^F, t^S (a, mem_cap) */
  double a;                 /* Alg. 3: 1 / p^F (2 in the paper) */
  int64_t mem_cap;          /* Alg. 3: device bytes available to filters */
  int32_t hidden;           /* hidden width h (0 = m, Sec. 5.1) */
  int32_t n_train;          /* training queries per filter, global + local (2000) */
  double global_local_ratio;/* global : local (3 -> 1500 global, 500 local per leaf);
                               +inf: global queries only (the ablation without local data) */
  double val_frac;          /* validation share of both kinds (0.2); the global validation
                               queries are the calibration set of Alg. 4 */
  double noise_lo, noise_hi;/* per-query noise sigma ~ U[noise_lo, noise_hi] (0.1, 0.4) */
  int32_t batch;            /* SGD minibatch (64) */
  int32_t max_epochs;       /* (1000) */
  int32_t patience;         /* epochs without a lower validation loss before lr /= 10 (10) */
  double lr0, lr_min;       /* 0.01, 1e-5 */
  int32_t n_kclasses;       /* auto-tuner k-classes, ascending, 1..LEAFI_MAX_KCLASSES */
  int32_t kclasses[LEAFI_MAX_KCLASSES];
  uint64_t seed;
  double confidence;        /* calibration confidence of the search's offsets (0.95; see
                               leafi_set_calibration_confidence) */
  int32_t tune_search;      /* 1: leafi_tune_search picks the wave width and work-item
                               balance of exact searches, then, after the auto-tuners
                               are fitted, those of LeaFi searches at target 0.99 (its
                               defaults; the tables are refitted for the chosen width) */
  int32_t model;            /* LEAFI_FILTER_MLP (Sec. 5.1) or LEAFI_FILTER_CNN (Sec. 5.2;
                               `hidden` is then the channel count C, 0 = m) */
  int32_t calib_mode;       /* LEAFI_CALIB_STEP (default) or LEAFI_CALIB_STEFFEN, installed
                               with the tables (leafi_set_calibration_mode) */
} leafi_train_params;

typedef struct {
  int32_t n_filters;                      /* filters installed */
  int32_t n_gtrain, n_gval, n_ltrain, n_lval;
  double select_threshold;                /* Alg. 3's th (series) when n_filters = -1, else 0 */
  double seconds_select, seconds_generate, seconds_train, seconds_calibrate;
} leafi_train_report;

/* Alg. 1 on the index (the index's previous filters and auto-tuners are
 * replaced).  Counts: n_global = round(n_train * r / (r + 1)), n_local =
 * n_train - n_global, validation = round(val_frac * count) of each kind
 * (n_gval >= 1).  epochs_run / best_val (nullable host arrays with room for
 * n_leaves entries) receive each filter's epochs and best validation loss.
 * LEAFI_EINVAL for bad parameters (nothing is changed). */
leafi_status leafi_train_filters(leafi_index* index, const leafi_train_params* params,
                                 int32_t* epochs_run, double* best_val,
                                 leafi_train_report* report);

/* Inspection exports of Alg. 1's draws, for parity checks.  The training
 * queries leafi_train_filters generates for the filtered leaves filter_leaf[F]:
 * Qg [n_global][m], Ql [F][n_local][m] (float32, host or device) and, nullable,
 * the original ids they come from, gpick [n_global], lpick [F][n_local]. */
leafi_status leafi_training_queries(leafi_index* index, const leafi_train_params* params,
                                    const int32_t* filter_leaf, int32_t F, float* Qg, float* Ql,
                                    int64_t* gpick, int64_t* lpick);
/* Initial weights of F filters of width h (layouts of leafi_set_filters). */
leafi_status leafi_initial_weights(leafi_index* index, int32_t F, int32_t h, uint64_t seed,
                                   float* W1, float* b1, float* w2, float* b2);
/* The SGD shuffles: int32 [epochs][n], each row a permutation of [0, n). */
leafi_status leafi_epoch_permutations(int32_t epochs, int32_t n, uint64_t seed, int32_t* perms);

/* SGD parameters of leafi_train_filters_on. */
typedef struct {
  int32_t n_gtrain, n_gval; /* global queries: first n_gtrain train, next n_gval validate */
  int32_t n_ltrain, n_lval; /* local queries per filter, same split */
  int32_t batch;            /* SGD minibatch */
  int32_t max_epochs;       /* <= 1000 in the paper */
  int32_t patience;         /* epochs without a lower validation loss before lr /= 10 */
  double lr0, lr_min;       /* 0.01 and 1e-5 in the paper */
} leafi_sgd_params;

/* Alg. 1's target collection and training on queries the caller supplies
 * (inspection export for parity checks): computes the targets of Qg [n_gtrain+n_gval][m] and
 * Ql [F][n_ltrain+n_lval][m] on the device, then trains every installed
 * filter (either model) by SGD on the MSE loss from its current weights, one shuffle
 * perms [max_epochs][n_gtrain+n_ltrain] per epoch; keeps the weights of the
 * lowest validation loss.  epochs_run / best_val (nullable, host, [F]). */
leafi_status leafi_train_filters_on(leafi_index* index, const leafi_sgd_params* p,
                                    const float* Qg, const float* Ql, const int32_t* perms,
                                    int32_t* epochs_run, double* best_val);

/* float64 z-normalisation (population sigma; a row whose sigma is below 1e-8
 * becomes zeros) of n rows of m floats on `device`: out = (x - mean) / sigma.
 * x and out may be host or device arrays and may be the same array.  The
 * paper's series and queries are z-normalised; this is the library's way to
 * meet that input contract. */
leafi_status leafi_znormalize(const float* x, int64_t n, int32_t m, float* out, int32_t device);

/* ------------------------------------------------------------------ */
/* Conformal auto-tuners (Sec. 4.4, Alg. 4)                            */
/* ------------------------------------------------------------------ */

/* Alg. 4 on calibration queries Qc [nc][m] for each k in kclasses (ascending,
 * <= LEAFI_MAX_KCLASSES): alpha = |d^L - d^f| sorted descending per filter;
 * at each sorted position j all filters take their j-th alpha, the search
 * (same wave schedule) is simulated for every calibration query, and
 * qprime[c][j] = running minimum over j of the mean recall@k. */
leafi_status leafi_fit_autotuners(leafi_index* index, const float* Qc, int64_t nc,
                                  const int32_t* kclasses, int32_t nk);
/* How the search turns a recall target t into a sorted position (Sec. 4.4.2,
 * STEP reading).  Position j of a k-class table misses M_j = N (1 - qprime_j)
 * of the N = min(k, n) nc true neighbours of the calibration queries; it is
 * accepted when the binomial tail P(Bin(N, 1 - t) <= M_j) is at most
 * 1 - confidence, and the positions are tested in order of decreasing
 * offsets, the first failure ending the sequence.  The chosen position then
 * has recall below t with probability at most 1 - confidence (over the draw of
 * the calibration queries); a target no position can certify runs exactly.
 * confidence 0 uses the point estimate qprime_j >= t.  Default 0.95. */
leafi_status leafi_set_calibration_confidence(leafi_index* index, double confidence);

/* LEAFI_CALIB_STEP (default): the certified position above.  LEAFI_CALIB_STEFFEN
 * (the paper's auto-tuner f^c: a monotone spline through each filter's
 * calibration points): for a query of k-class c and target t in (0, 1),
 * filter f's offset is Steffen's (1990) monotone cubic interpolation, in
 * float64, through the points (qprime[c][j], alpha_f,(j)) ordered by
 * increasing qprime (j from nc - 1 down to 0; of equal qprime values the one
 * of the largest j, i.e. the smallest offset, is kept), evaluated at t and
 * clamped to the end points outside them.  It carries no certificate (the
 * confidence setting does not apply); a query whose k exceeds every class or
 * whose target is >= 1 runs exactly in both modes. */
leafi_status leafi_set_calibration_mode(leafi_index* index, int32_t mode);
/* The offsets the search uses for one query of this k and recall target
 * under the index's current mode and confidence: offsets [F] (float64, host).
 * *uses_filters (nullable) receives 1, or 0 when the query runs exactly
 * (offsets are then left unchanged). */
leafi_status leafi_calibration_offsets(leafi_index* index, int32_t k, double recall_target,
                                       double* offsets, int32_t* uses_filters);

/* Read (alpha_sorted [F][nc] float64, qprime [nk][nc] float64) back. */
leafi_status leafi_get_autotuners(leafi_index* index, double* alpha_sorted, double* qprime);
/* Install auto-tuner tables computed elsewhere (same layouts). */
leafi_status leafi_set_autotuners(leafi_index* index, const double* alpha_sorted,
                                  const double* qprime, int64_t nc, const int32_t* kclasses,
                                  int32_t nk);

/* ------------------------------------------------------------------ */
/* Search (Alg. 2)                                                     */
/* ------------------------------------------------------------------ */

typedef struct {
  int64_t leaves_scanned;  /* (query, leaf) pairs searched */
  int64_t series_scanned;  /* (query, series) distances computed */
  int64_t filter_evals;    /* (query, filter) predictions made: after the route
                              leaves' round the tensor-core forward predicts
                              only the pairs that can reach a filter test
                              (leaf not searched, bound test passed against
                              the current best-so-far); the CUDA-core and CNN
                              forwards predict every pair */
  int64_t waves;           /* scan rounds launched, summed over batches (a full batch
                              always launches its first two, the second maybe empty) */
  int64_t batches;         /* internal query batches (256 queries each) */
  int64_t distinct_series; /* series of the distinct leaves each round read, summed */
  int64_t rechecks;        /* canonical float32 re-checks by the tensor-core scan */
  int64_t graph_batches;   /* batches replayed from a captured CUDA graph */
  double host_wait_ms;     /* host time the call spent waiting for the GPU (batch pair
                              counts, its end) */
  double host_ms;          /* host time of the whole call */
  int64_t filter_pruned;   /* (query, leaf) pairs pruned by the leaf's filter (Alg. 2) */
  int64_t lb_pruned;       /* (query, leaf) pairs neither searched nor filter-pruned: pruned
                              by the summarisation bound (Alg. 2) */
} leafi_search_stats;

/* k-NN of nq queries (1 <= k <= LEAFI_MAX_K).  recall_target >= 1 runs the
 * exact search (filters off); recall_target in (0, 1) uses the auto-tuned
 * offsets: the query's k picks the smallest calibrated k-class >= k, the
 * target picks the largest sorted position j whose calibrated quality
 * certifies it (leafi_set_calibration_confidence), and leaf f is pruned when
 * d^f - alpha_f,(j) > best-so-far.  A query whose class or target has no
 * certified position runs exactly.
 * LEAFI_ENOTTRAINED if recall_target < 1 and no auto-tuners exist.
 * ids [nq][k] int64, dists [nq][k] float32 Euclidean. stats nullable. */
leafi_status leafi_search(leafi_index* index, const float* queries, int64_t nq, int32_t k,
                          double recall_target, int64_t* ids, float* dists,
                          leafi_search_stats* stats);
/* Inspection export of Alg. 2: the same search as leafi_search, which also
 * writes scanned [nq][n_leaves] uint8 (host or device, caller-owned): 1 where
 * the leaf was searched for the query (its route leaf and every leaf a wave
 * took), 0 where the lower bound or the filter pruned it or the search ended
 * first.  Allocates nq * n_leaves bytes of device scratch for the call;
 * LEAFI_EINVAL on a NULL output, the errors of leafi_search otherwise. */
leafi_status leafi_search_scanned(leafi_index* index, const float* queries, int64_t nq,
                                  int32_t k, double recall_target, int64_t* ids, float* dists,
                                  uint8_t* scanned);
/* Search-schedule autotuner (no counterpart in the paper; the wave width W is
 * this implementation's batching parameter).  Times k-NN searches of n_probe
 * probe queries (dataset series drawn by the library's generator plus
 * Gaussian noise of sigma in [noise_lo, noise_hi], z-normalised) for every
 * candidate (wave width, work items per SM), `reps` timed runs after one
 * warm-up each, and keeps the fastest on the index.  target >= 1 (or 0) times
 * exact searches and sets the wave width of calls without filtered queries
 * (and of all calls while no auto-tuners are fitted).  target in (0, 1) times
 * LeaFi searches at that recall target: the wave width is part of what the
 * auto-tuners calibrate (Alg. 4 simulates the search), so every candidate
 * width first refits the tables from the calibration queries the index keeps
 * (LEAFI_EINVAL if it has none, e.g. tables set by leafi_set_autotuners);
 * the chosen width and its tables are installed.  Zero-length candidate
 * lists take the defaults: waves {16, 32, 64, 128, 256, 1024, n_leaves},
 * items per SM {2, 4, 8}. */
typedef struct {
  int32_t n_probe;          /* probe queries (8192: 32 batches) */
  int32_t k;                /* k of the probe searches (1) */
  double noise_lo, noise_hi;/* (0.1, 0.4) */
  uint64_t seed;
  int32_t reps;             /* timed runs per candidate (3) */
  int32_t n_waves;          /* candidates (<= 8; 0 = defaults) */
  int32_t waves[8];
  int32_t n_items;          /* candidates (<= 4; 0 = defaults) */
  int32_t items_per_sm[4];
  double target;            /* 0 or >= 1: exact searches; (0, 1): LeaFi searches */
} leafi_tune_params;
typedef struct {
  int32_t wave, items_per_sm;  /* chosen and installed */
  double ms_best;              /* probe search time of the choice (best of reps) */
  double ms_before;            /* ... of the index's settings before tuning */
  int32_t n_tried;
  int32_t tried_wave[32], tried_items[32];
  double tried_ms[32];
} leafi_tune_report;
leafi_status leafi_tune_search(leafi_index* index, const leafi_tune_params* params,
                               leafi_tune_report* report);

/* Batches of one search call in flight, 1..8 (default 8): each has its own
 * scratch and stream, so one batch's bounds, filters and host round trips
 * overlap another's scan.  One lane runs the batches one after another (the
 * scan launches are then serialised, e.g. to time them alone). */
leafi_status leafi_set_search_lanes(leafi_index* index, int32_t lanes);

/* Work items of the leaf scan.  A work item is (leaf, part of at most `rows`
 * series, group of queries); rows is a multiple of 128 in [128, 8192]
 * (default 2048).  The tensor-core scan picks each round's part on the device:
 * the largest of rows, rows / 2, ... but not below min_rows (a multiple of 128,
 * default 512) that gives the round at least items_per_sm items per SM
 * (default 4; 0 always uses rows), since a launch lasts as long as its most
 * loaded SM.  Smaller parts balance better, larger ones cost less per item; a
 * round too small for every SM leaves SMs to the other batches in flight.
 * `blocks`: thread blocks of a tensor-core scan launch (0 = one per SM).
 * Results do not depend on any of them. */
leafi_status leafi_set_scan_part(leafi_index* index, int32_t rows, int32_t items_per_sm,
                                 int32_t min_rows, int32_t blocks);

/* Queries per batch of a search call, 1..4096 (default 256).  A batch is
 * one unit of Alg. 2 on the device: one launch of each of its bound, filter
 * and preparation kernels, then waves of leaf-scan rounds over all of its
 * queries, so a leaf that several of its queries need is read once per wave
 * for all of them.  Each query is searched on its own terms (its own route
 * leaf, bound, offsets and best-so-far), so results do not depend on the
 * batch size; larger batches read fewer bytes per query, smaller ones answer
 * sooner. */
leafi_status leafi_set_search_batch(leafi_index* index, int32_t queries);

/* Query scheduling of calls with more than one internal batch (on by
 * default): the batches are cut from the queries in order of their route
 * leaf, so that each batch's queries need largely the same leaves and the
 * batch reads fewer distinct series.  Results and their order are the same
 * either way (every query is searched on its own terms); off keeps the
 * caller's order. */
leafi_status leafi_set_query_schedule(leafi_index* index, int32_t on);

/* Exact k-NN with summarisation-bound pruning only (the plain index). */
leafi_status leafi_exact_search(leafi_index* index, const float* queries, int64_t nq, int32_t k,
                                int64_t* ids, float* dists, leafi_search_stats* stats);
/* Per-query k [nq] and recall target [nq] (host or device); outputs are
 * [nq][kmax] with entries past a query's own k set to -1 / +inf. */
leafi_status leafi_search_mixed(leafi_index* index, const float* queries, int64_t nq,
                                const int32_t* k, const double* recall_target, int32_t kmax,
                                int64_t* ids, float* dists, leafi_search_stats* stats);

/* ------------------------------------------------------------------ */
/* Serving: a request loop over a resident index (no counterpart in the  */
/* paper, which answers one query at a time; the search it runs is       */
/* Alg. 2 as above).                                                     */
/* ------------------------------------------------------------------ */

/* A server owns a worker thread and its own pair of search lanes (scratch
 * and streams) on the index's device; the index, its filters and its
 * auto-tuner tables stay resident and are shared with the index's other
 * entry points (calls on the index are serialised with the server's batches
 * by the index mutex).  Requests carry their own k and recall target per
 * query.  Pending queries of all requests form batches of up to `max_batch`
 * (continuous batching: a request that arrives while batches are on the GPU
 * joins the next batch; up to four batches are in flight, so one's preparation
 * overlaps the other's scan), and each batch groups its (query, leaf) pairs
 * by leaf, so requests share leaf scans.  A partial batch launches when
 * nothing is in flight or its oldest query has waited `max_wait_ms`.
 * Results are those of leafi_search_mixed on the same queries: each is the
 * same alone and in any mix. */
typedef struct leafi_server leafi_server;

typedef struct {
  int32_t max_batch;    /* queries per batch, 1..4096 (default 256; larger batches share
                           each wave's leaf reads among more queries) */
  int32_t kmax;         /* largest k of any request, 1..LEAFI_MAX_K; results are [nq][kmax] */
  double max_wait_ms;   /* a partial batch waits at most this long for company (default 0.2) */
  int64_t max_bytes;    /* admission budget: host bytes of queries and results of the requests
                           admitted and not yet collected (0 = 1 GiB).  Device memory does not
                           grow with admitted work: each lane's scratch is sized for a full
                           batch at leafi_serve_start */
} leafi_serve_params;

/* Start serving `index` (device index, built and, for targets < 1, tuned).
 * The server must be stopped before the index is freed. */
leafi_status leafi_serve_start(leafi_index* index, const leafi_serve_params* params,
                               leafi_server** out);

/* Submit nq queries (host memory, [nq][m] float32; copied before returning)
 * with per-query k [nq] (1..kmax) and recall targets [nq] (>= 1 exact).
 * On success *ticket identifies the request.  LEAFI_EAGAIN: the admission
 * budget is full (collect results, then retry); LEAFI_ENOTTRAINED: a target
 * below 1 on an index without auto-tuners. */
leafi_status leafi_serve_submit(leafi_server* server, const float* queries, int64_t nq,
                                const int32_t* k, const double* recall_target, int64_t* ticket);

/* Wait up to wait_ms (0 = just look) for request `ticket`.  When it is done,
 * copies its results to ids / dists (host, [nq][kmax], entries past a
 * query's k are -1 / +inf), sets *done = 1 and *latency_ms (submit to last
 * result), and forgets the request (its budget is released); otherwise
 * *done = 0.  An unknown ticket is LEAFI_EINVAL. */
leafi_status leafi_serve_poll(leafi_server* server, int64_t ticket, int64_t* ids, float* dists,
                              double wait_ms, int32_t* done, double* latency_ms);

/* Counters since the start: requests and queries completed, batches run,
 * batches that replayed a captured graph, the search statistics summed over
 * the batches, requests admitted while at least one batch was on the GPU
 * (continuous batching), and the device bytes the server's lanes hold (fixed
 * per lane and reserved at leafi_serve_start; admitted requests wait in host
 * memory, which is why the admission budget counts host bytes). */
typedef struct {
  int64_t requests, queries, batches, graph_batches;
  leafi_search_stats search;
  int64_t admitted_in_flight;
  int64_t device_bytes;
} leafi_serve_stats;
leafi_status leafi_serve_get_stats(leafi_server* server, leafi_serve_stats* stats);

/* Finish every admitted request, stop the worker and free the server.
 * Results not yet collected are discarded. */
leafi_status leafi_serve_stop(leafi_server* server);

#ifdef __cplusplus
}
#endif
#endif /* LEAFI_H */
