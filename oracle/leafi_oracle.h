/*
 * LeaFi oracle — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU restatement of the LeaFi search path
 * (Wang, Ileana, Palpanas, "LeaFi: Data Series Indexes on Steroids with
 * Learned Filters", SIGMOD 2025).  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library; the product path never
 * does, and this file shares no code with the CUDA implementation.
 *
 * Floating point: distances are the canonical float32 definition below (the
 * decision precision of the product); everything else is float64.
 */
#ifndef LEAFI_ORACLE_H
#define LEAFI_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_tree or_tree;

enum { OR_DSTREE = 0, OR_ISAX = 1 };

/* Canonical squared Euclidean distance (Sec. 3, "Similarity search"):
 * acc = 0; for i in 0..m-1 { t = q_i - x_i; acc = fmaf(t, t, acc); }  (float32). */
float or_sqdist(const float* q, const float* x, int m);

/* Brute-force k-NN (Sec. 3 problem statement): the k series with the smallest
 * (canonical d^2, id), lexicographic.  Outputs nq x k; pads with -1 / +inf. */
void or_knn(const float* X, int64_t n, int m, const float* Q, int64_t nq, int k,
            int64_t* ids, float* d2);

/* Segment statistics of one series from float64 prefix sums. */
void or_segment_stats(const float* x, int m, int s, int e, double* mu, double* sd);

/* DSTree (EAPCA) build; X must stay alive while the tree is used. */
or_tree* or_dstree_build(const float* X, int64_t n, int m, int leaf_cap, int init_segments);
/* iSAX build: w PAA segments, 2^card_bits symbols. */
or_tree* or_isax_build(const float* X, int64_t n, int m, int leaf_cap, int w, int card_bits);
void or_tree_free(or_tree* t);

int32_t or_tree_n_leaves(const or_tree* t);
int32_t or_tree_n_nodes(const or_tree* t);
/* leaf id of every series (original id order) */
void or_tree_leaf_of(const or_tree* t, int32_t* leaf_of);
void or_tree_leaf_sizes(const or_tree* t, int64_t* sizes);
/* series ids of one leaf (ascending); returns the count */
int64_t or_tree_leaf_members(const or_tree* t, int32_t leaf, int64_t* ids, int64_t cap);
/* iSAX breakpoints beta_1..beta_{2^b - 1} (float64) */
void or_isax_breakpoints(int card_bits, double* beta);

/* Leaf lower bounds LB^2 (float64, max over the root-to-leaf path), nq x L. */
void or_leaf_lb2(const or_tree* t, const float* Q, int64_t nq, double* lb2);
/* Route leaf of each query (descend by the split rules). */
void or_route(const or_tree* t, const float* Q, int64_t nq, int32_t* leaf);

/* Per-(query, leaf) top-k inside one leaf: for each query i, leaf leaves[i*nl + j]
 * (j < nl); outputs [nq][nl][k] (d2, id), padded with +inf / -1. */
void or_leaf_topk(const or_tree* t, const float* Q, int64_t nq, const int32_t* leaves, int nl,
                  int k, float* d2, int64_t* ids);

/* MLP filters m -> h -> 1, ReLU hidden, linear output (Sec. 5.1): float64. */
void or_mlp_forward(const float* W1, const float* b1, const float* w2, const float* b2,
                    int F, int h, int m, const float* Q, int64_t nq, double* out);

/* Training targets d^L (Alg. 1, Sec. 4.3): global queries x filtered leaves and
 * local queries x their own leaf, Euclidean float32 (sqrtf of canonical d^2). */
void or_train_targets(const or_tree* t, const int32_t* filter_leaf, int F,
                      const float* Qg, int64_t ng, const float* Ql, int64_t nl,
                      float* Tg /* ng x F */, float* Tl /* F x nl */);

typedef struct {
  int32_t n_gtrain, n_gval;   /* global queries: first n_gtrain train, next n_gval val */
  int32_t n_ltrain, n_lval;   /* local queries per filter */
  int32_t batch;              /* minibatch size */
  int32_t max_epochs;
  int32_t patience;           /* epochs without improvement before lr /= 10 */
  double lr0, lr_min;
} or_train_params;

/* SGD training of all F filters (Sec. 5.1).  Weights in/out (float32, updated in
 * place with the best-validation weights).  perms: [max_epochs][n_gtrain+n_ltrain].
 * epochs_run/best_val (nullable) receive per-filter statistics. */
void or_train(const or_train_params* p, int F, int h, int m,
              const float* Qg, const float* Tg, const float* Ql, const float* Tl,
              const int32_t* perms, float* W1, float* b1, float* w2, float* b2,
              int32_t* epochs_run, double* best_val);

/* CNN filters (Sec. 5.2 model-type study): conv(1->C, k=3) + ReLU, conv(C->C,
 * k=3) + ReLU (stride 1, zero padding 1), mean over positions, linear C -> 1.
 * Flat float32 parameters per filter: w1 [C][3], b1 [C], w2 [C][C][3], b2 [C],
 * wo [C], bo; or_cnn_params(C) = 3C^2 + 6C + 1 values.  Forward in float64. */
int64_t or_cnn_params(int C);
void or_cnn_forward(const float* theta, int F, int C, int m, const float* Q, int64_t nq,
                    double* out);
/* U(-1/sqrt(fan_in), 1/sqrt(fan_in)) initial parameters (fan_in 3, 3C, C). */
void or_cnn_init(int F, int C, uint64_t seed, float* theta);
/* SGD of the CNN filters: the protocol of or_train; theta [F][P] in/out. */
void or_cnn_train(const or_train_params* p, int F, int C, int m,
                  const float* Qg, const float* Tg, const float* Ql, const float* Tl,
                  const int32_t* perms, float* theta, int32_t* epochs_run, double* best_val);

/* Alg. 4 and Alg. 2 on given filter predictions (float64, [nc][F] / [nq][F]),
 * for any filter model; or_fit_autotuner / or_leafi_search take MLP weights. */
void or_fit_autotuner_pred(const or_tree* t, const double* Pc, const int32_t* filter_leaf, int F,
                           const float* Qc, int64_t nc, int k, int wave,
                           double* alpha_sorted, double* qprime);
void or_leafi_search_pred(const or_tree* t, const double* P, const int32_t* filter_leaf, int F,
                          const double* alpha_sorted, int64_t nc,
                          const float* Q, int64_t nq, const int32_t* k, const int32_t* jpos,
                          int kmax, int wave, int64_t* ids, float* d2, int64_t* stats,
                          double* min_margin, unsigned char* scanned /* nullable: [nq][L], 1 =
                          the leaf was searched (Alg. 2) */);

/* Auto-tuner learning (Alg. 4) for one k: calibration queries Qc (nc).
 * Outputs alpha_sorted [F][nc] (descending) and qprime [nc] (running-min
 * of the calibration recall at each sorted position). */
void or_fit_autotuner(const or_tree* t, const float* W1, const float* b1, const float* w2,
                      const float* b2, const int32_t* filter_leaf, int F, int h,
                      const float* Qc, int64_t nc, int k, int wave,
                      double* alpha_sorted, double* qprime);

/* Leaf selection (Alg. 3): leaves by non-increasing size (ties: lower id);
 * a leaf is taken when its size is at least th = a t^F / t^S and one more
 * filter of w bytes still fits in the budget cap (reading of the memory test:
 * w^M + w <= c^M).  Writes the selected leaf ids to out, returns their count. */
int32_t or_select_leaves_alg3(const int64_t* sizes, int32_t L, double th, double w, double cap,
                              int32_t* out);

/* Philox4x32-10 (Salmon et al., SC 2011): out = bijection(ctr) under key. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Alg. 1's query generation: n_global queries from distinct dataset series (gpick,
 * original ids) and n_local queries per filtered leaf from its members (lpick
 * [F][n_local], original ids), each + Gaussian noise of sigma ~ U[lo, hi] and
 * re-z-normalised.  Qg [n_global][m], Ql [F][n_local][m]. */
void or_training_queries(const or_tree* t, const int32_t* filter_leaf, int F, int64_t n_global,
                         int64_t n_local, double noise_lo, double noise_hi, uint64_t seed,
                         float* Qg, float* Ql, int64_t* gpick, int64_t* lpick);
/* Initial filter weights U(-1/sqrt(fan_in), 1/sqrt(fan_in)); W1 [F][h][m]. */
void or_filter_init(int F, int h, int m, uint64_t seed, float* W1, float* b1, float* w2,
                    float* b2);
/* One shuffle of [0, n) per epoch (int32 [epochs][n]). */
void or_epoch_perms(int epochs, int n, uint64_t seed, int32_t* perms);

/* Calibration quality that certifies recall target t with probability
 * `confidence` from n_trials = k nc calibration neighbours (binomial tail of
 * the misses; Sec. 3 / Sec. 4.4 reading): (N - M*) / N with M* the most misses
 * whose tail P(Bin(N, 1 - t) <= M*) is at most 1 - confidence; 2 if none;
 * confidence <= 0: t itself. */
double or_required_quality(int64_t n_trials, double target, double confidence);

/* Sorted position j* for a target (STEP reading): the largest j with
 * qprime[j] >= or_required_quality(kk nc, target, confidence) (qprime is
 * non-increasing); -1 means "no position -> filters off". */
int32_t or_offset_position(const double* qprime, int64_t nc, int64_t kk, double target,
                           double confidence);

/* Steffen (1990) monotone interpolation through (x_i, y_i), x strictly increasing,
 * evaluated at xs (clamped to the end points). */
double or_steffen_eval(const double* x, const double* y, int n, double xs);

/* LeaFi search (Alg. 2) in wave semantics: route leaf first, then waves of up to
 * `wave` leaves in (LB^2, leaf id) order.  Per query: k[i], kclass index kc[i]
 * (-1 = filters off) and sorted position jpos[i] (-1 = filters off).  Offsets
 * o_f = alpha_sorted[f][jpos].  Outputs nq x kmax ids/d2 and per-query stats
 * [leaves_scanned, series_scanned, lb_pruned, filter_pruned] plus min_margin
 * = min over filter decisions of |d^F - bsf| (for near-tie accounting). */
void or_leafi_search(const or_tree* t, const float* W1, const float* b1, const float* w2,
                     const float* b2, const int32_t* filter_leaf, int F, int h,
                     const double* alpha_sorted, int64_t nc,
                     const float* Q, int64_t nq, const int32_t* k, const int32_t* jpos,
                     int kmax, int wave, int64_t* ids, float* d2, int64_t* stats,
                     double* min_margin);

#ifdef __cplusplus
}
#endif
#endif
