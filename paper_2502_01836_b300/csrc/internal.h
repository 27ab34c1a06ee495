// Internal declarations shared by the C-ABI layer and the kernels.
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <map>
#include <vector>

#include "host_tree.h"
#include "leafi.h"

namespace leafi {

// ----------------------------------------------------------------- errors
struct Failure {
  leafi_status status;
  std::string msg;
};
[[noreturn]] void fail(leafi_status st, const char* fmt, ...);
void set_last_error(const std::string& s);

#define LF_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      ::leafi::fail(e_ == cudaErrorMemoryAllocation ? LEAFI_ENOMEM : LEAFI_ECUDA,          \
                    "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,      \
                    __LINE__);                                                             \
  } while (0)

void count_launch();
void count_launches(long long delta);
long long launches_so_far();
#define LF_CHECK_LAUNCH()            \
  do {                               \
    ::leafi::count_launch();         \
    LF_CUDA(cudaGetLastError());     \
  } while (0)

// ------------------------------------------------ injected allocation failures
// Diagnostics (leafi_debug_fail_allocations): when armed, the allocation that
// finds the countdown at zero fails as if memory were exhausted (device
// buffers: LEAFI_ENOMEM before the buffer is touched; host steps that call
// host_alloc_gate: std::bad_alloc, reported as LEAFI_ENOMEM).
bool injected_alloc_failure();
void host_alloc_gate();

// ------------------------------------------------------ device buffers
// bumped whenever any DBuf reallocates: captured CUDA graphs that hold buffer
// addresses compare it to know whether they are still valid
extern unsigned long long g_realloc_epoch;

template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  // grow to at least `count` elements (contents not preserved)
  T* need(size_t count) {
    if (count <= n && p) return p;
    if (injected_alloc_failure())
      fail(LEAFI_ENOMEM, "device allocation of %zu bytes failed (injected)", count * sizeof(T));
    release();
    size_t c = count ? count : 1;
    LF_CUDA(cudaMalloc(&p, c * sizeof(T)));
    n = c;
    ++g_realloc_epoch;
    return p;
  }
  void upload(const T* h, size_t count, cudaStream_t s) {
    need(count);
    if (count) LF_CUDA(cudaMemcpyAsync(p, h, count * sizeof(T), cudaMemcpyHostToDevice, s));
  }
  void upload(const std::vector<T>& v, cudaStream_t s) { upload(v.data(), v.size(), s); }
  size_t bytes() const { return n * sizeof(T); }
};

// keys of candidate results: (float bits of d^2) << 32 | original id.  d^2 >= 0
// so the float bits order like the values; ties break on the lower id.
constexpr unsigned long long kNoKey = ~0ull;

// attempts a tensor-core scan work item makes at a query's result-list lock
// before it reports a timeout (leafi_debug_set_lock_tries changes it per index)
constexpr int kDefaultLockTries = 1 << 16;

// ----------------------------------------------------------------- tables
struct DsTables {  // device view of a DSTree
  int n_nodes, n_leaves, n_iv, root;
  const int32_t *iv_s, *iv_e;
  const int32_t *seg_off, *seg_iv;
  // per node segment row: the float32 enclosure of its synopsis ranges,
  // {mu_lo rounded down, mu_hi rounded up, sigma_lo down, sigma_hi up}
  const float4* syn32;
  const int32_t *left, *right, *node_leaf, *split_iv, *split_sd;
  const double* thresh;
  const int32_t *path_off, *path;
};

struct IsaxTables {  // device view of an iSAX tree
  int n_nodes, n_leaves, w, bits;
  const double* beta;    // 2^bits + 1
  const float2* beta32;  // 2^bits + 1: each breakpoint rounded {down, up} to float32
  const int32_t *root_child, *left, *right, *node_leaf, *isplit, *node_bits;
  const int32_t *lo_sym, *hi_sym;  // leaf x w
};

// work pairs of one scan round: query row `q` searches leaf `leaf`, results
// go to top-k slot `slot`
struct Pair {
  int32_t slot, q, leaf, pad;
};

// ----------------------------------------------------------------- kernels
// (declared here, defined in the k_*.cu files)
void launch_prefix(const float* Q, int nq, int mp, int m, double* P, cudaStream_t s);
// Scratch of the bound kernels, in doubles: DSTree interval statistics are
// [nq][n_iv] float64 {mu, sigma} followed by [nq][n_iv] float32 enclosures
// {mu down, mu up, sigma down, sigma up}; iSAX PAA values are [nq][w] float64
// followed by [nq][w] float32 {down, up}.
inline size_t ds_ivstat_doubles(size_t nq, size_t n_iv) { return nq * n_iv * 4; }
inline size_t isax_paa_doubles(size_t nq, size_t w) { return nq * w * 2; }
void launch_ds_bounds(const DsTables& T, const double* P, int nq, int m, double* ivstat,
                      double* node_lb, double* leaf_lb, int32_t* route, cudaStream_t s);
void launch_isax_bounds(const IsaxTables& T, const double* P, int nq, int m, double* paa,
                        double* leaf_lb, int32_t* route, cudaStream_t s);

// route leaf of every query from its prefix sums (scheduling keys of a
// multi-batch search; iSAX queries without a leaf on their path get n_leaves)
void launch_route_keys(const leafi_index* ix, const double* P, int nq, int32_t* key,
                       cudaStream_t s);
bool filter_tc_fits(int m, int h, int smem_optin);
void launch_wsplit(const float* W1t, int F, int m, int h, float* Ws, cudaStream_t s);
// device counters of a search pipeline: [0] leaves searched, [1] series
// scanned, [2] distinct series, [3] canonical re-checks, [4] filter-pruned
// (query, leaf) pairs, [5] filter predictions made by the tensor-core forward
constexpr int kPipelineStats = 6;
// queries per CTA of the tensor-core filter forward
constexpr int kFilterTile = 128;
// Qs: scratch for the query planes, 2 x ceil(nq / 128) * 128 rows of m
// rounded up to 32.  rows_of / cnt (nullable, together): predict filter f only
// for the queries rows_of[f][0 .. cnt[f]) (a row stride of nq); otherwise for
// every query.  evals (nullable) += the predictions made.
void launch_filter_tc(const CUtensorMap& wmap, const float* Q, int nq, int mp, int m, int F,
                      int h, float* Qs, const float* b1, const float* w2, const float* b2,
                      float* out, int32_t* err, cudaStream_t s, const int32_t* rows_of = nullptr,
                      const int32_t* cnt = nullptr, unsigned long long* evals = nullptr);
void launch_filter_forward(const float* Q, int nq, int mp, int m, int F, int h, const float* W1t,
                           const float* b1, const float* w2, const float* b2, float* out,
                           cudaStream_t s);

// Alg. 1 random draws (k_gen.cu): Philox4x32-10 addressed by (i, j, tag,
// stream) under the key (seed low, seed high)
enum : uint32_t {
  kTagGPick = 1, kTagLPick = 2, kTagSigma = 3, kTagNoise = 4, kTagW1 = 5, kTagB1 = 6,
  kTagW2 = 7, kTagB2 = 8, kTagPerm = 9, kTagCnn = 10
};
// k distinct values of [0, n) by Floyd's algorithm, in insertion order
void gen_floyd(uint64_t seed, uint32_t tag, uint32_t stream, uint64_t n, int64_t k, int64_t* out);
// k values of [0, n) drawn independently
void gen_with_replacement(uint64_t seed, uint32_t tag, uint32_t stream, uint64_t n, int64_t k,
                          int64_t* out);
// one shuffle of [0, n) per epoch: indices ordered by their 64-bit draws
void gen_epoch_perms(int epochs, int n, uint64_t seed, int32_t* perms);
// rows [ng + F*nl][mp]: source row pos[q] of X + noise, re-z-normalised
void launch_gen_queries(const float* X, int mp, int m, const int64_t* pos, int ng, int nl, int F,
                        uint64_t seed, double lo, double hi, float* out, cudaStream_t s);
void launch_gen_weights(int F, int h, int m, uint64_t seed, float* W1t, float* b1, float* w2,
                        float* b2, cudaStream_t s);
void launch_znorm(const float* in, int64_t in_stride, int64_t n, int m, float* out,
                  int64_t out_stride, cudaStream_t s);

struct TrainArgs {
  int F, h, m, mp;
  int n_gtrain, n_gval, n_ltrain, n_lval, batch, max_epochs, patience, max_decays;
  float lr0;
  const float *Qg, *Ql, *Tg, *Tl;  // Qg [ng][mp], Ql [F][nl][mp], Tg [ng][F], Tl [F][nl]
  const int32_t* perms;
  float *W1t, *b1, *w2, *b2;       // trained in place
  float *bW1t, *bb1, *bw2, *bb2;   // best-validation copies
  int32_t* epochs_run;
  double* best_val;
};
void launch_train(const TrainArgs& a, cudaStream_t s);

// CNN filters (k_cnn.cu): flat parameters [F][cnn_params(C)]
struct CnnTrainArgs {
  int F, C, m, mp;
  int n_gtrain, n_gval, n_ltrain, n_lval, batch, max_epochs, patience, max_decays;
  float lr0;
  const float *Qg, *Ql, *Tg, *Tl;
  const int32_t* perms;
  float* theta;   // trained in place
  float* btheta;  // best-validation copy
  float* grad;    // minibatch gradient accumulators
  int32_t* epochs_run;
  double* best_val;
};
int64_t cnn_params(int C);
bool cnn_fits(int m, int C, int smem_optin);
void launch_cnn_forward(const float* Q, int nq, int mp, int m, int F, int C, const float* theta,
                        float* out, cudaStream_t s);
void launch_cnn_train(const CnnTrainArgs& a, cudaStream_t s);
void launch_gen_cnn_weights(int F, int C, uint64_t seed, float* theta, cudaStream_t s);

struct ScanArgs {
  const float* X;        // [n][mp] leaf-major
  const int32_t* ids;    // position -> original id
  const int64_t* leaf_off;
  int L, mp, k;
  int part;              // series per work item
  const float* Q;        // [nq][mp]
  const Pair* pairs;     // grouped by leaf
  const int32_t* grp_off;   // L + 1: pair offsets per leaf
  const int32_t* item_off;  // L + 1: work-item offsets per leaf
  unsigned long long* thr;        // per slot: admission threshold key (lowered by finished items)
  unsigned long long* cand;       // per slot: candidate keys (cap each)
  int32_t* cand_cnt;              // per slot
  int cand_cap;
  int32_t* err;                   // error word (set on overflow)
};
size_t scan_smem_bytes(int mp, int k);
int scan_group_size();

struct TcScanArgs {
  const float* X;                  // [n][mp] float32 leaf-major (canonical re-check)
  const __half* Xh;                // [n][kp] float16 copy (tensor-core operand)
  const float* xn;                 // [n] |x|^2
  const int32_t* ids;
  const int64_t* leaf_off;
  int L, mp, kp, k;
  int part;
  const float* Q;                  // [nq][mp]
  const __half* Qh;                // [nq][kp] float16 queries (launch_tc_query_prep)
  const unsigned char* Q8;         // [nq][kp] e4m3 queries (launch_tc_query_prep8), or null
  const float* sx;                 // e4m3 operands: [n] power-of-two scale of every series
  int fp8;                         // 1: the operands are e4m3 (X8, Q8), kp bytes per row
  const float4* Qk;                // [nq][2] band constants (launch_tc_query_prep)
  int nbuf;                        // query tiles in shared memory (tc_scan_plan)
  int G;                           // queries per work item of the fixed grouping (tc_group_size)
  const Pair* pairs;
  const int32_t* grp_off;
  const int32_t* item_off;
  const int32_t* item_leaf;        // leaf of every work item
  const int32_t* gfirst;           // k > 1: first query group of each leaf (launch_var_groups),
  const int32_t* gbound;           //   group starts in `pairs`; null: groups of G queries
  int qkeys;                       // k > 1: keys per TMEM lane quarter's lists (tc_scan_plan)
  const int32_t* part_dev;         // the round's part size, chosen by the grouping kernels
                                   // (nullptr: `part`)
  int32_t* work;                   // work-item counter (zero at launch)
  unsigned long long* topk;        // [nslots][k] ascending keys, kNoKey padded
                                   // (launch_tc_round_prep); work items merge into it
  int32_t* glock;                  // per slot lock of its list (zero at the round's start)
  float* ub;                       // k = 1: per slot upper bound of the best canonical distance
                                   // over the rows scanned so far in the round (+inf at its
                                   // start), shared by the work items; null for k > 1
  int lock_tries;                  // attempts at a slot's lock before the item reports a timeout
  int32_t* err;
  unsigned long long* stat;        // nullable: [0] += canonical re-checks
  unsigned long long* prof;        // nullable: per-phase cycle counters (16)
};
int tc_group_size(int k);
// query tiles (2 or 1) the tensor-core scan can keep for rows of kp halves and
// top-k lists of k keys within `smem_optin` bytes (0 if it does not fit);
// qkeys: for k > 1 the keys of each lane quarter's lists (a group's sum of k)
int tc_scan_plan(int rb, int k, int smem_optin, size_t* smem, int* qkeys);  // rb: operand row bytes
// out[p][i] = X[order[p]][i] for i < m, 0 for m <= i < mp (leaf-major rows)
void launch_gather_rows(const float* X, int64_t n, int m, const int32_t* order, int mp, float* out,
                        cudaStream_t s);
void launch_tc_query_prep(const float* Q, int nq, int mp, int kp, __half* Qh, float4* Qk,
                          cudaStream_t s);
void launch_tc_query_prep8(const float* Q, int nq, int mp, int kp, unsigned char* Q8, float4* Qk,
                           cudaStream_t s);
void launch_tc_scan(const CUtensorMap& tmap, const TcScanArgs& a, const int32_t* n_items_dev,
                    const int32_t* slot_k, int grid, cudaStream_t s);
// before a tensor-core round: pad every slot's list (entries [cnt, k)) with
// kNoKey, release the slot locks, reset the shared upper bounds and zero the
// work-item counter; after it: count the list entries and set each slot's
// threshold (its k-th key, kNoKey while fewer than k)
void launch_tc_round_prep(int nslots, int kstride, const int32_t* slot_k, unsigned long long* topk,
                          const int32_t* topk_cnt, int32_t* glock, float* ub, int32_t* work,
                          cudaStream_t s);
void launch_tc_round_finish(int nslots, int kstride, const int32_t* slot_k,
                            const unsigned long long* topk, int32_t* topk_cnt,
                            unsigned long long* thr, cudaStream_t s);
void launch_scan(const ScanArgs& a, const int32_t* n_items_dev, const int32_t* slot_k, int grid,
                 cudaStream_t s);

// k > 1 on the tensor-core scan: each leaf's grouped pairs cut into groups of
// at most 64 queries whose k sum to at most `budget`; gfirst [L + 1] = first
// group of each leaf, gbound [groups + 1] = group starts in the grouped pairs,
// item_off [L + 1] / item_leaf / n_items for the (part, group) work items
// target_items > 0 (tensor-core scan): the round's part size is chosen on the
// device among part, part / 2, ... (>= 128 rows) so that the round has at least
// target_items work items if it can, and written to *part_out
void launch_var_groups(int L, const int64_t* leaf_off, int part, const int32_t* grp_off,
                       const Pair* grouped, const int32_t* slot_k, int kstride, int budget,
                       int32_t* ngroups, int32_t* gfirst, int32_t* gbound, int32_t* item_off,
                       int32_t* item_leaf, int32_t* n_items_dev, cudaStream_t s,
                       int target_items = 0, int32_t* part_out = nullptr, int min_part = 128);
// The tensor-core round's prep (launch_tc_round_prep's work), which the
// one-block grouping kernel takes on when it is small
struct RoundPrep {
  unsigned long long* topk = nullptr;  // null: nothing to prepare
  const int32_t* topk_cnt = nullptr;
  int32_t* glock = nullptr;
  float* ub = nullptr;
  int32_t* work = nullptr;
  int nslots = 0, kstride = 0;
};
// stat (nullable): stat[0] += series of the distinct leaves in this round;
// g = queries per work item of the scan kernel that follows; rp (nullable):
// returns true when the grouping launch also did the round's prep
bool launch_group(const Pair* pairs, const int32_t* npairs_dev, int npairs_max, int L,
                  const int64_t* leaf_off, int part, int g, int32_t* cnt, int32_t* grp_off,
                  int32_t* item_off, Pair* grouped, int32_t* n_items_dev,
                  unsigned long long* stat, cudaStream_t s, int32_t* item_leaf = nullptr,
                  bool pack_small = false, int target_items = 0, int32_t* part_out = nullptr,
                  int min_part = 128, const RoundPrep* rp = nullptr);

void launch_merge(int nslots, int kstride, const int32_t* slot_k, unsigned long long* topk,
                  int32_t* topk_cnt, unsigned long long* thr, const unsigned long long* cand,
                  int32_t* cand_cnt, int cand_cap, cudaStream_t s);

struct SelectArgs {
  int nq, L, W;
  const double* lb2;              // [nq][L]
  const unsigned long long* thr;  // per query admission key (k-th best)
  // filters (P null = filters off for all)
  const float* P;                 // [nq][F]
  int F;
  const int32_t* leaf_filter;     // [L] filter of a leaf or -1
  const double* alpha;            // [F][nc]
  int nc;
  const int32_t* jpos;            // [nq] sorted position or -1
  const int64_t* leaf_off;
  // state
  unsigned char* scanned;         // [nq][L]
  int32_t* done;                  // [nq]
  Pair* pairs;
  int32_t* npairs;
  unsigned long long* stat;       // [0] leaves searched, [1] series scanned, [4] leaves
                                  // pruned by their filter (each once per query)
};

// one captured search batch (full 256-query batch, route round + one wave)
struct BatchGraph {
  cudaGraphExec_t exec = nullptr;
  int nb = 0, kmax = 0, use_f = 0, profiling = 0, pre_p = 0;
  unsigned long long epoch = 0;
  unsigned long long gen = 0;   // leafi_index::graph_gen at capture
  long long launches = 0;       // kernels in the graph (added to the launch counter per replay)
  std::vector<cudaEvent_t> ev;  // start/stop pairs recorded inside the graph
  std::vector<int> kind;
};

// per-kernel device time on the index's stream (enabled by leafi_set_profiling)
struct KernelClock {
  std::vector<cudaEvent_t> ev;  // start/stop pairs
  std::vector<int> kind;
  double ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long n[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};
// wave selection (Alg. 2's leaf loop) walking a precomputed visiting order
// (`ord` [nq][L] ascending (LB^2, leaf id), cursor = next position per query)
void launch_select_walk(const SelectArgs& a, const int32_t* ord, int32_t* cursor, cudaStream_t s);
// the same picks for a wave at least as wide as the index (a.W >= a.L): no order needed
void launch_select_all(const SelectArgs& a, cudaStream_t s);
// rows_of[f][0 .. cnt[f]) = the queries (any order) whose prediction of
// filter f a later wave select may read: the query uses filters, f's leaf is
// not searched and passes the bound test against the current best-so-far
// (rows_of: F rows of stride nq; cnt: F counters, zeroed here)
void launch_filter_need(int nq, int F, int L, const int32_t* filter_leaf, const double* lb2,
                        const unsigned long long* thr, const unsigned char* scanned,
                        const int32_t* jpos, int32_t* rows_of, int32_t* cnt, cudaStream_t s);
void launch_leafknn_pairs(int nq, int nl, const int32_t* leaves, int L, Pair* pairs,
                          int32_t* npairs, cudaStream_t s);
void launch_fill_u64(unsigned long long* p, unsigned long long v, size_t n, cudaStream_t s);
// a batch's per-query state before its first wave in one launch: searched flags
// (route leaf only), route pairs (npairs = nq, stat[0..1] counted), cursor,
// list counts, thresholds, candidate counts, done flags and, with jpos non-null,
// the sorted offset positions
void launch_batch_init(int nq, int L, const int32_t* route, unsigned char* scanned,
                       const int64_t* leaf_off, Pair* pairs, int32_t* npairs,
                       unsigned long long* stat, int32_t* cursor, int32_t* topk_cnt,
                       unsigned long long* thr, int32_t* cand_cnt, int32_t* done,
                       const int32_t* k, const double* target, int nk, const int32_t* kclasses,
                       const double* qprime, int nc, int32_t* jpos, cudaStream_t s);
void launch_write_results(int nq, int kmax, const int32_t* kq, const unsigned long long* topk,
                          int kstride, const int32_t* topk_cnt, int64_t* ids, float* dists,
                          cudaStream_t s,
                          const int32_t* rows = nullptr);
void launch_leafknn_out(int nslots, int k, const unsigned long long* topk, const int32_t* topk_cnt,
                        float* d2, int64_t* ids, cudaStream_t s);

// calibration (Alg. 4)
struct CalibArgs {
  int nc, L, F, kc, W;
  const double* lb2;              // [nc][L]
  const int32_t* route;           // [nc]
  const unsigned long long* lk;   // [nc][L][lk_stride] per-leaf top keys (first kc used)
  int lk_stride;
  const float* P;                 // [nc][F]
  const int32_t* filter_leaf;     // [F]
  const int32_t* leaf_filter;     // [L]
  double* alpha;                  // [F][nc] (sorted descending after launch_calib_alpha)
  int32_t* ord;                   // [nc][L] scratch: visiting order
  int32_t* cnt_true;              // [nc][L] scratch
  unsigned long long* work;       // scratch, >= max(nc*nc*kc, nc*L/2 + 1) entries
  long long* hits;                // [nc] scratch
  double* qprime;                 // [nc] out
  int kk;                         // min(kc, n)
  void* order_scratch;            // leaf_order_scratch(nc, L) bytes (more than 4096 leaves)
};
int calib_max_sort();
// per query: leaves sorted by ascending (LB^2, leaf id), ord [nq][L]
// bytes of scratch launch_leaf_order needs for nq queries over L leaves (0 up to 4096 leaves)
size_t leaf_order_scratch(int nq, int L);
void launch_leaf_order(int nq, int L, const double* lb2, int32_t* ord, cudaStream_t s,
                       void* scratch = nullptr);
int calib_max_wave();
void launch_calib_alpha(const CalibArgs& a, cudaStream_t s);
void launch_calib_sim(const CalibArgs& a, cudaStream_t s);

}  // namespace leafi

namespace leafi {
constexpr int kMaxLanes = 8;  // search lanes an index (or a server) may use
// Per-lane scratch of the search driver and the other entry points.
struct Scratch {
  DBuf<float> sQ;
  DBuf<__half> sQh;        // float16 queries of the tensor-core scan
  DBuf<unsigned char> sQ8; // e4m3 queries of the tensor-core scan (scan_path 2)
  DBuf<float4> sQk;        // their band constants
  DBuf<float> sQs;         // tf32 hi/lo query planes of the tensor-core filter forward
  DBuf<int32_t> sItemLeaf; // leaf of every scan work item of a round
  DBuf<int32_t> sWork;     // work-item counter of the tensor-core scan
  DBuf<double> sP, sIv, sNode, sLb, sPaa, sTarget;
  DBuf<int32_t> sRoute, sK, sJpos, sCnt, sGrpOff, sItemOff, sNpairs, sCandCnt, sTopkCnt, sDone,
      sNItems, sOrd, sCursor;
  DBuf<unsigned char> sScanned, sOrderTmp;
  DBuf<Pair> sPairs, sGrouped;
  DBuf<unsigned long long> sTopk, sThr, sCand;
  DBuf<int32_t> sGlock;           // per slot locks of the tensor-core scan's top-k lists
  DBuf<float> sUb;                // k = 1: per slot upper bounds shared by a round's work items
  DBuf<int32_t> sPart;            // the round's work-item rows (chosen by the grouping kernels)
  DBuf<int32_t> sNGroups, sGFirst, sGBound;  // k > 1: query groups sized by k (launch_var_groups)
  DBuf<float> sPred, sOutD;
  DBuf<int32_t> sNeed;            // [F][batch] queries of each filter's predictions a batch needs,
                                  // then [F] their counts
  DBuf<int64_t> sOutI;
  // search lane
  cudaStream_t st = nullptr;       // created on first use (non-blocking)
  cudaEvent_t ev_np = nullptr;     // the pair count of the lane's batch reached the host
  int32_t* h_np = nullptr;         // pinned host word
  std::vector<BatchGraph> graphs;  // captured batches of this lane
  void release_lane();
  size_t bytes() const;            // device bytes held by the lane's buffers
};
// query scheduling of a multi-batch search call (search_impl)
struct Schedule {
  DBuf<float> Q;       // the call's queries, staged [nq][mp]
  DBuf<double> P;      // their prefix sums
  DBuf<int32_t> key;   // route leaf per query
  DBuf<int32_t> perm;  // queries in batch order
  DBuf<int64_t> out_i; // results in the caller's row order (host outputs)
  DBuf<float> out_d;
};
}  // namespace leafi

// ----------------------------------------------------------------- index
struct leafi_index {
  std::mutex mu;
  int device = 0;          // -1: host-only index (tree inspection, no device data)
  cudaStream_t stream = nullptr;
  leafi::HostTree tree;
  int m = 0, mp = 0, wave = 8, scan_path = 0;
  int wave_exact = 8;      // wave width of calls without filtered queries (tuned on its own)
  int64_t n = 0;

  // resident data
  leafi::DBuf<float> X;          // [n][mp] leaf-major
  leafi::DBuf<__half> Xh;        // [n][kp] float16 copy for the tensor-core scan (scan_path 0)
  leafi::DBuf<unsigned char> X8; // [n][kp] e4m3 copy (scan_path 2), with
  leafi::DBuf<float> sx;         //   [n] power-of-two scales (x ~ sx * e4m3 row)
  leafi::DBuf<float> xn;         // [n] squared norms
  int kp = 0;                    // operand row length (fp16: m rounded up to 64; e4m3: to 128)
  bool tc_ok = false;            // tensor-core scan usable for this index
  bool pack_small = false;       // some window of 8 consecutive leaves fits one 128-row chunk
  CUtensorMap xh_map;            // 2-D TMA map of Xh (box {64, 128}) or X8 (box {128, 128})
  bool tc_scan() const { return tc_ok && scan_path != 1; }  // leaf scans on tensor cores
  int op_row_bytes() const { return scan_path == 2 ? kp : 2 * kp; }
  int smem_optin = 0;            // opt-in shared memory per block of the device
  leafi::DBuf<int32_t> ids;      // position -> original id
  leafi::DBuf<int64_t> leaf_off;
  // DSTree tables
  leafi::DBuf<int32_t> iv_s, iv_e, seg_off, seg_iv, left, right, node_leaf, split_iv, split_sd,
      path_off, path;
  leafi::DBuf<float4> syn32;
  leafi::DBuf<double> thresh;
  // iSAX tables
  leafi::DBuf<double> beta;
  leafi::DBuf<float2> beta32;
  leafi::DBuf<int32_t> root_child, isplit, node_bits, lo_sym, hi_sym;

  // filters
  int F = 0, h = 0;                    // h: MLP hidden width, or CNN channels C
  int model = LEAFI_FILTER_MLP;
  bool trained = false;
  std::vector<int32_t> filter_leaf;
  leafi::DBuf<int32_t> d_filter_leaf, d_leaf_filter;
  leafi::DBuf<float> W1t, b1, w2, b2;  // MLP: W1t [F][m][h]
  leafi::DBuf<float> cnn;              // CNN: [F][cnn_params(h)]

  // auto-tuners
  int nc = 0, nk = 0;
  int kclasses[LEAFI_MAX_KCLASSES] = {0, 0, 0, 0};
  leafi::DBuf<double> alpha, qprime;
  leafi::DBuf<int32_t> d_kclasses;
  leafi::DBuf<float> calib_q;    // the calibration queries [nc][mp] behind the tables (kept so
                                 // that the tables can be refitted for another wave width)
  // query-time offsets: LEAFI_CALIB_STEP reads alpha at a certified position;
  // LEAFI_CALIB_STEFFEN interpolates each filter's (q', alpha) points at the
  // target.  The Steffen offsets of each (k-class, target) in use are extra
  // columns of `offs` [F][offs_stride] (the alpha table in the first nc columns).
  int calib_mode = LEAFI_CALIB_STEP;
  unsigned long long tables_gen = 0;       // bumped whenever alpha / qprime change
  unsigned long long offs_gen = ~0ull;     // tables_gen `offs` was built from
  std::vector<double> h_alpha, h_qprime;   // host copies behind `offs`
  std::map<std::pair<int, double>, int> steffen_cols;  // (k-class, target) -> column
  leafi::DBuf<double> offs;
  int offs_stride = 0;

  // scratch (grown on demand): lanes[0] serves every entry point; a search of
  // more than one batch spreads its batches over several lanes in turn
  leafi::Scratch lanes[leafi::kMaxLanes];
  leafi::Scratch* sc = &lanes[0];  // lane in use
  leafi::DBuf<int32_t> sErr;       // error word shared by all launches
  leafi::DBuf<unsigned long long> sStat;  // search counters of one call
  leafi::DBuf<float> Ws;         // tf32 hi/lo weight planes of the tensor-core filter forward
  CUtensorMap wmap;              // TMA descriptor of Ws
  bool ws_dirty = true;          // weights changed since Ws was built
  std::map<int, std::pair<int, int>> tc_plan;  // k -> (query tiles of the tensor-core scan (0: does
                                               // not fit), keys per lane quarter's lists)

  bool schedule = true;    // multi-batch calls cut batches in route-leaf order
  int search_lanes = 8;    // batches of one search call in flight (leafi_set_search_lanes)
  int search_batch = 256;  // queries per batch of a search call (leafi_set_search_batch)
  int part = 2048;         // series per scan work item (leafi_set_scan_part); the tensor-core
                           // scan's rounds may take part / 2, ... (>= 128) for balance
  int items_per_sm = 4;    // work items per SM a tensor-core round aims at
  int min_part = 512;      // smallest part a tensor-core round may take
  int scan_blocks = 0;     // blocks of a tensor-core scan launch (0: one per SM)
  leafi::Schedule sched;
  int lock_tries = leafi::kDefaultLockTries;  // see leafi_debug_set_lock_tries
  double calib_confidence = 0.95;  // probability that a certified position meets its target
  std::map<std::pair<int64_t, double>, double> rq_cache;  // (N, target) -> required quality
  int profiling = 0;       // 0 off, 1 leaf-scan kernel times, 2 every kind + scan phases
  bool ticked = false;     // the last tick() recorded a start event
  leafi::BatchGraph* capturing = nullptr;  // entry being captured (tick/tock record into it)
  bool graphs_ok = true;                   // cleared if capture is not possible
  unsigned long long graph_gen = 0;        // bumped by drop_graphs (filters, tables, profiling)
  void drop_graphs();
  leafi::DBuf<unsigned long long> scan_prof;  // tensor-core scan phase cycles (profiling)
  leafi::KernelClock clock;
  void tick(int kind);   // record a start event of `kind` on the stream
  void tock();           // record the matching stop event
  void settle();         // accumulate finished event pairs (stream synchronised)

  leafi::DsTables ds() const;
  leafi::IsaxTables isax() const;
};
