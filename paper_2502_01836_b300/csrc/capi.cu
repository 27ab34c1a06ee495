// C ABI (include/leafi.h): argument checks, host/device staging, and the
// search driver that runs the LeaFi path (Alg. 2) on the GPU in waves.
#include <cuda_fp8.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>
#include <unordered_map>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <memory>
#include <new>
#include <numeric>
#include <stdexcept>

#include "internal.h"

namespace leafi {

unsigned long long g_realloc_epoch = 0;

namespace {
thread_local std::string g_last_error;
constexpr int kBatch = 256;       // queries per search batch (default)
constexpr int kMaxBatch = 4096;   // largest batch of a search call or a server
constexpr int kSearchLanes = 8;   // batches of one search call in flight
constexpr int kServeLanes = 4;    // batches of a server in flight
constexpr size_t kKnnBudget = 256ull << 20;  // bytes of candidate buffer per leaf-knn batch
}  // namespace

void set_last_error(const std::string& s) { g_last_error = s; }

namespace {
std::atomic<long long> g_launches{0};
}
std::atomic<long long> g_fail_alloc_countdown{-1};

bool injected_alloc_failure() {
  long long v = g_fail_alloc_countdown.load(std::memory_order_relaxed);
  while (v >= 0) {
    if (g_fail_alloc_countdown.compare_exchange_weak(v, v - 1, std::memory_order_relaxed))
      return v == 0;  // the armed allocation fails; the countdown then stays at -1
  }
  return false;
}

void host_alloc_gate() {
  if (injected_alloc_failure()) throw std::bad_alloc();
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long delta) { g_launches.fetch_add(delta, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(); }

void fail(leafi_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  throw Failure{st, buf};
}

namespace {

template <class Fn>
leafi_status guarded(Fn&& fn) {
  try {
    fn();
    return LEAFI_OK;
  } catch (const Failure& e) {
    set_last_error(e.msg);
    return e.status;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return LEAFI_ENOMEM;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return LEAFI_EINTERNAL;
  }
}

// float32 values enclosing a float64 one: the largest float at or below it and
// the smallest at or above it (the bound kernels widen every synopsis range
// and breakpoint outward, so their float32 gaps never exceed the float64 ones)
float f32_below(double v) {
  const float f = (float)v;
  return (double)f > v ? std::nextafter(f, -std::numeric_limits<float>::infinity()) : f;
}
float f32_above(double v) {
  const float f = (float)v;
  return (double)f < v ? std::nextafter(f, std::numeric_limits<float>::infinity()) : f;
}

bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) LF_CUDA(cudaSetDevice(dev));
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// copy `count` elements from a host or device array into a device buffer
template <class T>
const T* to_device(const T* user, size_t count, DBuf<T>& tmp, cudaStream_t s) {
  if (on_device(user)) return user;
  tmp.upload(user, count, s);
  return tmp.p;
}

template <class T>
void to_host(std::vector<T>& out, const T* user, size_t count, cudaStream_t s) {
  out.resize(count);
  if (!count) return;
  if (on_device(user)) {
    LF_CUDA(cudaMemcpyAsync(out.data(), user, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    LF_CUDA(cudaStreamSynchronize(s));
  } else {
    std::memcpy(out.data(), user, count * sizeof(T));
  }
}

// write device results to a user array that may be host or device
template <class T>
void deliver(T* user, const T* dev, size_t count, cudaStream_t s) {
  if (!count) return;
  LF_CUDA(cudaMemcpyAsync(user, dev, count * sizeof(T),
                          on_device(user) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
}

// queries [nq][m] (host or device) -> padded device rows [nq][mp] in `buf`
const float* stage_queries(leafi_index* ix, const float* q, int64_t nq, DBuf<float>& buf) {
  cudaStream_t s = ix->stream;
  const bool dev = on_device(q);
  if (dev && ix->m == ix->mp && (reinterpret_cast<uintptr_t>(q) % 16) == 0) return q;
  float* d = buf.need((size_t)nq * ix->mp);
  if (ix->mp != ix->m) LF_CUDA(cudaMemsetAsync(d, 0, sizeof(float) * nq * ix->mp, s));
  LF_CUDA(cudaMemcpy2DAsync(d, sizeof(float) * ix->mp, q, sizeof(float) * ix->m,
                            sizeof(float) * ix->m, (size_t)nq,
                            dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  return d;
}

int sm_count(int dev) {
  int v = 0;
  LF_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
  return v;
}

int64_t max_leaf_size(const HostTree& t) {
  int64_t mx = 0;
  for (int l = 0; l < t.n_leaves; ++l) mx = std::max(mx, t.leaf_off[l + 1] - t.leaf_off[l]);
  return mx;
}

// parts (work items of ix->part series) of the largest leaf
int max_parts(const leafi_index* ix) {
  return (int)((max_leaf_size(ix->tree) + ix->part - 1) / ix->part);
}

__global__ void sqrt_kernel(const float* __restrict__ in, float* __restrict__ out, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __fsqrt_rn(in[i]);
}

__global__ void slots_init_kernel(int nslots, int32_t* topk_cnt, unsigned long long* thr,
                                  int32_t* cand_cnt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nslots) return;
  topk_cnt[t] = 0;
  thr[t] = kNoKey;
  cand_cnt[t] = 0;
}

// float16 copy (rows of kp, zero padded) and squared norms of the series;
// maxabs receives max |x| (as float bits) to decide whether float16 is safe
__global__ void half_copy_kernel(const float* __restrict__ X, int64_t n, int mp, int m, int kp,
                                 __half* __restrict__ Xh, float* __restrict__ xn,
                                 unsigned int* __restrict__ maxabs) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x / 32);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  float ss = 0.0f, mx = 0.0f;
  for (int i = lane; i < kp; i += 32) {
    const float v = i < m ? X[row * mp + i] : 0.0f;
    ss = fmaf(v, v, ss);
    mx = fmaxf(mx, fabsf(v));
    Xh[row * kp + i] = __float2half_rn(v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (lane == 0) {
    xn[row] = ss;
    atomicMax(maxabs, __float_as_uint(mx));
  }
}

// e4m3 copy (rows of kp bytes, zero padded) with a power-of-two scale per
// series (max |x_i| / sx <= 448, the largest finite e4m3 value) and the
// squared norms, one warp per series
__global__ void fp8_copy_kernel(const float* __restrict__ X, int64_t n, int mp, int m, int kp,
                                unsigned char* __restrict__ X8, float* __restrict__ sx,
                                float* __restrict__ xn) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x / 32);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  float ss = 0.0f, mx = 0.0f;
  for (int i = lane; i < m; i += 32) {
    const float v = X[row * mp + i];
    ss = fmaf(v, v, ss);
    mx = fmaxf(mx, fabsf(v));
  }
  for (int o = 16; o > 0; o >>= 1) {
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  int e = 0;
  if (mx > 0.0f) frexpf(mx / 448.0f, &e);
  const float sc = mx > 0.0f ? ldexpf(1.0f, e) : 1.0f;
  for (int i = lane; i < kp; i += 32) {
    const float v = i < m ? X[row * mp + i] : 0.0f;
    X8[row * kp + i] = (unsigned char)__nv_cvt_float_to_fp8(v / sc, __NV_SATFINITE, __NV_E4M3);
  }
  if (lane == 0) {
    xn[row] = ss;
    sx[row] = sc;
  }
}

__global__ void transpose_kernel(const float* __restrict__ in, float* __restrict__ out, int F,
                                 int rows, int cols) {
  // in [F][rows][cols] -> out [F][cols][rows]
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t per = (size_t)rows * cols;
  if (t >= per * F) return;
  const size_t f = t / per, r = (t % per) / cols, c = t % cols;
  out[f * per + c * rows + r] = in[t];
}

// 2-D TMA descriptor of the float16 copy: dims {kp, n}, row stride kp*2 bytes,
// box {64 columns, 128 rows} with 128-byte swizzle (one 16 KB block of a chunk)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// 2-D tiled TMA descriptor with 128-byte swizzle: `inner` elements per row
// (row stride `row_bytes`), `outer` rows, boxes of box_inner x box_outer
bool encode_2d(CUtensorMap* map, CUtensorMapDataType dt, void* base, uint64_t inner, uint64_t outer,
               uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  static void* fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      fn = nullptr;
      return false;
    }
  }
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = reinterpret_cast<EncodeTiledFn>(fn)(
      map, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
      CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 2-D TMA descriptor of the operand copy: dims {kp, n}, 128-byte boxes of
// 128 rows (64 float16 or 128 e4m3 columns)
bool encode_xh_map(leafi_index* ix) {
  if (ix->scan_path == 2)
    return encode_2d(&ix->xh_map, CU_TENSOR_MAP_DATA_TYPE_UINT8, ix->X8.p, (uint64_t)ix->kp,
                     (uint64_t)ix->n, (uint64_t)ix->kp, 128, 128);
  return encode_2d(&ix->xh_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, ix->Xh.p, (uint64_t)ix->kp,
                   (uint64_t)ix->n, (uint64_t)ix->kp * 2, 64, 128);
}

// ---------------------------------------------------------------- filters
// The tensor-core forward (3xTF32) serves indexes on the tensor-core scan path
// whose hidden width fits one MMA (h <= 256); the CUDA-core forward the rest.
bool filter_tc(const leafi_index* ix) {
  return ix->model == LEAFI_FILTER_MLP && ix->scan_path != 1 && ix->F > 0 &&
         filter_tc_fits(ix->m, ix->h, ix->smem_optin);
}

// (re)build the tf32 weight planes after the weights changed
void ensure_wsplit(leafi_index* ix) {
  if (!filter_tc(ix) || !ix->ws_dirty) return;
  const int hp = (ix->h + 15) / 16 * 16, Kq = (ix->m + 31) / 32 * 32;
  float* Ws = ix->Ws.need((size_t)2 * ix->F * hp * Kq);
  launch_wsplit(ix->W1t.p, ix->F, ix->m, ix->h, Ws, ix->stream);
  // slice-major planes: rows of 32 floats, one box = one slice of one plane
  if (!encode_2d(&ix->wmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, Ws, 32,
                 (uint64_t)2 * ix->F * (Kq / 32) * hp, 128, 32, (uint32_t)hp))
    fail(LEAFI_ECUDA, "cannot encode the filter weight tensor map");
  ix->ws_dirty = false;
}

// P[q][f] for nq queries (device rows of mp floats); `cap_rows` sizes the
// scratch for later calls of up to that many queries.  rows_of / cnt / evals
// (the tensor-core forward only): predict filter f only for the queries
// rows_of[f][0 .. cnt[f]) and count the predictions made.
void filter_forward(leafi_index* ix, const float* dQ, int nq, float* P, int cap_rows = 0,
                    const int32_t* rows_of = nullptr, const int32_t* cnt = nullptr,
                    unsigned long long* evals = nullptr) {
  if (nq <= 0 || ix->F <= 0) return;
  if (ix->model == LEAFI_FILTER_CNN) {
    launch_cnn_forward(dQ, nq, ix->mp, ix->m, ix->F, ix->h, ix->cnn.p, P, ix->stream);
    return;
  }
  if (!filter_tc(ix)) {
    launch_filter_forward(dQ, nq, ix->mp, ix->m, ix->F, ix->h, ix->W1t.p, ix->b1.p, ix->w2.p,
                          ix->b2.p, P, ix->stream);
    return;
  }
  if (ix->ws_dirty) fail(LEAFI_EINTERNAL, "filter weight planes are stale");
  const int Kq = (ix->m + 31) / 32 * 32;
  const int capp = (std::max(nq, cap_rows) + 127) / 128 * 128;
  float* Qs = ix->sc->sQs.need((size_t)2 * capp * Kq);
  launch_filter_tc(ix->wmap, dQ, nq, ix->mp, ix->m, ix->F, ix->h, Qs, ix->b1.p, ix->w2.p,
                   ix->b2.p, P, ix->sErr.p, ix->stream, rows_of, cnt, evals);
}

// One scan round: group pairs by leaf, scan, merge candidates into slots.
// query tiles of the tensor-core scan for top-k lists of k keys (0: CUDA-core scan)
int tc_nbuf(leafi_index* ix, int k, int* qkeys = nullptr) {
  if (!ix->tc_scan()) return 0;
  auto it = ix->tc_plan.find(k);
  if (it == ix->tc_plan.end()) {
    int qk = 0;
    const int nb = tc_scan_plan(ix->op_row_bytes(), k, ix->smem_optin, nullptr, &qk);
    it = ix->tc_plan.emplace(k, std::make_pair(nb, qk)).first;
  }
  if (qkeys) *qkeys = it->second.second;
  return it->second.first;
}

// float16 (or e4m3) rows and band constants of nq queries for the tensor-core
// scan (null pointers when the index scans on CUDA cores)
struct TcQueries {
  __half* Qh = nullptr;
  unsigned char* Q8 = nullptr;
  float4* Qk = nullptr;
  bool on() const { return Qh || Q8; }
};
void launch_query_prep(const leafi_index* ix, const float* dQ, int nq, const TcQueries& t,
                       cudaStream_t s) {
  if (t.Q8) launch_tc_query_prep8(dQ, nq, ix->mp, ix->kp, t.Q8, t.Qk, s);
  else if (t.Qh) launch_tc_query_prep(dQ, nq, ix->mp, ix->kp, t.Qh, t.Qk, s);
}
TcQueries prep_tc_queries(leafi_index* ix, const float* dQ, int nq, int cap_rows) {
  TcQueries r;
  if (!ix->tc_scan()) return r;
  const size_t rows = (size_t)std::max(nq, cap_rows);
  if (ix->scan_path == 2) r.Q8 = ix->sc->sQ8.need(rows * ix->kp);
  else r.Qh = ix->sc->sQh.need(rows * ix->kp);
  r.Qk = ix->sc->sQk.need(2 * rows);
  launch_query_prep(ix, dQ, nq, r, ix->stream);
  return r;
}

void run_round(leafi_index* ix, const float* dQ, const TcQueries& tq, const Pair* pairs,
               const int32_t* dNpairs, int npairs_max, int nslots, int kstride,
               const int32_t* slot_k, unsigned long long* topk, int32_t* topk_cnt,
               unsigned long long* thr, unsigned long long* cand, int32_t* cand_cnt, int cap,
               unsigned long long* distinct_stat = nullptr,
               unsigned long long* recheck_stat = nullptr) {
  cudaStream_t s = ix->stream;
  const int L = ix->tree.n_leaves;
  int32_t* cnt = ix->sc->sCnt.need(L);
  int32_t* goff = ix->sc->sGrpOff.need(L + 1);
  int32_t* ioff = ix->sc->sItemOff.need(L + 1);
  Pair* grouped = ix->sc->sGrouped.need(std::max(npairs_max, 1));
  int32_t* nitems = ix->sc->sNItems.need(1);
  int qkeys = 0;
  const int nbuf = tq.on() ? tc_nbuf(ix, kstride, &qkeys) : 0;
  const bool use_tc = nbuf > 0;
  const bool var_groups = use_tc && kstride > 1;  // groups bounded by the sum of their k
  // the tensor-core scan's rounds pick their work-item size on the device: the
  // largest of part, part / 2, ... that gives every SM several items
  const int target = use_tc ? ix->items_per_sm * sm_count(ix->device) : 0;
  int32_t* part_dev = use_tc ? ix->sc->sPart.need(1) : nullptr;
  int32_t* item_leaf =
      use_tc ? ix->sc->sItemLeaf.need(std::max((size_t)std::max(npairs_max, 1) * max_parts(ix),
                                               (size_t)3 * target + 1))
             : nullptr;
  // the tensor-core round's prep rides on the one-block grouping kernel when small
  RoundPrep rp;
  if (use_tc) {
    rp.topk = topk;
    rp.topk_cnt = topk_cnt;
    rp.glock = ix->sc->sGlock.need(nslots);
    rp.ub = kstride == 1 ? ix->sc->sUb.need(nslots) : nullptr;
    rp.work = ix->sc->sWork.need(1);
    rp.nslots = nslots;
    rp.kstride = kstride;
  }
  const bool prepped =
      launch_group(pairs, dNpairs, npairs_max, L, ix->leaf_off.p, ix->part,
                   use_tc ? tc_group_size(kstride) : scan_group_size(), cnt, goff, ioff, grouped,
                   nitems, distinct_stat, s, var_groups ? nullptr : item_leaf,
                   use_tc && !var_groups && ix->pack_small, var_groups ? 0 : target,
                   var_groups ? nullptr : part_dev, std::min(ix->min_part, ix->part),
                   use_tc ? &rp : nullptr);
  int32_t *gfirst = nullptr, *gbound = nullptr;
  if (var_groups) {
    int32_t* ngr = ix->sc->sNGroups.need(L);
    gfirst = ix->sc->sGFirst.need(L + 1);
    gbound = ix->sc->sGBound.need((size_t)std::max(npairs_max, 1) + 1);
    launch_var_groups(L, ix->leaf_off.p, ix->part, goff, grouped, slot_k, kstride, qkeys, ngr, gfirst,
                      gbound, ioff, item_leaf, nitems, s, target, part_dev,
                      std::min(ix->min_part, ix->part));
  }
  const int grid = use_tc ? (ix->scan_blocks > 0 ? ix->scan_blocks : sm_count(ix->device))
                          : sm_count(ix->device) * 2;
  if (use_tc) {
    TcScanArgs t;
    t.X = ix->X.p;
    t.Xh = ix->Xh.p;
    t.xn = ix->xn.p;
    t.ids = ix->ids.p;
    t.leaf_off = ix->leaf_off.p;
    t.L = L;
    t.mp = ix->mp;
    t.kp = ix->kp;
    t.k = kstride;
    t.part = ix->part;
    t.part_dev = part_dev;
    t.Q = dQ;
    t.Qh = tq.Qh;
    t.Q8 = tq.Q8;
    t.sx = ix->sx.p;
    t.fp8 = ix->scan_path == 2 ? 1 : 0;
    t.Qk = tq.Qk;
    t.nbuf = nbuf;
    t.G = tc_group_size(kstride);
    t.pairs = grouped;
    t.grp_off = goff;
    t.item_off = ioff;
    t.item_leaf = item_leaf;
    t.gfirst = gfirst;
    t.gbound = gbound;
    t.qkeys = qkeys;
    t.work = rp.work;  // zeroed by the round's prep
    t.topk = topk;
    t.glock = rp.glock;
    t.ub = rp.ub;
    t.lock_tries = ix->lock_tries;
    if (!prepped) launch_tc_round_prep(nslots, kstride, slot_k, topk, topk_cnt, t.glock, t.ub, t.work, s);
    t.err = ix->sErr.p;
    t.stat = recheck_stat;
    t.prof = ix->profiling >= 2 ? ix->scan_prof.p : nullptr;
    ix->tick(0);
    launch_tc_scan(ix->xh_map, t, nitems, slot_k, grid, s);
    ix->tock();
    ix->tick(1);
    launch_tc_round_finish(nslots, kstride, slot_k, topk, topk_cnt, thr, s);
    ix->tock();
    return;
  }
  ScanArgs a;
  a.X = ix->X.p;
  a.ids = ix->ids.p;
  a.leaf_off = ix->leaf_off.p;
  a.L = L;
  a.mp = ix->mp;
  a.k = kstride;
  a.part = ix->part;
  a.Q = dQ;
  a.pairs = grouped;
  a.grp_off = goff;
  a.item_off = ioff;
  a.thr = thr;
  a.cand = cand;
  a.cand_cnt = cand_cnt;
  a.cand_cap = cap;
  a.err = ix->sErr.p;
  ix->tick(0);
  launch_scan(a, nitems, slot_k, grid, s);
  ix->tock();
  ix->tick(1);
  launch_merge(nslots, kstride, slot_k, topk, topk_cnt, thr, cand, cand_cnt, cap, s);
  ix->tock();
}

void check_err_word(leafi_index* ix) {
  int32_t err = 0;
  LF_CUDA(cudaMemcpyAsync(&err, ix->sErr.p, sizeof(err), cudaMemcpyDeviceToHost, ix->stream));
  LF_CUDA(cudaStreamSynchronize(ix->stream));
  if (err) {
    LF_CUDA(cudaMemsetAsync(ix->sErr.p, 0, sizeof(int32_t), ix->stream));
    if (err & 2) fail(LEAFI_ETIMEOUT, "a tensor-core scan wait timed out (error word %d)", err);
    fail(LEAFI_EINTERNAL, "candidate buffer overflow (error word %d)", err);
  }
}

// bounds and routes for nq padded device queries
// (have_p: the prefix sums are already in the lane's sP)
void compute_bounds(leafi_index* ix, const float* dQ, int nq, double* lb2, int32_t* route,
                    bool have_p = false) {
  cudaStream_t s = ix->stream;
  const HostTree& t = ix->tree;
  double* P = ix->sc->sP.need((size_t)nq * 2 * (ix->m + 1));
  if (!have_p) launch_prefix(dQ, nq, ix->mp, ix->m, P, s);
  if (t.type == LEAFI_DSTREE) {
    double* iv = ix->sc->sIv.need(ds_ivstat_doubles(nq, t.iv_s.size()));
    double* nodes = ix->sc->sNode.need((size_t)nq * t.n_nodes);
    launch_ds_bounds(ix->ds(), P, nq, ix->m, iv, nodes, lb2, route, s);
  } else {
    double* paa = ix->sc->sPaa.need(isax_paa_doubles(nq, t.w));
    launch_isax_bounds(ix->isax(), P, nq, ix->m, paa, lb2, route, s);
  }
}

// per-(query, leaf) top-k inside leaves: slots [nq][nl], keys stride k
void leaf_knn_device(leafi_index* ix, const float* dQ, int nq, const int32_t* dLeaves, int nl,
                     int k, DBuf<unsigned long long>& topk, DBuf<int32_t>& topk_cnt) {
  cudaStream_t s = ix->stream;
  const int L = ix->tree.n_leaves;
  const int nslots = nq * nl;
  const int cap = max_parts(ix) * k;
  topk.need((size_t)nslots * k);
  topk_cnt.need(nslots);
  unsigned long long* thr = ix->sc->sThr.need(nslots);
  int32_t* cand_cnt = ix->sc->sCandCnt.need(nslots);
  if (nslots == 0) return;
  slots_init_kernel<<<(nslots + 255) / 256, 256, 0, s>>>(nslots, topk_cnt.p, thr, cand_cnt);
  LF_CHECK_LAUNCH();
  const TcQueries tq = prep_tc_queries(ix, dQ, nq, 0);
  // batches of queries keep the CUDA-core scan's candidate buffer bounded
  // (the tensor-core scan merges into the lists directly)
  const bool direct = tq.on() && tc_nbuf(ix, k) > 0;
  const size_t per_query = (size_t)nl * cap * sizeof(unsigned long long);
  int qb = (int)std::max<size_t>(1, kKnnBudget / std::max<size_t>(per_query, 1));
  qb = direct ? nq : std::min(qb, nq);
  unsigned long long* cand = direct ? nullptr : ix->sc->sCand.need((size_t)qb * nl * cap);
  Pair* pairs = ix->sc->sPairs.need((size_t)qb * nl);
  int32_t* np = ix->sc->sNpairs.need(1);
  for (int q0 = 0; q0 < nq; q0 += qb) {
    const int nb = std::min(qb, nq - q0);
    const int ns = nb * nl;
    launch_leafknn_pairs(nb, nl, dLeaves + (size_t)q0 * nl, L, pairs, np, s);
    TcQueries tb;
    if (tq.on()) {
      if (tq.Qh) tb.Qh = tq.Qh + (size_t)q0 * ix->kp;
      if (tq.Q8) tb.Q8 = tq.Q8 + (size_t)q0 * ix->kp;
      tb.Qk = tq.Qk + (size_t)2 * q0;
    }
    // slots of this batch are [q0*nl, q0*nl + ns): shift the bases
    run_round(ix, dQ + (size_t)q0 * ix->mp, tb, pairs, np, ns, ns, k, nullptr,
              topk.p + (size_t)q0 * nl * k, topk_cnt.p + (size_t)q0 * nl, thr + (size_t)q0 * nl,
              cand, cand_cnt + (size_t)q0 * nl, cap);
  }
  check_err_word(ix);
}

void require_index(const leafi_index* ix) {
  if (!ix) fail(LEAFI_EINVAL, "index is NULL");
}

void require_device(const leafi_index* ix) {
  require_index(ix);
  if (ix->device < 0) fail(LEAFI_EINVAL, "index was built host-only (device -1)");
}

void check_queries(const leafi_index* ix, const float* q, int64_t nq) {
  if (nq < 0 || nq > (int64_t)std::numeric_limits<int32_t>::max() / 4)
    fail(LEAFI_EINVAL, "nq out of range");
  if (nq > 0 && !q) fail(LEAFI_EINVAL, "queries is NULL");
  (void)ix;
}

// Calibration quality that certifies recall target t with probability `conf`
// from N calibration neighbours: a position whose misses M satisfy
// P(Bin(N, 1 - t) <= M) <= 1 - conf is accepted, and since the calibrated
// quality only falls along the sorted positions, testing them in order and
// stopping at the first failure bounds the chance that the chosen position's
// recall is below t by 1 - conf.  Returns (N - M*) / N for the largest such
// M*, 2 (no position: exact search) if even M = 0 fails or t >= 1, and t itself
// for conf <= 0 (the point estimate).
double required_quality(int64_t N, double t, double conf) {
  if (!(t < 1.0) || N < 1) return 2.0;
  if (conf <= 0.0) return t;
  const double p = 1.0 - t, log_delta = std::log(1.0 - conf);
  const double lratio = std::log(p) - std::log1p(-p);
  double lpmf = (double)N * std::log1p(-p);  // log P(Bin = 0)
  double lcdf = lpmf;
  int64_t m_star = -1;
  for (int64_t i = 0; i <= N && lcdf <= log_delta; ++i) {
    m_star = i;
    // next term: pmf(i + 1) = pmf(i) (N - i) / (i + 1) p / (1 - p)
    lpmf += std::log((double)(N - i)) - std::log((double)(i + 1)) + lratio;
    const double hi = std::max(lcdf, lpmf), lo = std::min(lcdf, lpmf);
    lcdf = hi + std::log1p(std::exp(lo - hi));
  }
  if (m_star < 0) return 2.0;
  return (double)(N - m_star) / (double)N;
}

// Steffen (1990) monotone cubic interpolation at t through points of strictly
// increasing x, clamped to the end values: the cubic Hermite piece of each
// interval with slopes limited to keep monotone data monotone.
double steffen_at(const std::vector<double>& x, const std::vector<double>& y, double t) {
  const int n = (int)x.size();
  if (n == 1 || t <= x[0]) return y[0];
  if (t >= x[n - 1]) return y[n - 1];
  auto secant = [&](int i) { return (y[i + 1] - y[i]) / (x[i + 1] - x[i]); };
  auto sign = [](double v) { return (double)((v > 0.0) - (v < 0.0)); };
  // slope at node i (interior: limited harmonic-style choice; ends: one-sided
  // parabola through three points, limited)
  auto slope = [&](int i) {
    if (n == 2) return secant(0);
    if (i > 0 && i < n - 1) {
      const double h0 = x[i] - x[i - 1], h1 = x[i + 1] - x[i];
      const double s0 = secant(i - 1), s1 = secant(i);
      const double p = (s0 * h1 + s1 * h0) / (h0 + h1);
      return (sign(s0) + sign(s1)) * std::min(std::min(std::fabs(s0), std::fabs(s1)),
                                              0.5 * std::fabs(p));
    }
    const int a = i == 0 ? 0 : n - 2, b = i == 0 ? 1 : n - 3;
    const double h0 = x[a + 1] - x[a], h1 = x[b + 1] - x[b];
    const double s0 = secant(a), s1 = secant(b);
    const double p = s0 * (1.0 + h0 / (h0 + h1)) - s1 * h0 / (h0 + h1);
    if (p * s0 <= 0.0) return 0.0;
    return std::fabs(p) > 2.0 * std::fabs(s0) ? 2.0 * s0 : p;
  };
  int i = 0;
  while (i < n - 2 && t >= x[i + 1]) ++i;
  const double h = x[i + 1] - x[i], s = secant(i);
  const double d0 = slope(i), d1 = slope(i + 1);
  const double a3 = (d0 + d1 - 2.0 * s) / (h * h);
  const double a2 = (3.0 * s - 2.0 * d0 - d1) / h;
  const double u = t - x[i];
  return ((a3 * u + a2) * u + d0) * u + y[i];
}

constexpr int kSteffenCols = 64;  // (k-class, target) columns of the offset table

// Steffen offsets of every filter for k-class c at target t (host tables)
void steffen_offsets(const leafi_index* ix, int c, double t, double* out) {
  const int nc = ix->nc;
  const double* qp = ix->h_qprime.data() + (size_t)c * nc;
  std::vector<int> js;  // nodes by increasing qprime, the largest j of equal values
  for (int j = nc - 1; j >= 0; --j)
    if (js.empty() || qp[j] > qp[js.back()]) js.push_back(j);
  std::vector<double> x(js.size()), y(js.size());
  for (size_t z = 0; z < js.size(); ++z) x[z] = qp[js[z]];
  for (int f = 0; f < ix->F; ++f) {
    const double* a = ix->h_alpha.data() + (size_t)f * nc;
    for (size_t z = 0; z < js.size(); ++z) y[z] = a[js[z]];
    out[f] = steffen_at(x, y, t);
  }
}

// the offset table of STEFFEN mode: alpha in the first nc columns, one column
// per (k-class, target) in use after them; rebuilt when the tables change.
// Returns the column for (c, t).  The caller holds the index mutex.
int steffen_column(leafi_index* ix, int c, double t) {
  cudaStream_t s = ix->stream;
  const int F = ix->F, nc = ix->nc;
  if (ix->offs_gen != ix->tables_gen) {
    ix->h_alpha.resize((size_t)F * nc);
    ix->h_qprime.resize((size_t)ix->nk * nc);
    LF_CUDA(cudaMemcpyAsync(ix->h_alpha.data(), ix->alpha.p, sizeof(double) * F * nc,
                            cudaMemcpyDeviceToHost, s));
    LF_CUDA(cudaMemcpyAsync(ix->h_qprime.data(), ix->qprime.p, sizeof(double) * ix->nk * nc,
                            cudaMemcpyDeviceToHost, s));
    LF_CUDA(cudaStreamSynchronize(s));
    ix->steffen_cols.clear();
    ix->offs_stride = nc + kSteffenCols;
    double* o = ix->offs.need((size_t)F * ix->offs_stride);
    LF_CUDA(cudaMemcpy2DAsync(o, sizeof(double) * ix->offs_stride, ix->alpha.p, sizeof(double) * nc,
                              sizeof(double) * nc, (size_t)F, cudaMemcpyDeviceToDevice, s));
    LF_CUDA(cudaStreamSynchronize(s));
    ix->offs_gen = ix->tables_gen;
  }
  const auto key = std::make_pair(c, t);
  auto it = ix->steffen_cols.find(key);
  if (it != ix->steffen_cols.end()) return it->second;
  if ((int)ix->steffen_cols.size() >= kSteffenCols) {
    // every column in use: start over (the graphs hold no column numbers)
    ix->steffen_cols.clear();
  }
  const int col = nc + (int)ix->steffen_cols.size();
  std::vector<double> v(F);
  steffen_offsets(ix, c, t, v.data());
  LF_CUDA(cudaMemcpy2DAsync(ix->offs.p + col, sizeof(double) * ix->offs_stride, v.data(),
                            sizeof(double), sizeof(double), (size_t)F, cudaMemcpyHostToDevice, s));
  LF_CUDA(cudaStreamSynchronize(s));
  ix->steffen_cols.emplace(key, col);
  return col;
}

// per query: the quality its k-class table must reach for its target (2 when
// the query runs exactly); cached per (N, target) on the index.  STEFFEN mode:
// -(column + 1) of the query's offsets in the offset table.
void required_qualities(leafi_index* ix, int nb, const int32_t* kq, const double* target,
                        bool uniform, std::vector<double>& out) {
  out.resize(uniform ? 1 : nb);
  for (size_t i = 0; i < out.size(); ++i) {
    const double t = target[i];
    int c = -1;
    for (int z = 0; z < ix->nk; ++z)
      if (ix->kclasses[z] >= kq[i]) {
        c = z;
        break;
      }
    if (c < 0 || !(t < 1.0) || ix->nc == 0) {
      out[i] = 2.0;
      continue;
    }
    if (ix->calib_mode == LEAFI_CALIB_STEFFEN) {
      out[i] = -(double)(steffen_column(ix, c, t) + 1);
      continue;
    }
    const int64_t N = std::min<int64_t>(ix->kclasses[c], ix->n) * ix->nc;
    const auto key = std::make_pair(N, t);
    auto it = ix->rq_cache.find(key);
    if (it == ix->rq_cache.end())
      it = ix->rq_cache.emplace(key, required_quality(N, t, ix->calib_confidence)).first;
    out[i] = it->second;
  }
}


// a scheduled batch's inputs in one launch: query rows and prefix-sum rows
// gathered from the call's staged arrays, and (uniform batches) every query's k
// and required quality
__global__ void batch_prep_kernel(const float* __restrict__ Qall, const double* __restrict__ Pall,
                                  const int32_t* __restrict__ rows, int nb, int mp, int w,
                                  float* __restrict__ gQ, double* __restrict__ P, int uniform,
                                  int32_t* __restrict__ k, double* __restrict__ rq, int kval,
                                  double rqval) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int mp4 = mp / 4;
  const int64_t nq4 = (int64_t)nb * mp4, np = (int64_t)nb * w;
  if (t < nq4) {
    const int i = (int)(t / mp4), c = (int)(t % mp4);
    reinterpret_cast<float4*>(gQ)[t] = reinterpret_cast<const float4*>(Qall)[(int64_t)rows[i] * mp4 + c];
  } else if (t < nq4 + np) {
    const int64_t u = t - nq4;
    const int i = (int)(u / w), c = (int)(u % w);
    P[u] = Pall[(int64_t)rows[i] * w + c];
  } else if (uniform && t < nq4 + np + nb) {
    const int i = (int)(t - nq4 - np);
    k[i] = kval;
    rq[i] = rqval;
  }
}


__global__ void fill_batch_kernel(int nb, int32_t* k, double* target, int kval, double tval) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nb) {
    k[i] = kval;
    target[i] = tval;
  }
}

// Device pointers of one lane's batch scratch, sized for a full batch.
struct LaneView {
  float* gQ;
  int32_t *dK, *jpos, *route, *topk_cnt, *cand_cnt, *done, *np, *ord, *cursor;
  double *dT, *lb2;  // dT: the calibration quality each query's target needs
  float *P, *out_d;
  unsigned char* scanned;
  unsigned long long *topk, *thr, *cand;
  Pair* pairs;
  int64_t* out_i;
  unsigned char* order_tmp;  // sort scratch for more than 4096 leaves
  TcQueries tq;
};

// one batch in flight on a lane
struct InFlight {
  bool active = false;
  int nb = 0;
  bool use_f = false;
  BatchGraph* g = nullptr;
  int waves = 0;
  int64_t* ids = nullptr;   // where its results go (host or device)
  float* dists = nullptr;
  const int32_t* rows = nullptr;  // scheduled batch: output row of each query (device);
                                  // ids / dists are then the call's device arrays
  int64_t row0 = 0;               // otherwise: the call's row of the batch's first query
};

// inspection: a finished batch's searched-leaf flags [nb][L] to the call's rows
// (rows[i], or row0 + i) of out [nq][L]
__global__ void scanned_out_kernel(int nb, int L, const unsigned char* __restrict__ scanned,
                                   const int32_t* __restrict__ rows, int64_t row0,
                                   unsigned char* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nb * L) return;
  const int i = (int)(t / L), l = (int)(t % L);
  const int64_t row = rows ? (int64_t)rows[i] : row0 + i;
  out[row * L + l] = scanned[t];
}

}  // namespace

// The batch pipeline of Alg. 2: batches of up to kBatch queries alternate
// between lanes (up to kSearchLanes for a search call, kServeLanes for a
// server), each with its own scratch and stream, so the preparation
// of one batch (bounds, filters, leaf order) and the host's wait for its wave
// count overlap the other batch's scan.  A full batch replays a captured graph
// of its first two waves; later waves are enqueued as the host learns that
// pairs remain.  Used by the search entry points (one call, many batches) and
// by the serving loop (batches formed from pending requests).
struct Pipeline {
  leafi_index* ix = nullptr;
  Scratch* lanes = nullptr;
  int nlanes = 1;
  int kmax = 1, W = 1, L = 0, cap = 0, qb = kBatch;
  unsigned long long* stat = nullptr;   // device counters of the pipeline's batches
                                        // (kPipelineStats)
  bool pre_p = false;                   // scheduled batches: prefix sums gathered, not computed
  unsigned char* scanned_out = nullptr; // inspection (device, nullable): [nq][L] searched flags
  leafi_search_stats st{};
  LaneView lv[kMaxLanes];
  InFlight fl[kMaxLanes];
  std::vector<double> rq_host[kMaxLanes];  // required qualities copied to each lane (kept alive
                                           // until the lane's next batch)
  SelectArgs sa;
  int cur_lane = 0;
  cudaStream_t s = nullptr;

  // size every buffer of a full batch on each lane (before any graph capture)
  void setup(leafi_index* index, Scratch* lane_array, int n_lanes, int k_max, bool any_filtered,
             unsigned long long* counters, int batch = kBatch);
  void use_lane(int li);
  void make_sa(const LaneView& v, int nb, bool use_f);
  void select(const LaneView& v);
  void round(const LaneView& v, int nb);
  void enqueue_head(const LaneView& v, int nb, bool use_f);
  BatchGraph* graph_for(const LaneView& v, int nb, bool use_f);
  void post_np(const LaneView& v);
  bool busy(int li) const { return fl[li].active; }
  // stage nb queries (rows of m floats, host or device) with their k and targets
  // (uniform: kq[0] / target[0] for all) and enqueue the batch on lane li
  void start(int li, const float* queries, int nb, const int32_t* kq, const double* target,
             bool uniform, int64_t* ids, float* dists);
  // the same for a scheduled batch: its queries are rows `rows` (device) of the
  // staged query array dQall and its results go to those rows of out_i / out_d
  void start_rows(int li, const float* dQall, const double* Pall, const int32_t* rows, int nb,
                  const int32_t* kq, const double* target, bool uniform, int64_t* out_i,
                  float* out_d);
  void launch_batch(int li, int nb, const int32_t* kq, const double* target, bool uniform,
                    bool inputs_ready = false);
  // wait for lane li's batch, run its remaining waves, deliver its results
  void finish(int li);
  // lane li's pair count has reached the host (its event completed): enqueue the
  // next wave, or deliver the results; returns true when the batch is done
  bool step(int li);
};

namespace {
}  // namespace

void Pipeline::setup(leafi_index* index, Scratch* lane_array, int n_lanes, int k_max,
                     bool any_filtered, unsigned long long* counters, int batch) {
  ix = index;
  lanes = lane_array;
  nlanes = n_lanes;
  kmax = k_max;
  stat = counters;
  const HostTree& t = ix->tree;
  L = t.n_leaves;
  // wider waves take every leaf all the same; calls without filtered queries
  // take the exact searches' own width
  W = std::min(any_filtered ? ix->wave : ix->wave_exact, std::max(L, 1));
  // the tensor-core scan merges into the top-k lists directly; the CUDA-core
  // scan appends every work item's list to a candidate buffer
  cap = tc_nbuf(ix, kmax) > 0 ? 0 : std::max(W, 1) * max_parts(ix) * kmax;
  qb = batch;
  for (int li = 0; li < nlanes; ++li) {
    Scratch& S = lanes[li];
    if (!S.st) {
      LF_CUDA(cudaStreamCreateWithFlags(&S.st, cudaStreamNonBlocking));
      LF_CUDA(cudaEventCreateWithFlags(&S.ev_np, cudaEventDisableTiming));
      LF_CUDA(cudaMallocHost(&S.h_np, sizeof(int32_t)));
    }
    LaneView& v = lv[li];
    v.gQ = S.sQ.need((size_t)qb * ix->mp);
    v.dK = S.sK.need(qb);
    v.dT = S.sTarget.need(qb);
    v.jpos = S.sJpos.need(qb);
    v.lb2 = S.sLb.need((size_t)qb * L);
    v.route = S.sRoute.need(qb);
    v.P = ix->F ? S.sPred.need((size_t)qb * ix->F) : nullptr;
    v.scanned = S.sScanned.need((size_t)qb * L);
    v.topk = S.sTopk.need((size_t)qb * kmax);
    v.topk_cnt = S.sTopkCnt.need(qb);
    v.thr = S.sThr.need(qb);
    v.cand = cap ? S.sCand.need((size_t)qb * cap) : nullptr;
    v.cand_cnt = S.sCandCnt.need(qb);
    v.done = S.sDone.need(qb);
    v.pairs = S.sPairs.need((size_t)qb * std::max(W, 1));
    v.np = S.sNpairs.need(1);
    v.out_i = S.sOutI.need((size_t)qb * kmax);
    v.out_d = S.sOutD.need((size_t)qb * kmax);
    v.ord = S.sOrd.need((size_t)qb * L);
    v.cursor = S.sCursor.need(qb);
    v.order_tmp = L > calib_max_sort() ? S.sOrderTmp.need(leaf_order_scratch(qb, L)) : nullptr;
    if (any_filtered && filter_tc(ix)) {
      S.sQs.need((size_t)2 * ((qb + 127) / 128 * 128) * ((ix->m + 31) / 32 * 32));
      S.sNeed.need((size_t)(qb + 1) * ix->F);
    }
    v.tq = TcQueries();
    if (ix->tc_scan()) {
      if (ix->scan_path == 2) v.tq.Q8 = S.sQ8.need((size_t)qb * ix->kp);
      else v.tq.Qh = S.sQh.need((size_t)qb * ix->kp);
      v.tq.Qk = S.sQk.need((size_t)2 * qb);
      S.sItemLeaf.need(std::max((size_t)qb * std::max(W, 1) * max_parts(ix),
                                (size_t)3 * ix->items_per_sm * sm_count(ix->device) + 1));
      S.sPart.need(1);
      S.sWork.need(1);
      S.sGlock.need(qb);
      S.sUb.need(qb);
      if (kmax > 1) {
        S.sNGroups.need(L);
        S.sGFirst.need(L + 1);
        S.sGBound.need((size_t)qb * std::max(W, 1) + 1);
      }
    }
    S.sCnt.need(L);
    S.sGrpOff.need(L + 1);
    S.sItemOff.need(L + 1);
    S.sGrouped.need((size_t)qb * std::max(W, 1));
    S.sNItems.need(1);
    S.sP.need((size_t)qb * 2 * (ix->m + 1));
    if (t.type == LEAFI_DSTREE) {
      S.sIv.need(ds_ivstat_doubles(qb, t.iv_s.size()));
      S.sNode.need((size_t)qb * t.n_nodes);
    } else {
      S.sPaa.need(isax_paa_doubles(qb, t.w));
    }
  }
}

void Pipeline::use_lane(int li) {
  cur_lane = li;
  ix->sc = &lanes[li];
  s = lanes[li].st;
  ix->stream = s;
}

void Pipeline::make_sa(const LaneView& v, int nb, bool use_f) {
  sa = SelectArgs();
  sa.L = L;
  sa.W = W;
  sa.nq = nb;
  sa.lb2 = v.lb2;
  sa.thr = v.thr;
  sa.F = ix->F;
  sa.leaf_filter = ix->d_leaf_filter.p;
  // STEFFEN mode: the offset table whose extra columns hold interpolated offsets
  const bool steff = ix->calib_mode == LEAFI_CALIB_STEFFEN && ix->offs.p;
  sa.alpha = steff ? ix->offs.p : ix->alpha.p;
  sa.nc = steff ? ix->offs_stride : ix->nc;
  sa.leaf_off = ix->leaf_off.p;
  sa.scanned = v.scanned;
  sa.done = v.done;
  sa.pairs = v.pairs;
  sa.npairs = v.np;
  sa.stat = stat;
  sa.P = use_f ? v.P : nullptr;
  sa.jpos = use_f ? v.jpos : nullptr;
}

void Pipeline::select(const LaneView& v) {
  LF_CUDA(cudaMemsetAsync(v.np, 0, sizeof(int32_t), s));
  ix->tick(5);
  if (W >= L)
    launch_select_all(sa, s);
  else
    launch_select_walk(sa, v.ord, v.cursor, s);
  ix->tock();
}

void Pipeline::round(const LaneView& v, int nb) {
  run_round(ix, v.gQ, v.tq, v.pairs, v.np, nb * W, nb, kmax, v.dK, v.topk, v.topk_cnt, v.thr,
            v.cand, v.cand_cnt, cap, stat + 2, stat + 3);
  select(v);
}

// everything of one batch up to (and including) the select of its first wave
void Pipeline::enqueue_head(const LaneView& v, int nb, bool use_f) {
  make_sa(v, nb, use_f);
  ix->tick(2);
  compute_bounds(ix, v.gQ, nb, v.lb2, v.route, pre_p);
  ix->tock();
  launch_query_prep(ix, v.gQ, nb, v.tq, s);
  if (W < L) launch_leaf_order(nb, L, v.lb2, v.ord, s, v.order_tmp);  // a wave of W >= L needs no order
  // per-query state and wave 0: every query searches its route leaf
  launch_batch_init(nb, L, v.route, v.scanned, ix->leaf_off.p, v.pairs, v.np, stat, v.cursor,
                    v.topk_cnt, v.thr, v.cand_cnt, v.done, v.dK, v.dT, ix->nk, ix->d_kclasses.p,
                    ix->qprime.p, ix->nc, use_f ? v.jpos : nullptr, s);
  run_round(ix, v.gQ, v.tq, v.pairs, v.np, nb, nb, kmax, v.dK, v.topk, v.topk_cnt, v.thr, v.cand,
            v.cand_cnt, cap, stat + 2, stat + 3);
  // the filters run once the route leaves have set a best-so-far: only the
  // (filter, query tile) blocks whose predictions a wave select can read
  if (use_f) {
    ix->tick(4);
    int32_t* need = lanes[cur_lane].sNeed.p;  // sized by setup for filtered calls
    if (filter_tc(ix) && need) {
      int32_t* cnt = need + (size_t)nb * ix->F;
      launch_filter_need(nb, ix->F, L, ix->d_filter_leaf.p, v.lb2, v.thr, v.scanned, v.jpos, need,
                         cnt, s);
      filter_forward(ix, v.gQ, nb, v.P, qb, need, cnt, stat + 5);
    } else {
      filter_forward(ix, v.gQ, nb, v.P, qb);
    }
    ix->tock();
  }
  select(v);
}

// a full batch of the same shape replays a captured graph of enqueue_head
// followed by its second wave and the next select (captured per lane)
BatchGraph* Pipeline::graph_for(const LaneView& v, int nb, bool use_f) {
  if (!ix->graphs_ok || nb != qb) return nullptr;
  std::vector<BatchGraph>& graphs = lanes[cur_lane].graphs;
  const unsigned long long epoch0 = g_realloc_epoch;
  for (auto& g : graphs)
    if (g.nb == nb && g.kmax == kmax && g.use_f == (int)use_f &&
        g.profiling == (int)ix->profiling && g.pre_p == (int)pre_p && g.epoch == epoch0 &&
        g.gen == ix->graph_gen)
      return &g;
  // graphs of an older epoch point at freed scratch, of an older generation
  // at replaced filters or tables: drop them
  for (size_t i = 0; i < graphs.size();) {
    BatchGraph& o = graphs[i];
    if (o.epoch == epoch0 && o.gen == ix->graph_gen) {
      ++i;
      continue;
    }
    if (o.exec) cudaGraphExecDestroy(o.exec);
    for (cudaEvent_t e : o.ev) cudaEventDestroy(e);
    graphs.erase(graphs.begin() + i);
  }
  graphs.emplace_back();
  BatchGraph& g = graphs.back();
  g.nb = nb;
  g.kmax = kmax;
  g.use_f = use_f;
  g.profiling = ix->profiling;
  g.pre_p = pre_p;
  g.epoch = epoch0;
  g.gen = ix->graph_gen;
  // the lane stream is the library's own (never the legacy default stream);
  // nothing runs while capturing
  cudaGraph_t graph = nullptr;
  ix->capturing = &g;
  const long long l0 = launches_so_far();
  bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    try {
      enqueue_head(v, nb, use_f);
      round(v, nb);
    } catch (...) {
      ok = false;
    }
    const cudaError_t e = cudaStreamEndCapture(s, &graph);
    ok = ok && e == cudaSuccess && graph;
  }
  g.launches = launches_so_far() - l0;
  count_launches(-g.launches);
  ix->capturing = nullptr;
  if (ok) ok = cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
  // a scratch buffer that grew while capturing invalidates the capture
  const bool stale = g_realloc_epoch != epoch0;
  if (!ok || stale) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (cudaEvent_t e2 : g.ev) cudaEventDestroy(e2);
    graphs.pop_back();
    // a failure without a reallocation means capture is not available here
    if (!ok && !stale) ix->graphs_ok = false;
    return nullptr;
  }
  return &g;
}

// the lane's pair count goes to its pinned word; the host waits on the event
void Pipeline::post_np(const LaneView& v) {
  Scratch& S = lanes[cur_lane];
  LF_CUDA(cudaMemcpyAsync(S.h_np, v.np, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  LF_CUDA(cudaEventRecord(S.ev_np, s));
}

void Pipeline::start(int li, const float* queries, int nb, const int32_t* kq, const double* target,
                     bool uniform, int64_t* ids, float* dists) {
  use_lane(li);
  const LaneView& v = lv[li];
  const bool dev = on_device(queries);
  if (ix->mp != ix->m) LF_CUDA(cudaMemsetAsync(v.gQ, 0, sizeof(float) * nb * ix->mp, s));
  LF_CUDA(cudaMemcpy2DAsync(v.gQ, sizeof(float) * ix->mp, queries, sizeof(float) * ix->m,
                            sizeof(float) * ix->m, (size_t)nb,
                            dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  fl[li] = InFlight();
  fl[li].ids = ids;
  fl[li].dists = dists;
  launch_batch(li, nb, kq, target, uniform);
}

void Pipeline::start_rows(int li, const float* dQall, const double* Pall, const int32_t* rows,
                          int nb, const int32_t* kq, const double* target, bool uniform,
                          int64_t* out_i, float* out_d) {
  use_lane(li);
  const LaneView& v = lv[li];
  // query rows and the call's prefix sums (computed once for scheduling) in one
  // launch, with the k and required quality of a uniform batch
  std::vector<double>& rq = rq_host[li];
  required_qualities(ix, nb, kq, target, uniform, rq);
  const int w = 2 * (ix->m + 1);
  const int64_t tot = (int64_t)nb * (ix->mp / 4) + (int64_t)nb * w + (uniform ? nb : 0);
  batch_prep_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
      dQall, Pall, rows, nb, ix->mp, w, v.gQ, lanes[li].sP.p, uniform ? 1 : 0, v.dK, v.dT, kq[0],
      rq[0]);
  LF_CHECK_LAUNCH();
  fl[li] = InFlight();
  fl[li].ids = out_i;
  fl[li].dists = out_d;
  fl[li].rows = rows;
  launch_batch(li, nb, kq, target, uniform, /*inputs_ready=*/uniform);
}

// k, targets and the batch's head (graph replay or eager) on the current lane;
// inputs_ready: k and the required qualities are already on the device
void Pipeline::launch_batch(int li, int nb, const int32_t* kq, const double* target,
                            bool uniform, bool inputs_ready) {
  const LaneView& v = lv[li];
  // the position kernel compares the tables with the quality each target needs
  std::vector<double>& rq = rq_host[li];
  if (!inputs_ready) {
    required_qualities(ix, nb, kq, target, uniform, rq);
    if (uniform) {
      fill_batch_kernel<<<(nb + 127) / 128, 128, 0, s>>>(nb, v.dK, v.dT, kq[0], rq[0]);
      LF_CHECK_LAUNCH();
    } else {
      LF_CUDA(cudaMemcpyAsync(v.dK, kq, sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s));
      LF_CUDA(cudaMemcpyAsync(v.dT, rq.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, s));
    }
  }
  InFlight& f = fl[li];
  f.active = true;
  f.nb = nb;
  f.use_f = false;
  for (int i = 0; i < (uniform ? 1 : nb); ++i) f.use_f = f.use_f || target[i] < 1.0;
  // the tensor-core forward of a pipeline counts its own predictions (stat[5])
  if (f.use_f && !(filter_tc(ix) && lanes[li].sNeed.p)) st.filter_evals += (int64_t)nb * ix->F;
  f.g = graph_for(v, nb, f.use_f);
  if (f.g) {
    LF_CUDA(cudaGraphLaunch(f.g->exec, s));
    count_launches(f.g->launches);
    st.graph_batches += 1;
    f.waves = 2;
  } else {
    enqueue_head(v, nb, f.use_f);
    f.waves = 1;
  }
  post_np(v);
}

bool Pipeline::step(int li) {
  InFlight& f = fl[li];
  use_lane(li);
  const LaneView& v = lv[li];
  make_sa(v, f.nb, f.use_f);
  Scratch& S = lanes[li];
  if (f.g && ix->profiling) {
    for (size_t i = 0; i < f.g->kind.size(); ++i) {
      float ms = 0.0f;
      LF_CUDA(cudaEventElapsedTime(&ms, f.g->ev[2 * i], f.g->ev[2 * i + 1]));
      ix->clock.ms[f.g->kind[i]] += ms;
      ix->clock.n[f.g->kind[i]] += 1;
    }
  }
  f.g = nullptr;
  if (*S.h_np != 0) {
    if (++f.waves > L + 2) fail(LEAFI_EINTERNAL, "wave loop did not terminate");
    round(v, f.nb);
    post_np(v);
    return false;
  }
  st.waves += f.waves;
  st.batches += 1;
  if (scanned_out && f.nb > 0) {
    const int64_t tot = (int64_t)f.nb * L;
    scanned_out_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(f.nb, L, v.scanned, f.rows,
                                                                      f.row0, scanned_out);
    LF_CHECK_LAUNCH();
  }
  if (f.rows) {
    launch_write_results(f.nb, kmax, v.dK, v.topk, kmax, v.topk_cnt, f.ids, f.dists, s, f.rows);
  } else {
    launch_write_results(f.nb, kmax, v.dK, v.topk, kmax, v.topk_cnt, v.out_i, v.out_d, s);
    deliver(f.ids, v.out_i, (size_t)f.nb * kmax, s);
    deliver(f.dists, v.out_d, (size_t)f.nb * kmax, s);
  }
  f.active = false;
  return true;
}

void Pipeline::finish(int li) {
  if (!fl[li].active) return;
  for (;;) {
    const auto w0 = std::chrono::steady_clock::now();
    LF_CUDA(cudaEventSynchronize(lanes[li].ev_np));
    st.host_wait_ms +=
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
    if (step(li)) return;
  }
}

namespace {

// the search entry points: one call, batches of kBatch through the index's pipeline
void search_impl(leafi_index* ix, const float* queries, int64_t nq, const std::vector<int32_t>& kq,
                 const std::vector<double>& target, int kmax, int64_t* ids, float* dists,
                 leafi_search_stats* stats, unsigned char* scanned_dev = nullptr) {
  const auto t_call = std::chrono::steady_clock::now();
  const bool any_filtered = std::any_of(target.begin(), target.end(), [](double v) { return v < 1.0; });
  if (any_filtered && (ix->nc == 0 || ix->F == 0))
    fail(LEAFI_ENOTTRAINED, "recall_target < 1 needs fitted auto-tuners");
  if (any_filtered) ensure_wsplit(ix);
  const int qb = ix->search_batch;
  const int nlanes = (int)std::min<int64_t>(ix->search_lanes, (nq + qb - 1) / qb);
  const cudaStream_t user = ix->stream;
  // every entry point after this one runs on lanes[0] and the caller's stream
  struct Restore {
    leafi_index* ix;
    cudaStream_t user;
    ~Restore() {
      ix->sc = &ix->lanes[0];
      ix->stream = user;
      ix->capturing = nullptr;
    }
  } restore{ix, user};
  unsigned long long* stat = ix->sStat.need(kPipelineStats);
  Pipeline pl;
  pl.setup(ix, ix->lanes, nlanes, kmax, any_filtered, stat, qb);
  pl.scanned_out = scanned_dev;
  const bool uniform =
      std::all_of(kq.begin(), kq.end(), [&](int32_t v) { return v == kq[0]; }) &&
      std::all_of(target.begin(), target.end(), [&](double v) { return v == target[0]; });
  // the lanes start after the caller's stream (inputs written there are visible)
  LF_CUDA(cudaMemsetAsync(stat, 0, kPipelineStats * sizeof(unsigned long long), user));
  cudaEvent_t ev_start = nullptr;
  LF_CUDA(cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming));
  struct EvGuard {
    cudaEvent_t e;
    ~EvGuard() { cudaEventDestroy(e); }
  } evg{ev_start};
  // Scheduling (a call of more than one batch): queries that route to the same
  // leaf need mostly the same leaves, so batches are cut from the queries in
  // order of their route leaf (original order among equals); each batch then
  // reads a smaller union of leaves.  Results go back to the callers' rows.
  const bool sched = ix->schedule && nq > qb;
  pl.pre_p = sched;
  const float* dQall = nullptr;
  const int32_t* dperm = nullptr;
  int64_t* out_i = ids;
  float* out_d = dists;
  std::vector<int32_t> kq_s;
  std::vector<double> tg_s;
  if (sched) {
    Schedule& sc = ix->sched;
    dQall = stage_queries(ix, queries, nq, sc.Q);
    double* P = sc.P.need((size_t)nq * 2 * (ix->m + 1));
    int32_t* keys = sc.key.need(nq);
    launch_prefix(dQall, (int)nq, ix->mp, ix->m, P, user);
    launch_route_keys(ix, P, (int)nq, keys, user);
    std::vector<int32_t> hkey(nq);
    LF_CUDA(cudaMemcpyAsync(hkey.data(), keys, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, user));
    LF_CUDA(cudaStreamSynchronize(user));
    // counting sort by route leaf (keys in [0, n_leaves]), stable
    std::vector<int32_t> perm(nq), start(ix->tree.n_leaves + 2, 0);
    for (int64_t i = 0; i < nq; ++i) start[hkey[i] + 1] += 1;
    for (size_t l = 1; l < start.size(); ++l) start[l] += start[l - 1];
    for (int64_t i = 0; i < nq; ++i) perm[start[hkey[i]]++] = (int32_t)i;
    sc.perm.upload(perm, user);
    dperm = sc.perm.p;
    if (!uniform) {
      kq_s.resize(nq);
      tg_s.resize(nq);
      for (int64_t i = 0; i < nq; ++i) {
        kq_s[i] = kq[perm[i]];
        tg_s[i] = target[perm[i]];
      }
    }
    if (!on_device(ids) || !on_device(dists)) {
      out_i = sc.out_i.need((size_t)nq * kmax);
      out_d = sc.out_d.need((size_t)nq * kmax);
    }
    LF_CUDA(cudaStreamSynchronize(user));  // the host's permuted copies are read below
  }
  LF_CUDA(cudaEventRecord(ev_start, user));
  for (int li = 0; li < nlanes; ++li) LF_CUDA(cudaStreamWaitEvent(ix->lanes[li].st, ev_start, 0));

  // The host serves whichever lane is ready: a lane whose pair count has
  // arrived gets its next wave (or delivers its results and takes the next
  // batch) at once, so no lane waits while the host is busy with another.
  int64_t next_b0 = 0;
  auto start_next = [&](int li) {
    const int64_t b0 = next_b0;
    const int nb = (int)std::min<int64_t>(qb, nq - b0);
    next_b0 += nb;
    if (sched)
      pl.start_rows(li, dQall, ix->sched.P.p, dperm + b0, nb,
                    (uniform ? kq.data() : kq_s.data() + b0),
                    (uniform ? target.data() : tg_s.data() + b0), uniform, out_i, out_d);
    else {
      pl.start(li, queries + (size_t)b0 * ix->m, nb, kq.data() + (uniform ? 0 : b0),
               target.data() + (uniform ? 0 : b0), uniform, ids + (size_t)b0 * kmax,
               dists + (size_t)b0 * kmax);
      pl.fl[li].row0 = b0;
    }
  };
  for (int li = 0; li < nlanes && next_b0 < nq; ++li) start_next(li);
  for (;;) {
    const auto t_it = std::chrono::steady_clock::now();
    bool active = false, progress = false;
    for (int li = 0; li < nlanes; ++li) {
      if (!pl.busy(li)) continue;
      active = true;
      const cudaError_t q = cudaEventQuery(ix->lanes[li].ev_np);
      if (q == cudaErrorNotReady) continue;
      LF_CUDA(q);
      progress = true;
      if (pl.step(li) && next_b0 < nq) start_next(li);
    }
    if (!active) break;
    if (!progress) {
      // nothing ready: every lane waits for the GPU
      std::this_thread::yield();
      pl.st.host_wait_ms +=
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_it).count();
    }
  }

  // the caller's stream continues after both lanes
  for (int li = 0; li < nlanes; ++li) {
    LF_CUDA(cudaEventRecord(ix->lanes[li].ev_np, ix->lanes[li].st));
    LF_CUDA(cudaStreamWaitEvent(user, ix->lanes[li].ev_np, 0));
  }
  ix->sc = &ix->lanes[0];
  ix->stream = user;
  if (sched && out_i != ids) {
    deliver(ids, out_i, (size_t)nq * kmax, user);
    deliver(dists, out_d, (size_t)nq * kmax, user);
  }
  unsigned long long h_stat[kPipelineStats] = {};
  LF_CUDA(cudaMemcpyAsync(h_stat, stat, sizeof(h_stat), cudaMemcpyDeviceToHost, user));
  const auto w_end = std::chrono::steady_clock::now();
  LF_CUDA(cudaStreamSynchronize(user));
  pl.st.host_wait_ms +=
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w_end).count();
  check_err_word(ix);
  leafi_search_stats st = pl.st;
  st.host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_call).count();
  st.leaves_scanned = (int64_t)h_stat[0];
  st.series_scanned = (int64_t)h_stat[1];
  st.distinct_series = (int64_t)h_stat[2];
  st.rechecks = (int64_t)h_stat[3];
  st.filter_pruned = (int64_t)h_stat[4];
  st.filter_evals += (int64_t)h_stat[5];
  st.lb_pruned = nq * (int64_t)ix->tree.n_leaves - st.leaves_scanned - st.filter_pruned;
  ix->settle();
  if (stats) *stats = st;
}

}  // namespace
}  // namespace leafi

using namespace leafi;

leafi::DsTables leafi_index::ds() const {
  DsTables T;
  T.n_nodes = tree.n_nodes;
  T.n_leaves = tree.n_leaves;
  T.n_iv = (int)tree.iv_s.size();
  T.root = tree.root;
  T.iv_s = iv_s.p;
  T.iv_e = iv_e.p;
  T.seg_off = seg_off.p;
  T.seg_iv = seg_iv.p;
  T.syn32 = syn32.p;
  T.left = left.p;
  T.right = right.p;
  T.node_leaf = node_leaf.p;
  T.split_iv = split_iv.p;
  T.split_sd = split_sd.p;
  T.thresh = thresh.p;
  T.path_off = path_off.p;
  T.path = path.p;
  return T;
}

void leafi_index::drop_graphs() {
  ++graph_gen;  // graphs held elsewhere (a server's lanes) are re-captured
  for (auto& lane : lanes) {
    for (auto& g : lane.graphs) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      for (cudaEvent_t e : g.ev) cudaEventDestroy(e);
    }
    lane.graphs.clear();
  }
}

size_t leafi::Scratch::bytes() const {
  return sQ.bytes() + sQh.bytes() + sQ8.bytes() + sQk.bytes() + sQs.bytes() + sItemLeaf.bytes() +
         sWork.bytes() + sP.bytes() + sIv.bytes() + sNode.bytes() + sLb.bytes() + sPaa.bytes() +
         sTarget.bytes() + sRoute.bytes() + sK.bytes() + sJpos.bytes() + sCnt.bytes() +
         sGrpOff.bytes() + sItemOff.bytes() + sNpairs.bytes() + sCandCnt.bytes() +
         sTopkCnt.bytes() + sDone.bytes() + sNItems.bytes() + sOrd.bytes() + sCursor.bytes() +
         sScanned.bytes() + sOrderTmp.bytes() + sPairs.bytes() + sGrouped.bytes() +
         sTopk.bytes() + sThr.bytes() + sCand.bytes() + sGlock.bytes() + sPart.bytes() +
         sNGroups.bytes() + sGFirst.bytes() + sGBound.bytes() + sPred.bytes() + sOutD.bytes() +
         sOutI.bytes();
}

void leafi::Scratch::release_lane() {
  if (st) cudaStreamDestroy(st);
  if (ev_np) cudaEventDestroy(ev_np);
  if (h_np) cudaFreeHost(h_np);
  st = nullptr;
  ev_np = nullptr;
  h_np = nullptr;
}

void leafi_index::tick(int kind) {
  if (!profiling || (profiling == 1 && kind != 0)) {
    ticked = false;
    return;
  }
  ticked = true;
  if (capturing) {
    cudaEvent_t a, b;
    LF_CUDA(cudaEventCreate(&a));
    LF_CUDA(cudaEventCreate(&b));
    // an external record becomes an event-record node of the graph
    LF_CUDA(cudaEventRecordWithFlags(a, stream, cudaEventRecordExternal));
    capturing->ev.push_back(a);
    capturing->ev.push_back(b);
    capturing->kind.push_back(kind);
    return;
  }
  cudaEvent_t a, b;
  LF_CUDA(cudaEventCreate(&a));
  LF_CUDA(cudaEventCreate(&b));
  LF_CUDA(cudaEventRecord(a, stream));
  clock.ev.push_back(a);
  clock.ev.push_back(b);
  clock.kind.push_back(kind);
}

void leafi_index::tock() {
  if (!ticked) return;
  if (capturing) {
    LF_CUDA(cudaEventRecordWithFlags(capturing->ev.back(), stream, cudaEventRecordExternal));
    return;
  }
  LF_CUDA(cudaEventRecord(clock.ev.back(), stream));
}

void leafi_index::settle() {
  if (clock.ev.empty()) return;
  LF_CUDA(cudaStreamSynchronize(stream));
  for (size_t i = 0; i < clock.kind.size(); ++i) {
    float ms = 0.0f;
    LF_CUDA(cudaEventElapsedTime(&ms, clock.ev[2 * i], clock.ev[2 * i + 1]));
    clock.ms[clock.kind[i]] += ms;
    clock.n[clock.kind[i]] += 1;
  }
  for (cudaEvent_t e : clock.ev) cudaEventDestroy(e);
  clock.ev.clear();
  clock.kind.clear();
}

leafi::IsaxTables leafi_index::isax() const {
  IsaxTables T;
  T.n_nodes = tree.n_nodes;
  T.n_leaves = tree.n_leaves;
  T.w = tree.w;
  T.bits = tree.bits;
  T.beta = beta.p;
  T.beta32 = beta32.p;
  T.root_child = root_child.p;
  T.left = left.p;
  T.right = right.p;
  T.node_leaf = node_leaf.p;
  T.isplit = isplit.p;
  T.node_bits = node_bits.p;
  T.lo_sym = lo_sym.p;
  T.hi_sym = hi_sym.p;
  return T;
}

extern "C" {

const char* leafi_last_error(void) { return g_last_error.c_str(); }

int64_t leafi_launch_count(void) { return (int64_t)g_launches.load(); }

leafi_status leafi_build(const float* series, int64_t n, int32_t m, const leafi_build_params* p,
                         leafi_index** out) {
  return guarded([&] {
    if (!out) fail(LEAFI_EINVAL, "out is NULL");
    *out = nullptr;
    if (!series || !p) fail(LEAFI_EINVAL, "series / params is NULL");
    if (n < 1 || n > std::numeric_limits<int32_t>::max()) fail(LEAFI_EINVAL, "n out of range");
    if (m < 1 || m > 512) fail(LEAFI_EINVAL, "m must be in [1, 512]");
    if (p->leaf_capacity < 1) fail(LEAFI_EINVAL, "leaf_capacity < 1");
    if (p->wave < 1 || p->wave > calib_max_wave()) fail(LEAFI_EINVAL, "wave must be in [1, %d]", calib_max_wave());
    if (p->scan_path < 0 || p->scan_path > 2) fail(LEAFI_EINVAL, "scan_path must be 0, 1 or 2");
    if (p->host_build < 0 || p->host_build > 1) fail(LEAFI_EINVAL, "host_build must be 0 or 1");
    if (p->index_type == LEAFI_DSTREE) {
      if (p->dstree_init_segments < 1 || p->dstree_init_segments > m)
        fail(LEAFI_EINVAL, "dstree_init_segments must be in [1, m]");
    } else if (p->index_type == LEAFI_ISAX) {
      if (p->isax_segments < 1 || p->isax_segments > 20 || m % p->isax_segments)
        fail(LEAFI_EINVAL, "isax_segments must divide m and be <= 20");
      if (p->isax_card_bits < 1 || p->isax_card_bits > 16) fail(LEAFI_EINVAL, "isax_card_bits in [1, 16]");
    } else {
      fail(LEAFI_EINVAL, "unknown index_type %d", p->index_type);
    }
    if (p->device == -1) {
      // host-only: the tree alone, for inspection (series must be host memory)
      host_alloc_gate();
      std::unique_ptr<leafi_index> ix(new leafi_index);
      ix->device = -1;
      ix->m = m;
      ix->mp = (m + 3) / 4 * 4;
      ix->n = n;
      ix->wave = ix->wave_exact = p->wave;
      if (p->index_type == LEAFI_DSTREE)
        ix->tree = build_dstree(series, n, m, p->leaf_capacity, p->dstree_init_segments);
      else
        ix->tree = build_isax(series, n, m, p->leaf_capacity, p->isax_segments, p->isax_card_bits);
      *out = ix.release();
      return;
    }
    int ndev = 0;
    LF_CUDA(cudaGetDeviceCount(&ndev));
    if (p->device < 0 || p->device >= ndev) fail(LEAFI_EINVAL, "device %d not present", p->device);
    DeviceGuard dg(p->device);
    std::unique_ptr<leafi_index> ix(new leafi_index);
    ix->device = p->device;
    ix->m = m;
    ix->mp = (m + 3) / 4 * 4;
    ix->n = n;
    ix->wave = ix->wave_exact = p->wave;
    cudaStream_t s = ix->stream;
    float* X = nullptr;
    if (!p->host_build) {
      // the tree is built on the device from the series in id order
      DBuf<float> idX;
      const float* dX = series;
      if (!on_device(series)) {
        idX.upload(series, (size_t)n * m, s);
        dX = idX.p;
      }
      if (p->index_type == LEAFI_DSTREE)
        ix->tree = build_dstree_device(dX, n, m, p->leaf_capacity, p->dstree_init_segments, s);
      else
        ix->tree = build_isax_device(dX, n, m, p->leaf_capacity, p->isax_segments,
                                     p->isax_card_bits, s);
      HostTree& t = ix->tree;
      // leaf-major, 16-byte aligned rows of mp floats, gathered on the device
      ix->ids.upload(t.order, s);
      X = ix->X.need((size_t)n * ix->mp);
      launch_gather_rows(dX, n, m, ix->ids.p, ix->mp, X, s);
      LF_CUDA(cudaStreamSynchronize(s));
    } else {
      // the tree is built on the host from a host copy of the series
      host_alloc_gate();
      std::vector<float> hostX;
      const float* hx = series;
      if (on_device(series)) {
        to_host(hostX, series, (size_t)n * m, s);
        hx = hostX.data();
      }
      if (p->index_type == LEAFI_DSTREE)
        ix->tree = build_dstree(hx, n, m, p->leaf_capacity, p->dstree_init_segments);
      else
        ix->tree = build_isax(hx, n, m, p->leaf_capacity, p->isax_segments, p->isax_card_bits);
      HostTree& t = ix->tree;
      // leaf-major, 16-byte aligned rows of mp floats, uploaded in chunks
      X = ix->X.need((size_t)n * ix->mp);
      const int64_t chunk = 1 << 16;
      std::vector<float> stage((size_t)std::min<int64_t>(chunk, n) * ix->mp, 0.0f);
      for (int64_t p0 = 0; p0 < n; p0 += chunk) {
        const int64_t cnt = std::min(chunk, n - p0);
        for (int64_t r = 0; r < cnt; ++r)
          std::memcpy(&stage[(size_t)r * ix->mp], hx + (size_t)t.order[p0 + r] * m, sizeof(float) * m);
        LF_CUDA(cudaMemcpy(X + (size_t)p0 * ix->mp, stage.data(), sizeof(float) * cnt * ix->mp,
                           cudaMemcpyHostToDevice));
      }
      ix->ids.upload(t.order, s);
    }
    HostTree& t = ix->tree;
    ix->leaf_off.upload(t.leaf_off, s);
    ix->left.upload(t.node_left, s);
    ix->right.upload(t.node_right, s);
    ix->node_leaf.upload(t.node_leaf, s);
    ix->path_off.upload(t.path_off, s);
    ix->path.upload(t.path, s);
    if (t.type == LEAFI_DSTREE) {
      ix->iv_s.upload(t.iv_s, s);
      ix->iv_e.upload(t.iv_e, s);
      ix->seg_off.upload(t.node_seg_off, s);
      ix->seg_iv.upload(t.seg_iv, s);
      std::vector<float4> syn(t.seg_mlo.size());
      for (size_t r = 0; r < syn.size(); ++r)
        syn[r] = make_float4(f32_below(t.seg_mlo[r]), f32_above(t.seg_mhi[r]),
                             f32_below(t.seg_slo[r]), f32_above(t.seg_shi[r]));
      ix->syn32.upload(syn, s);
      LF_CUDA(cudaStreamSynchronize(s));  // `syn` is released on return
      ix->split_iv.upload(t.split_iv, s);
      ix->split_sd.upload(t.split_sd, s);
      ix->thresh.upload(t.split_thresh, s);
    } else {
      ix->beta.upload(t.beta, s);
      std::vector<float2> b32(t.beta.size());
      for (size_t i = 0; i < b32.size(); ++i)
        b32[i] = make_float2(f32_below(t.beta[i]), f32_above(t.beta[i]));
      ix->beta32.upload(b32, s);
      LF_CUDA(cudaStreamSynchronize(s));  // `b32` is released on return
      ix->root_child.upload(t.root_child, s);
      ix->isplit.upload(t.isax_split, s);
      ix->node_bits.upload(t.node_bits, s);
      ix->lo_sym.upload(t.leaf_lo_sym, s);
      ix->hi_sym.upload(t.leaf_hi_sym, s);
    }
    // float16 copy for the tensor-core scan (rows of kp = m rounded up to 32)
    ix->scan_path = p->scan_path;
    ix->kp = (m + 63) / 64 * 64;
    LF_CUDA(cudaDeviceGetAttribute(&ix->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    if (ix->kp <= 256 && p->scan_path == 0) {
      __half* Xh = ix->Xh.need((size_t)n * ix->kp);
      float* xn = ix->xn.need((size_t)n);
      DBuf<unsigned int> mx;
      unsigned int zero_u = 0;
      mx.upload(&zero_u, 1, s);
      half_copy_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(X, n, ix->mp, m, ix->kp, Xh, xn, mx.p);
      LF_CHECK_LAUNCH();
      unsigned int h_mx = 0;
      LF_CUDA(cudaMemcpyAsync(&h_mx, mx.p, sizeof(h_mx), cudaMemcpyDeviceToHost, s));
      LF_CUDA(cudaStreamSynchronize(s));
      float fmx;
      std::memcpy(&fmx, &h_mx, sizeof(fmx));
      ix->tc_ok = fmx < 30000.0f && encode_xh_map(ix.get());  // float16 is safe and TMA is available
      // small-leaf packing pays only where a window of 8 leaves fits one chunk
      for (int w0 = 0; w0 < t.n_leaves && !ix->pack_small; w0 += 8)
        ix->pack_small = t.leaf_off[std::min(w0 + 8, t.n_leaves)] - t.leaf_off[w0] <= 128;
      if (!ix->tc_ok) {
        ix->Xh.release();
        ix->xn.release();
      }
    } else if (p->scan_path == 2 && (m + 127) / 128 * 128 <= 256) {
      // e4m3 operands with per-series scales: rows of m rounded up to 128 bytes
      ix->kp = (m + 127) / 128 * 128;
      unsigned char* X8 = ix->X8.need((size_t)n * ix->kp);
      float* sx = ix->sx.need((size_t)n);
      float* xn = ix->xn.need((size_t)n);
      fp8_copy_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(X, n, ix->mp, m, ix->kp, X8, sx, xn);
      LF_CHECK_LAUNCH();
      LF_CUDA(cudaStreamSynchronize(s));
      ix->tc_ok = encode_xh_map(ix.get());
      for (int w0 = 0; w0 < t.n_leaves && !ix->pack_small; w0 += 8)
        ix->pack_small = t.leaf_off[std::min(w0 + 8, t.n_leaves)] - t.leaf_off[w0] <= 128;
      if (!ix->tc_ok) {
        ix->X8.release();
        ix->sx.release();
        ix->xn.release();
      }
    }
    std::vector<int32_t> lf(t.n_leaves, -1);
    ix->d_leaf_filter.upload(lf, s);
    int32_t zero = 0;
    ix->sErr.upload(&zero, 1, s);
    LF_CUDA(cudaStreamSynchronize(s));
    *out = ix.release();
  });
}

void leafi_free(leafi_index* index) {
  if (!index) return;
  if (index->device < 0) {
    delete index;
    return;
  }
  {
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(index->device);
    if (index->stream) cudaStreamSynchronize(index->stream);
    index->drop_graphs();
    for (auto& lane : index->lanes) lane.release_lane();
    delete index;
    if (prev >= 0) cudaSetDevice(prev);
  }
}

leafi_status leafi_debug_set_lock_tries(leafi_index* index, int32_t tries) {
  return guarded([&] {
    require_device(index);
    if (tries < -1) fail(LEAFI_EINVAL, "tries must be >= -1");
    std::lock_guard<std::mutex> lk(index->mu);
    index->drop_graphs();
    index->lock_tries = tries < 0 ? kDefaultLockTries : tries;
  });
}

leafi_status leafi_debug_fail_allocations(int64_t after) {
  if (after < -1) {
    set_last_error("after must be >= -1");
    return LEAFI_EINVAL;
  }
  g_fail_alloc_countdown.store(after, std::memory_order_relaxed);
  return LEAFI_OK;
}

leafi_status leafi_set_stream(leafi_index* index, void* cuda_stream) {
  return guarded([&] {
    require_device(index);
    std::lock_guard<std::mutex> lk(index->mu);
    index->stream = static_cast<cudaStream_t>(cuda_stream);
  });
}

leafi_status leafi_set_profiling(leafi_index* index, int32_t on) {
  return guarded([&] {
    require_device(index);
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    index->drop_graphs();
    index->settle();
    index->profiling = on < 0 ? 0 : (on > 2 ? 2 : on);
    index->scan_prof.need(24);
    LF_CUDA(cudaMemset(index->scan_prof.p, 0, 20 * sizeof(unsigned long long)));
    // the current launch's timeline: min slots at the largest value, max slots at 0
    const unsigned long long init[4] = {~0ull, 0ull, ~0ull, 0ull};
    LF_CUDA(cudaMemcpy(index->scan_prof.p + 20, init, sizeof(init), cudaMemcpyHostToDevice));
    for (int i = 0; i < 8; ++i) {
      index->clock.ms[i] = 0.0;
      index->clock.n[i] = 0;
    }
  });
}

leafi_status leafi_get_kernel_times(leafi_index* index, double* ms, int64_t* launches) {
  return guarded([&] {
    require_device(index);
    if (!ms || !launches) fail(LEAFI_EINVAL, "NULL output");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    index->settle();
    for (int i = 0; i < LEAFI_KERNEL_KINDS; ++i) {
      ms[i] = index->clock.ms[i];
      launches[i] = index->clock.n[i];
    }
  });
}

leafi_status leafi_get_scan_phases(leafi_index* index, double* cycles) {
  return guarded([&] {
    require_device(index);
    if (!cycles) fail(LEAFI_EINVAL, "NULL output");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    unsigned long long h[20] = {0};
    if (index->scan_prof.p)
      LF_CUDA(cudaMemcpy(h, index->scan_prof.p, sizeof(h), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 20; ++i) cycles[i] = (double)h[i];
  });
}

leafi_status leafi_get_info(const leafi_index* index, leafi_index_info* info) {
  return guarded([&] {
    require_index(index);
    if (!info) fail(LEAFI_EINVAL, "info is NULL");
    leafi_index_info r{};
    r.n = index->n;
    r.m = index->m;
    r.index_type = index->tree.type;
    r.n_leaves = index->tree.n_leaves;
    r.n_nodes = index->tree.n_nodes;
    r.wave = index->wave;
    r.wave_exact = index->wave_exact;
    r.items_per_sm = index->items_per_sm;
    r.n_filters = index->F;
    r.filters_trained = index->trained ? 1 : 0;
    r.n_calib = index->nc;
    r.n_kclasses = index->nk;
    for (int i = 0; i < LEAFI_MAX_KCLASSES; ++i) r.kclasses[i] = index->kclasses[i];
    r.device_bytes = (int64_t)(index->X.bytes() + index->Xh.bytes() + index->X8.bytes() +
                               index->sx.bytes() + index->xn.bytes() +
                               index->ids.bytes() + index->W1t.bytes() + index->cnn.bytes());
    r.tensor_scan = index->tc_scan() ? 1 : 0;
    r.scan_row_bytes = r.tensor_scan ? index->op_row_bytes() : index->mp * 4;
    r.calib_confidence = index->calib_confidence;
    r.filter_model = index->model;
    r.filter_width = index->F ? index->h : 0;
    *info = r;
  });
}

leafi_status leafi_leaf_sizes(const leafi_index* index, int64_t* sizes) {
  return guarded([&] {
    require_index(index);
    if (!sizes) fail(LEAFI_EINVAL, "sizes is NULL");
    const HostTree& t = index->tree;
    for (int l = 0; l < t.n_leaves; ++l) sizes[l] = t.leaf_off[l + 1] - t.leaf_off[l];
  });
}

leafi_status leafi_leaf_of(const leafi_index* index, int32_t* leaf_of) {
  return guarded([&] {
    require_index(index);
    if (!leaf_of) fail(LEAFI_EINVAL, "leaf_of is NULL");
    const HostTree& t = index->tree;
    for (int l = 0; l < t.n_leaves; ++l)
      for (int64_t p = t.leaf_off[l]; p < t.leaf_off[l + 1]; ++p) leaf_of[t.order[p]] = l;
  });
}

leafi_status leafi_leaf_lower_bounds(leafi_index* index, const float* queries, int64_t nq,
                                     double* lb2) {
  return guarded([&] {
    require_device(index);
    check_queries(index, queries, nq);
    if (nq > 0 && !lb2) fail(LEAFI_EINVAL, "lb2 is NULL");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    DBuf<float> qtmp;
    const int L = index->tree.n_leaves;
    for (int64_t b0 = 0; b0 < nq; b0 += 4096) {
      const int nb = (int)std::min<int64_t>(4096, nq - b0);
      const float* dQ = stage_queries(index, queries + (size_t)b0 * index->m, nb, qtmp);
      double* out = index->sc->sLb.need((size_t)nb * L);
      compute_bounds(index, dQ, nb, out, index->sc->sRoute.need(nb));
      deliver(lb2 + (size_t)b0 * L, out, (size_t)nb * L, index->stream);
    }
    LF_CUDA(cudaStreamSynchronize(index->stream));
  });
}

leafi_status leafi_route(leafi_index* index, const float* queries, int64_t nq, int32_t* leaf) {
  return guarded([&] {
    require_device(index);
    check_queries(index, queries, nq);
    if (nq > 0 && !leaf) fail(LEAFI_EINVAL, "leaf is NULL");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    DBuf<float> qtmp;
    const int L = index->tree.n_leaves;
    for (int64_t b0 = 0; b0 < nq; b0 += 4096) {
      const int nb = (int)std::min<int64_t>(4096, nq - b0);
      const float* dQ = stage_queries(index, queries + (size_t)b0 * index->m, nb, qtmp);
      int32_t* r = index->sc->sRoute.need(nb);
      compute_bounds(index, dQ, nb, index->sc->sLb.need((size_t)nb * L), r);
      deliver(leaf + b0, r, (size_t)nb, index->stream);
    }
    LF_CUDA(cudaStreamSynchronize(index->stream));
  });
}

leafi_status leafi_select_leaves(const leafi_index* index, int32_t n_filters, int32_t* filter_leaf) {
  return guarded([&] {
    require_index(index);
    const HostTree& t = index->tree;
    if (n_filters < 0 || n_filters > t.n_leaves) fail(LEAFI_EINVAL, "n_filters out of range");
    if (n_filters > 0 && !filter_leaf) fail(LEAFI_EINVAL, "filter_leaf is NULL");
    std::vector<int32_t> idx(t.n_leaves);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
      return (t.leaf_off[a + 1] - t.leaf_off[a]) > (t.leaf_off[b + 1] - t.leaf_off[b]);
    });
    for (int i = 0; i < n_filters; ++i) filter_leaf[i] = idx[i];
  });
}

}  // extern "C"

namespace leafi {
namespace {

// Alg. 3 with this device's measured costs; the caller holds the index mutex
// and has made the index's device current
void select_auto_core(leafi_index* index, const leafi_select_params* params,
                      int32_t* filter_leaf, leafi_select_report* report) {
  const int h = params->hidden > 0 ? params->hidden : index->m;
  if (h > 4096) fail(LEAFI_EINVAL, "hidden width out of range");
  leafi_index* ix = index;
  cudaStream_t s = ix->stream;
  const HostTree& t = ix->tree;
  const int m = ix->m, mp = ix->mp;
  const int nq = (int)std::min<int64_t>(256, ix->n);
  const float* dQ = ix->X.p;  // the first nq stored series serve as probe queries
  cudaEvent_t e0, e1;
  LF_CUDA(cudaEventCreate(&e0));
  LF_CUDA(cudaEventCreate(&e1));
  struct Ev {
    cudaEvent_t a, b;
    ~Ev() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evg{e0, e1};
  auto timed = [&](auto&& body, int reps) {
    for (int i = 0; i < 2; ++i) body();
    LF_CUDA(cudaEventRecord(e0, s));
    for (int i = 0; i < reps; ++i) body();
    LF_CUDA(cudaEventRecord(e1, s));
    LF_CUDA(cudaEventSynchronize(e1));
    float ms = 0.0f;
    LF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return (double)ms / 1e3 / reps;
  };
  // t^F: 256 probe queries against 64 probe filters through the forward the
  // index uses (tensor cores when the width fits one MMA)
  const int Fp = 64;
  const int hp = (h + 15) / 16 * 16, Kq = (m + 31) / 32 * 32;
  const bool cnn = params->model == LEAFI_FILTER_CNN;
  if (params->model != LEAFI_FILTER_MLP && !cnn) fail(LEAFI_EINVAL, "unknown filter model");
  if (cnn && !cnn_fits(m, h, ix->smem_optin))
    fail(LEAFI_EINVAL, "CNN filters of %d channels at m = %d exceed shared memory", h, m);
  const bool tc = !cnn && ix->scan_path != 1 && filter_tc_fits(m, h, ix->smem_optin);
  DBuf<float> W1t, b1, w2, b2, P, Ws, Qs, theta;
  P.need((size_t)nq * Fp);
  double t_f = 0.0;
  if (cnn) {
    const size_t np = (size_t)Fp * cnn_params(h);
    LF_CUDA(cudaMemsetAsync(theta.need(np), 0, sizeof(float) * np, s));
  } else {
    LF_CUDA(cudaMemsetAsync(W1t.need((size_t)Fp * m * h), 0, sizeof(float) * Fp * m * h, s));
    LF_CUDA(cudaMemsetAsync(b1.need((size_t)Fp * h), 0, sizeof(float) * Fp * h, s));
    LF_CUDA(cudaMemsetAsync(w2.need((size_t)Fp * h), 0, sizeof(float) * Fp * h, s));
    LF_CUDA(cudaMemsetAsync(b2.need(Fp), 0, sizeof(float) * Fp, s));
  }
  if (cnn) {
    t_f = timed([&] { launch_cnn_forward(dQ, nq, mp, m, Fp, h, theta.p, P.p, s); }, 3);
  } else if (tc) {
    launch_wsplit(W1t.p, Fp, m, h, Ws.need((size_t)2 * Fp * hp * Kq), s);
    CUtensorMap wm;
    const int nqp = (nq + 127) / 128 * 128;
    Qs.need((size_t)2 * nqp * Kq);
    if (!encode_2d(&wm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, Ws.p, 32,
                   (uint64_t)2 * Fp * (Kq / 32) * hp, 128, 32, (uint32_t)hp))
      fail(LEAFI_ECUDA, "cannot encode the probe tensor map");
    t_f = timed([&] {
      launch_filter_tc(wm, dQ, nq, mp, m, Fp, h, Qs.p, b1.p, w2.p, b2.p, P.p, ix->sErr.p, s);
    }, 10);
  } else {
    t_f = timed([&] {
      launch_filter_forward(dQ, nq, mp, m, Fp, h, W1t.p, b1.p, w2.p, b2.p, P.p, s);
    }, 10);
  }
  t_f /= (double)nq * Fp;
  // t^S: the same probe queries against the largest leaf, through the scan
  int big = 0;
  for (int l = 1; l < t.n_leaves; ++l)
    if (t.leaf_off[l + 1] - t.leaf_off[l] > t.leaf_off[big + 1] - t.leaf_off[big]) big = l;
  const int64_t bigsz = t.leaf_off[big + 1] - t.leaf_off[big];
  std::vector<int32_t> lv(nq, big);
  DBuf<int32_t> dl;
  dl.upload(lv, s);
  DBuf<unsigned long long> keys;
  DBuf<int32_t> cnt;
  double t_s = timed([&] { leaf_knn_device(ix, dQ, nq, dl.p, 1, 1, keys, cnt); }, 5);
  t_s /= (double)nq * (double)bigsz;
  const double th = params->a * t_f / t_s;
  const double w = cnn ? (double)cnn_params(h) * 4.0 + 300.0 * 8.0
                      : (double)((size_t)h * m + 2 * (size_t)h + 1) * 4.0 +
                            (tc ? 2.0 * hp * Kq * 4.0 : 0.0) + 300.0 * 8.0;
  std::vector<int32_t> idx(t.n_leaves);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
    return (t.leaf_off[x + 1] - t.leaf_off[x]) > (t.leaf_off[y + 1] - t.leaf_off[y]);
  });
  double used = 0.0;
  int32_t n = 0;
  for (int j : idx) {
    if ((double)(t.leaf_off[j + 1] - t.leaf_off[j]) >= th && used + w <= (double)params->mem_cap) {
      filter_leaf[n++] = j;
      used += w;
    }
  }
  if (report) *report = leafi_select_report{t_f, t_s, th, w, n};
}

}  // namespace
}  // namespace leafi

extern "C" {

leafi_status leafi_select_leaves_auto(leafi_index* index, const leafi_select_params* params,
                                      int32_t* filter_leaf, leafi_select_report* report) {
  return guarded([&] {
    require_device(index);
    if (!params || !filter_leaf) fail(LEAFI_EINVAL, "NULL argument");
    if (!(params->a > 0.0)) fail(LEAFI_EINVAL, "a must be > 0");
    if (params->mem_cap < 0) fail(LEAFI_EINVAL, "mem_cap must be >= 0");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    select_auto_core(index, params, filter_leaf, report);
  });
}

}  // extern "C"

namespace leafi {
namespace {

// installs filters of `model` on the leaves fl (host) with hidden width (MLP)
// or channel count (CNN) h: validates the leaves, sizes the weight buffers
// (contents left to the caller), uploads the leaf <-> filter tables and clears
// training and auto-tuner state.  The caller holds the index mutex with the
// device current.
void install_filters(leafi_index* index, const std::vector<int32_t>& fl, int h,
                     int model = LEAFI_FILTER_MLP) {
  const int F = (int)fl.size();
  if (F < 1 || F > index->tree.n_leaves) fail(LEAFI_EINVAL, "F out of range");
  if (h < 1 || h > 4096) fail(LEAFI_EINVAL, "h out of range");
  if (index->m > 1024) fail(LEAFI_EINVAL, "filters support m <= 1024");
  if (model != LEAFI_FILTER_MLP && model != LEAFI_FILTER_CNN)
    fail(LEAFI_EINVAL, "unknown filter model %d", model);
  if (model == LEAFI_FILTER_CNN && !cnn_fits(index->m, h, index->smem_optin))
    fail(LEAFI_EINVAL, "CNN filters of %d channels at m = %d exceed shared memory", h, index->m);
  std::vector<int32_t> leaf_filter(index->tree.n_leaves, -1);
  for (int f = 0; f < F; ++f) {
    if (fl[f] < 0 || fl[f] >= index->tree.n_leaves) fail(LEAFI_EINVAL, "filter leaf out of range");
    if (leaf_filter[fl[f]] >= 0) fail(LEAFI_EINVAL, "leaf %d has two filters", fl[f]);
    leaf_filter[fl[f]] = f;
  }
  index->drop_graphs();
  cudaStream_t s = index->stream;
  const int m = index->m;
  if (model == LEAFI_FILTER_CNN) {
    index->cnn.need((size_t)F * cnn_params(h));
  } else {
    index->W1t.need((size_t)F * m * h);
    index->b1.need((size_t)F * h);
    index->w2.need((size_t)F * h);
    index->b2.need(F);
  }
  index->d_filter_leaf.upload(fl, s);
  index->d_leaf_filter.upload(leaf_filter, s);
  LF_CUDA(cudaStreamSynchronize(s));
  index->filter_leaf = fl;
  index->F = F;
  index->h = h;
  index->model = model;
  index->ws_dirty = true;
  index->trained = false;
  index->nc = 0;
  index->nk = 0;
  index->calib_q.release();
  index->tables_gen += 1;
}

}  // namespace
}  // namespace leafi

extern "C" {

leafi_status leafi_set_filters(leafi_index* index, const int32_t* filter_leaf, int32_t F, int32_t h,
                               const float* W1, const float* b1, const float* w2, const float* b2) {
  return guarded([&] {
    require_device(index);
    if (F < 1 || F > index->tree.n_leaves) fail(LEAFI_EINVAL, "F out of range");
    if (!filter_leaf || !W1 || !b1 || !w2 || !b2) fail(LEAFI_EINVAL, "NULL filter argument");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    cudaStream_t s = index->stream;
    std::vector<int32_t> fl;
    to_host(fl, filter_leaf, F, s);
    install_filters(index, fl, h);
    const int m = index->m;
    DBuf<float> tmp;
    const float* dW = to_device(W1, (size_t)F * h * m, tmp, s);
    const size_t tot = (size_t)F * h * m;
    transpose_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(dW, index->W1t.p, F, h, m);
    LF_CHECK_LAUNCH();
    DBuf<float> t1, t2, t3;
    const float* db1 = to_device(b1, (size_t)F * h, t1, s);
    const float* dw2 = to_device(w2, (size_t)F * h, t2, s);
    const float* db2 = to_device(b2, (size_t)F, t3, s);
    LF_CUDA(cudaMemcpyAsync(index->b1.p, db1, sizeof(float) * F * h, cudaMemcpyDeviceToDevice, s));
    LF_CUDA(cudaMemcpyAsync(index->w2.p, dw2, sizeof(float) * F * h, cudaMemcpyDeviceToDevice, s));
    LF_CUDA(cudaMemcpyAsync(index->b2.p, db2, sizeof(float) * F, cudaMemcpyDeviceToDevice, s));
    LF_CUDA(cudaStreamSynchronize(s));
  });
}

int64_t leafi_cnn_params(int32_t C) { return C >= 1 ? cnn_params(C) : 0; }

leafi_status leafi_set_cnn_filters(leafi_index* index, const int32_t* filter_leaf, int32_t F,
                                   int32_t C, const float* theta) {
  return guarded([&] {
    require_device(index);
    if (F < 1 || F > index->tree.n_leaves) fail(LEAFI_EINVAL, "F out of range");
    if (!filter_leaf || !theta) fail(LEAFI_EINVAL, "NULL filter argument");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    cudaStream_t s = index->stream;
    std::vector<int32_t> fl;
    to_host(fl, filter_leaf, F, s);
    install_filters(index, fl, C, LEAFI_FILTER_CNN);
    const size_t n = (size_t)F * cnn_params(C);
    DBuf<float> tmp;
    const float* d = to_device(theta, n, tmp, s);
    LF_CUDA(cudaMemcpyAsync(index->cnn.p, d, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    LF_CUDA(cudaStreamSynchronize(s));
  });
}

leafi_status leafi_get_cnn_filters(leafi_index* index, float* theta) {
  return guarded([&] {
    require_device(index);
    if (index->F == 0) fail(LEAFI_ENOTTRAINED, "no filters installed");
    if (!theta) fail(LEAFI_EINVAL, "NULL output");
    if (index->model != LEAFI_FILTER_CNN) fail(LEAFI_EINVAL, "the filters are not CNNs");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    deliver(theta, index->cnn.p, (size_t)index->F * cnn_params(index->h), index->stream);
    LF_CUDA(cudaStreamSynchronize(index->stream));
  });
}

leafi_status leafi_initial_cnn_weights(leafi_index* index, int32_t F, int32_t C, uint64_t seed,
                                       float* theta) {
  return guarded([&] {
    require_device(index);
    if (F < 1 || C < 1 || C > 4096) fail(LEAFI_EINVAL, "F / C out of range");
    if (!theta) fail(LEAFI_EINVAL, "NULL output");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    DBuf<float> t;
    const size_t n = (size_t)F * cnn_params(C);
    launch_gen_cnn_weights(F, C, seed, t.need(n), index->stream);
    deliver(theta, t.p, n, index->stream);
    LF_CUDA(cudaStreamSynchronize(index->stream));
  });
}

leafi_status leafi_get_filter_leaves(const leafi_index* index, int32_t* filter_leaf) {
  return guarded([&] {
    require_device(index);
    if (index->F == 0) fail(LEAFI_ENOTTRAINED, "no filters installed");
    if (!filter_leaf) fail(LEAFI_EINVAL, "NULL output");
    std::memcpy(filter_leaf, index->filter_leaf.data(), sizeof(int32_t) * index->F);
  });
}

leafi_status leafi_get_filters(leafi_index* index, float* W1, float* b1, float* w2, float* b2) {
  return guarded([&] {
    require_device(index);
    if (index->F == 0) fail(LEAFI_ENOTTRAINED, "no filters installed");
    if (!W1 || !b1 || !w2 || !b2) fail(LEAFI_EINVAL, "NULL output");
    if (index->model != LEAFI_FILTER_MLP) fail(LEAFI_EINVAL, "the filters are not MLPs");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    cudaStream_t s = index->stream;
    const int F = index->F, h = index->h, m = index->m;
    DBuf<float> tmp;
    float* d = tmp.need((size_t)F * h * m);
    const size_t tot = (size_t)F * h * m;
    transpose_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(index->W1t.p, d, F, m, h);
    LF_CHECK_LAUNCH();
    deliver(W1, d, tot, s);
    deliver(b1, index->b1.p, (size_t)F * h, s);
    deliver(w2, index->w2.p, (size_t)F * h, s);
    deliver(b2, index->b2.p, (size_t)F, s);
    LF_CUDA(cudaStreamSynchronize(s));
  });
}

leafi_status leafi_filter_predict(leafi_index* index, const float* queries, int64_t nq, float* out) {
  return guarded([&] {
    require_device(index);
    check_queries(index, queries, nq);
    if (index->F == 0) fail(LEAFI_ENOTTRAINED, "no filters installed");
    if (nq > 0 && !out) fail(LEAFI_EINVAL, "out is NULL");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    DBuf<float> qtmp;
    for (int64_t b0 = 0; b0 < nq; b0 += 4096) {
      const int nb = (int)std::min<int64_t>(4096, nq - b0);
      const float* dQ = stage_queries(index, queries + (size_t)b0 * index->m, nb, qtmp);
      float* P = index->sc->sPred.need((size_t)nb * index->F);
      ensure_wsplit(index);
      filter_forward(index, dQ, nb, P);
      deliver(out + (size_t)b0 * index->F, P, (size_t)nb * index->F, index->stream);
    }
    LF_CUDA(cudaStreamSynchronize(index->stream));
  });
}

leafi_status leafi_leaf_knn(leafi_index* index, const float* queries, int64_t nq,
                            const int32_t* leaves, int32_t nl, int32_t k, float* d2, int64_t* ids) {
  return guarded([&] {
    require_device(index);
    check_queries(index, queries, nq);
    if (k < 1 || k > LEAFI_MAX_K) fail(LEAFI_EINVAL, "k must be in [1, %d]", LEAFI_MAX_K);
    if (nl < 1 || (nq > 0 && (!leaves || !d2 || !ids))) fail(LEAFI_EINVAL, "bad leaves / outputs");
    if ((int64_t)nq * nl > std::numeric_limits<int32_t>::max() / 2) fail(LEAFI_EINVAL, "nq * nl too large");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    cudaStream_t s = index->stream;
    DBuf<float> qtmp;
    DBuf<int32_t> ltmp;
    const float* dQ = stage_queries(index, queries, nq, qtmp);
    const int32_t* dL = to_device(leaves, (size_t)nq * nl, ltmp, s);
    DBuf<unsigned long long> topk;
    DBuf<int32_t> cnt;
    leaf_knn_device(index, dQ, (int)nq, dL, nl, k, topk, cnt);
    DBuf<float> od;
    DBuf<int64_t> oi;
    const int ns = (int)(nq * nl);
    launch_leafknn_out(ns, k, topk.p, cnt.p, od.need((size_t)ns * k), oi.need((size_t)ns * k), s);
    deliver(d2, od.p, (size_t)ns * k, s);
    deliver(ids, oi.p, (size_t)ns * k, s);
    LF_CUDA(cudaStreamSynchronize(s));
  });
}

}  // extern "C"

namespace leafi {
namespace {

// Tg [ng][F] and Tl [F][nl] (Euclidean) on the device
void train_targets_device(leafi_index* ix, const float* dQg, int ng, const float* dQl, int nl,
                          float* Tg, float* Tl) {
  cudaStream_t s = ix->stream;
  const int F = ix->F;
  DBuf<unsigned long long> topk;
  DBuf<int32_t> cnt;
  DBuf<float> d2;
  DBuf<int64_t> id;
  if (ng > 0) {
    std::vector<int32_t> lv((size_t)ng * F);
    for (int g = 0; g < ng; ++g)
      for (int f = 0; f < F; ++f) lv[(size_t)g * F + f] = ix->filter_leaf[f];
    DBuf<int32_t> dl;
    dl.upload(lv, s);
    leaf_knn_device(ix, dQg, ng, dl.p, F, 1, topk, cnt);
    launch_leafknn_out(ng * F, 1, topk.p, cnt.p, d2.need((size_t)ng * F), id.need((size_t)ng * F), s);
    sqrt_kernel<<<(unsigned)(((size_t)ng * F + 255) / 256), 256, 0, s>>>(d2.p, Tg, (size_t)ng * F);
    LF_CHECK_LAUNCH();
  }
  if (nl > 0) {
    std::vector<int32_t> lv((size_t)F * nl);
    for (int f = 0; f < F; ++f)
      for (int i = 0; i < nl; ++i) lv[(size_t)f * nl + i] = ix->filter_leaf[f];
    DBuf<int32_t> dl;
    dl.upload(lv, s);
    leaf_knn_device(ix, dQl, F * nl, dl.p, 1, 1, topk, cnt);
    launch_leafknn_out(F * nl, 1, topk.p, cnt.p, d2.need((size_t)F * nl), id.need((size_t)F * nl), s);
    sqrt_kernel<<<(unsigned)(((size_t)F * nl + 255) / 256), 256, 0, s>>>(d2.p, Tl, (size_t)F * nl);
    LF_CHECK_LAUNCH();
  }
  LF_CUDA(cudaStreamSynchronize(s));
}

}  // namespace
}  // namespace leafi

extern "C" {

leafi_status leafi_train_targets(leafi_index* index, const float* Qg, int64_t ng, const float* Ql,
                                 int64_t nl, float* Tg, float* Tl) {
  return guarded([&] {
    require_device(index);
    if (index->F == 0) fail(LEAFI_ENOTTRAINED, "no filters installed");
    check_queries(index, Qg, ng);
    check_queries(index, Ql, nl * index->F);
    if ((ng > 0 && !Tg) || (nl > 0 && !Tl)) fail(LEAFI_EINVAL, "NULL output");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    cudaStream_t s = index->stream;
    DBuf<float> qg, ql, tg, tl;
    const float* dQg = ng ? stage_queries(index, Qg, ng, qg) : nullptr;
    const float* dQl = nl ? stage_queries(index, Ql, nl * index->F, ql) : nullptr;
    float* dTg = tg.need((size_t)ng * index->F);
    float* dTl = tl.need((size_t)nl * index->F);
    train_targets_device(index, dQg, (int)ng, dQl, (int)nl, dTg, dTl);
    deliver(Tg, dTg, (size_t)ng * index->F, s);
    deliver(Tl, dTl, (size_t)nl * index->F, s);
    LF_CUDA(cudaStreamSynchronize(s));
  });
}

}  // extern "C"

namespace leafi {
namespace {

// after a training launch: per-filter statistics to the host, state flags
void finish_training(leafi_index* index, int F, const int32_t* d_ep, const double* d_bv,
                     int32_t* epochs_run, double* best_val) {
  cudaStream_t s = index->stream;
  index->ws_dirty = true;
  std::vector<int32_t> hep(F);
  std::vector<double> hbv(F);
  LF_CUDA(cudaMemcpyAsync(hep.data(), d_ep, sizeof(int32_t) * F, cudaMemcpyDeviceToHost, s));
  LF_CUDA(cudaMemcpyAsync(hbv.data(), d_bv, sizeof(double) * F, cudaMemcpyDeviceToHost, s));
  LF_CUDA(cudaStreamSynchronize(s));
  if (epochs_run) std::memcpy(epochs_run, hep.data(), sizeof(int32_t) * F);
  if (best_val) std::memcpy(best_val, hbv.data(), sizeof(double) * F);
  index->trained = true;
  index->nc = 0;
  index->nk = 0;
}

// Alg. 1 target collection and training on staged queries: targets of Qg [ng][mp] and Ql
// [F][nl][mp] on the device, then SGD of every filter from its installed
// weights with one shuffle per epoch (hperm [max_epochs][n_gtrain + n_ltrain]).
// The caller holds the index mutex with the device current.
void train_core(leafi_index* index, const leafi_sgd_params* p, const float* dQg, const float* dQl,
                const std::vector<int32_t>& hperm, int32_t* epochs_run, double* best_val) {
  index->drop_graphs();
  cudaStream_t s = index->stream;
  const int F = index->F, h = index->h, m = index->m;
  const int ng = p->n_gtrain + p->n_gval, nl = p->n_ltrain + p->n_lval;
  DBuf<float> tg, tl;
  float* dTg = tg.need((size_t)ng * F);
  float* dTl = tl.need((size_t)std::max(nl, 1) * F);
  train_targets_device(index, dQg, ng, dQl, nl, dTg, dTl);
  const size_t ntr = (size_t)p->n_gtrain + p->n_ltrain;
  for (int32_t v : hperm)
    if (v < 0 || (size_t)v >= ntr) fail(LEAFI_EINVAL, "perms entry %d outside [0, %zu)", v, ntr);
  DBuf<int32_t> dperm;
  dperm.upload(hperm, s);
  DBuf<float> bW, bb1, bw2, bb2;
  // number of lr divisions before stopping: the last one keeping lr >= lr_min
  int max_decays = 0;
  {
    double lr = p->lr0;
    for (;;) {
      lr /= 10.0;
      if (lr < p->lr_min * (1.0 - 1e-9)) break;
      ++max_decays;
    }
  }
  DBuf<int32_t> dep;
  DBuf<double> dbv;
  if (index->model == LEAFI_FILTER_CNN) {
    DBuf<float> bt, gr;
    const size_t np = (size_t)F * cnn_params(h);
    CnnTrainArgs c;
    c.F = F;
    c.C = h;
    c.m = m;
    c.mp = index->mp;
    c.n_gtrain = p->n_gtrain;
    c.n_gval = p->n_gval;
    c.n_ltrain = p->n_ltrain;
    c.n_lval = p->n_lval;
    c.batch = p->batch;
    c.max_epochs = p->max_epochs;
    c.patience = p->patience;
    c.max_decays = max_decays;
    c.lr0 = (float)p->lr0;
    c.Qg = dQg;
    c.Ql = dQl;
    c.Tg = dTg;
    c.Tl = dTl;
    c.perms = dperm.p;
    c.theta = index->cnn.p;
    c.btheta = bt.need(np);
    c.grad = gr.need(np);
    c.epochs_run = dep.need(F);
    c.best_val = dbv.need(F);
    launch_cnn_train(c, s);
    finish_training(index, F, c.epochs_run, c.best_val, epochs_run, best_val);
    return;
  }
  TrainArgs a;
  a.F = F;
  a.h = h;
  a.m = m;
  a.mp = index->mp;
  a.n_gtrain = p->n_gtrain;
  a.n_gval = p->n_gval;
  a.n_ltrain = p->n_ltrain;
  a.n_lval = p->n_lval;
  a.batch = p->batch;
  a.max_epochs = p->max_epochs;
  a.patience = p->patience;
  a.max_decays = max_decays;
  a.lr0 = (float)p->lr0;
  a.Qg = dQg;
  a.Ql = dQl;
  a.Tg = dTg;
  a.Tl = dTl;
  a.perms = dperm.p;
  a.W1t = index->W1t.p;
  a.b1 = index->b1.p;
  a.w2 = index->w2.p;
  a.b2 = index->b2.p;
  a.bW1t = bW.need((size_t)F * m * h);
  a.bb1 = bb1.need((size_t)F * h);
  a.bw2 = bw2.need((size_t)F * h);
  a.bb2 = bb2.need(F);
  a.epochs_run = dep.need(F);
  a.best_val = dbv.need(F);
  launch_train(a, s);
  finish_training(index, F, a.epochs_run, a.best_val, epochs_run, best_val);
}

void check_sgd_params(const leafi_sgd_params* p) {
  if (p->n_gtrain < 0 || p->n_gval < 1 || p->n_ltrain < 0 || p->n_lval < 0 ||
      p->n_gtrain + p->n_ltrain < 1 || p->batch < 1 || p->max_epochs < 1 || p->patience < 1 ||
      !(p->lr0 > 0) || !(p->lr_min > 0) || p->lr_min > p->lr0)
    fail(LEAFI_EINVAL, "bad training parameters");
}

void check_kclasses(const int32_t* kclasses, int32_t nk) {
  if (nk < 1 || nk > LEAFI_MAX_KCLASSES || !kclasses) fail(LEAFI_EINVAL, "bad k-classes");
  for (int i = 0; i < nk; ++i) {
    if (kclasses[i] < 1 || kclasses[i] > LEAFI_MAX_K) fail(LEAFI_EINVAL, "k-class out of range");
    if (i && kclasses[i] <= kclasses[i - 1]) fail(LEAFI_EINVAL, "k-classes must ascend");
  }
}

// Alg. 4 in two steps: everything that does not depend on the wave width
// (bounds, routes, per-leaf top keys and predictions of the calibration
// queries, the sorted alpha table) and, per wave width, the search simulation
// that fills the q' tables.
struct CalibState {
  DBuf<double> lb2;
  DBuf<int32_t> route, dl, lk_cnt, ord, cnt_true;
  DBuf<unsigned long long> lk_keys, work;
  DBuf<float> P;
  DBuf<long long> hits;
  DBuf<unsigned char> order_tmp;
  CalibArgs a;
  std::vector<int32_t> kc;
};

void calib_prepare(leafi_index* index, const float* dQ, int64_t nc, const int32_t* kclasses,
                   int32_t nk, CalibState& cs) {
  if (nc < 1 || nc > calib_max_sort()) fail(LEAFI_EINVAL, "nc must be in [1, %d]", calib_max_sort());
  check_kclasses(kclasses, nk);
  const int L = index->tree.n_leaves;
  index->drop_graphs();
  cudaStream_t s = index->stream;
  const int F = index->F;
  const int kmax = kclasses[nk - 1];
  compute_bounds(index, dQ, (int)nc, cs.lb2.need((size_t)nc * L), cs.route.need(nc));
  std::vector<int32_t> lv((size_t)nc * L);
  for (int64_t c = 0; c < nc; ++c)
    for (int l = 0; l < L; ++l) lv[(size_t)c * L + l] = l;
  cs.dl.upload(lv, s);
  leaf_knn_device(index, dQ, (int)nc, cs.dl.p, L, kmax, cs.lk_keys, cs.lk_cnt);
  ensure_wsplit(index);
  filter_forward(index, dQ, (int)nc, cs.P.need((size_t)nc * F));
  CalibArgs& a = cs.a;
  a = CalibArgs();
  a.order_scratch =
      L > calib_max_sort() ? cs.order_tmp.need(leaf_order_scratch((int)nc, L)) : nullptr;
  a.nc = (int)nc;
  a.L = L;
  a.F = F;
  a.W = index->wave;
  a.lb2 = cs.lb2.p;
  a.route = cs.route.p;
  a.lk = cs.lk_keys.p;
  a.lk_stride = kmax;
  a.P = cs.P.p;
  a.filter_leaf = index->d_filter_leaf.p;
  a.leaf_filter = index->d_leaf_filter.p;
  a.alpha = index->alpha.need((size_t)F * nc);
  a.ord = cs.ord.need((size_t)nc * L);
  a.cnt_true = cs.cnt_true.need((size_t)nc * L);
  a.hits = cs.hits.need(nc);
  a.kc = 1;
  launch_calib_alpha(a, s);
  cs.kc.assign(kclasses, kclasses + nk);
}

// q' tables for wave width W (installed on the index with the k-classes)
void calib_simulate(leafi_index* index, CalibState& cs, int W) {
  cudaStream_t s = index->stream;
  CalibArgs& a = cs.a;
  const int nk = (int)cs.kc.size();
  const int64_t nc = a.nc;
  index->drop_graphs();
  double* qprime = index->qprime.need((size_t)nk * nc);
  a.W = W;
  for (int ci = 0; ci < nk; ++ci) {
    a.kc = cs.kc[ci];
    a.kk = (int)std::min<int64_t>(a.kc, index->n);
    a.work = cs.work.need(std::max((size_t)nc * nc * a.kc, (size_t)nc * a.L / 2 + 1));
    a.qprime = qprime + (size_t)ci * nc;
    launch_calib_sim(a, s);
  }
  index->d_kclasses.upload(cs.kc, s);
  LF_CUDA(cudaStreamSynchronize(s));
  index->nc = (int)nc;
  index->nk = nk;
  for (int i = 0; i < LEAFI_MAX_KCLASSES; ++i) index->kclasses[i] = i < nk ? cs.kc[i] : 0;
  index->rq_cache.clear();
  index->tables_gen += 1;
}

// Alg. 4 on staged calibration queries dQ [nc][mp] for the k-classes at the
// index's wave width; the queries are kept for later refits.  The caller holds
// the index mutex with the device current.
void fit_core(leafi_index* index, const float* dQ, int64_t nc, const int32_t* kclasses,
              int32_t nk) {
  CalibState cs;
  calib_prepare(index, dQ, nc, kclasses, nk, cs);
  calib_simulate(index, cs, index->wave);
  if (dQ != index->calib_q.p) {
    float* keep = index->calib_q.need((size_t)nc * index->mp);
    LF_CUDA(cudaMemcpyAsync(keep, dQ, sizeof(float) * nc * index->mp, cudaMemcpyDeviceToDevice,
                            index->stream));
    LF_CUDA(cudaStreamSynchronize(index->stream));
  }
}

}  // namespace
}  // namespace leafi

extern "C" {

leafi_status leafi_train_filters_on(leafi_index* index, const leafi_sgd_params* p, const float* Qg,
                                    const float* Ql, const int32_t* perms, int32_t* epochs_run,
                                    double* best_val) {
  return guarded([&] {
    require_device(index);
    if (!p || !Qg || !Ql || !perms) fail(LEAFI_EINVAL, "NULL argument");
    if (index->F == 0) fail(LEAFI_ENOTTRAINED, "no filters installed");
    check_sgd_params(p);
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    cudaStream_t s = index->stream;
    const int F = index->F;
    const int ng = p->n_gtrain + p->n_gval, nl = p->n_ltrain + p->n_lval;
    DBuf<float> qg, ql;
    const float* dQg = stage_queries(index, Qg, ng, qg);
    const float* dQl = stage_queries(index, Ql, (int64_t)F * nl, ql);
    std::vector<int32_t> hperm;
    to_host(hperm, perms, (size_t)p->max_epochs * (p->n_gtrain + p->n_ltrain), s);
    train_core(index, p, dQg, dQl, hperm, epochs_run, best_val);
  });
}

leafi_status leafi_fit_autotuners(leafi_index* index, const float* Qc, int64_t nc,
                                  const int32_t* kclasses, int32_t nk) {
  return guarded([&] {
    require_device(index);
    if (index->F == 0) fail(LEAFI_ENOTTRAINED, "no filters installed");
    check_queries(index, Qc, nc);
    if (nc < 1 || nc > calib_max_sort()) fail(LEAFI_EINVAL, "nc must be in [1, %d]", calib_max_sort());
    check_kclasses(kclasses, nk);
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    DBuf<float> qtmp;
    const float* dQ = stage_queries(index, Qc, nc, qtmp);
    fit_core(index, dQ, nc, kclasses, nk);
  });
}

}  // extern "C"

namespace leafi {
namespace {

struct Alg1Counts {
  int ng, nl, n_gtrain, n_gval, n_ltrain, n_lval;
};

Alg1Counts alg1_counts(const leafi_train_params* p) {
  if (p->n_train < 2 || !(p->global_local_ratio > 0.0) || !(p->val_frac > 0.0) ||
      !(p->val_frac < 1.0) || !(p->noise_lo >= 0.0) || !(p->noise_hi >= p->noise_lo))
    fail(LEAFI_EINVAL, "bad training-query parameters");
  Alg1Counts c;
  const double r = p->global_local_ratio;
  // an infinite ratio means global queries only (the paper's ablation without local data)
  c.ng = std::isinf(r) ? p->n_train : (int)std::floor((double)p->n_train * r / (r + 1.0) + 0.5);
  c.ng = std::min(std::max(c.ng, 2), p->n_train);
  c.nl = p->n_train - c.ng;
  c.n_gval = std::min(std::max((int)std::floor(p->val_frac * c.ng + 0.5), 1), c.ng - 1);
  c.n_gtrain = c.ng - c.n_gval;
  c.n_lval = std::min((int)std::floor(p->val_frac * c.nl + 0.5), c.nl);
  c.n_ltrain = c.nl - c.n_lval;
  return c;
}

// Alg. 1 GenerateGlobalQueries / GenerateLocalQueries for the leaves fl: rows [ng + F*nl][mp] of out, the
// global queries first, then filter by filter; picks (original ids) to gpick
// [ng] and lpick [F][nl] when given.  Caller holds the mutex, device current.
void generate_training_queries(leafi_index* ix, const leafi_train_params* p, const Alg1Counts& c,
                               const std::vector<int32_t>& fl, DBuf<float>& out,
                               std::vector<int64_t>* gpick, std::vector<int64_t>* lpick) {
  const HostTree& t = ix->tree;
  const int F = (int)fl.size();
  cudaStream_t s = ix->stream;
  const int64_t rows = (int64_t)c.ng + (int64_t)F * c.nl;
  if (rows > (int64_t)std::numeric_limits<int32_t>::max() / 2)
    fail(LEAFI_EINVAL, "too many training queries");
  if ((int64_t)c.ng > t.n) fail(LEAFI_EINVAL, "more global queries (%d) than series", c.ng);
  std::vector<int64_t> pos((size_t)rows);
  // global picks: distinct original ids, then their storage positions
  std::vector<int64_t> g((size_t)c.ng);
  gen_floyd(p->seed, kTagGPick, 0, (uint64_t)t.n, c.ng, g.data());
  {
    std::unordered_map<int64_t, std::vector<int>> want;
    want.reserve((size_t)c.ng * 2);
    for (int i = 0; i < c.ng; ++i) want[g[i]].push_back(i);
    for (int64_t q = 0; q < t.n; ++q) {
      auto it = want.find(t.order[q]);
      if (it != want.end())
        for (int i : it->second) pos[i] = q;
    }
  }
  // local picks: ranks among a leaf's members (ascending ids = storage order)
  std::vector<int64_t> r((size_t)c.nl);
  if (lpick) lpick->assign((size_t)F * c.nl, 0);
  for (int f = 0; f < F; ++f) {
    const int64_t lo = t.leaf_off[fl[f]], sz = t.leaf_off[fl[f] + 1] - lo;
    if (sz >= c.nl)
      gen_floyd(p->seed, kTagLPick, (uint32_t)(1 + f), (uint64_t)sz, c.nl, r.data());
    else
      gen_with_replacement(p->seed, kTagLPick, (uint32_t)(1 + f), (uint64_t)sz, c.nl, r.data());
    for (int i = 0; i < c.nl; ++i) {
      pos[(size_t)c.ng + (size_t)f * c.nl + i] = lo + r[i];
      if (lpick) (*lpick)[(size_t)f * c.nl + i] = t.order[lo + r[i]];
    }
  }
  if (gpick) *gpick = g;
  DBuf<int64_t> dpos;
  dpos.upload(pos, s);
  launch_gen_queries(ix->X.p, ix->mp, ix->m, dpos.p, c.ng, c.nl, F, p->seed, p->noise_lo,
                     p->noise_hi, out.need((size_t)std::max<int64_t>(rows, 1) * ix->mp), s);
  LF_CUDA(cudaStreamSynchronize(s));
}

double seconds_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// the search-schedule autotuner (leafi_tune_search); caller holds the mutex.
// Exact mode times exact searches and sets the exact searches' wave width (and
// the index's while no tables are fitted); LeaFi mode times searches at the
// target after refitting the tables for every candidate wave width.
void tune_core(leafi_index* ix, const leafi_tune_params* p, leafi_tune_report* rep) {
  const bool leafi_mode = p->target > 0.0 && p->target < 1.0;
  if (p->n_probe < 1 || p->k < 1 || p->k > LEAFI_MAX_K || p->reps < 1 || p->n_waves < 0 ||
      p->n_waves > 8 || p->n_items < 0 || p->n_items > 4 || !(p->target >= 0.0))
    fail(LEAFI_EINVAL, "bad tuning parameters");
  if (leafi_mode && (ix->F == 0 || ix->nc == 0 || !ix->calib_q.p))
    fail(LEAFI_EINVAL, "LeaFi-mode tuning needs auto-tuners fitted from calibration queries");
  const int L = ix->tree.n_leaves;
  std::vector<int> waves, items;
  if (p->n_waves) waves.assign(p->waves, p->waves + p->n_waves);
  else waves = {16, 32, 64, 128, 256, 1024, L};
  if (p->n_items) items.assign(p->items_per_sm, p->items_per_sm + p->n_items);
  else items = {2, 4, 8};
  for (int& w : waves) {
    if (w < 1 || w > calib_max_wave()) fail(LEAFI_EINVAL, "wave %d out of range", w);
    w = std::min(w, std::max(L, 1));  // wider waves all take every leaf
  }
  std::sort(waves.begin(), waves.end());
  waves.erase(std::unique(waves.begin(), waves.end()), waves.end());
  for (int v : items)
    if (v < 0 || v > 64) fail(LEAFI_EINVAL, "items per SM %d out of range", v);
  // probe queries: the generator's global draw under a seed of their own
  leafi_train_params gp{};
  gp.n_train = p->n_probe;
  gp.global_local_ratio = std::numeric_limits<double>::infinity();
  gp.noise_lo = p->noise_lo;
  gp.noise_hi = p->noise_hi;
  gp.seed = p->seed ^ 0x6a09e667f3bcc909ull;
  Alg1Counts c{p->n_probe, 0, p->n_probe, 0, 0, 0};
  DBuf<float> Qp, Qm;
  generate_training_queries(ix, &gp, c, {}, Qp, nullptr, nullptr);
  const float* dQ = Qp.p;
  if (ix->mp != ix->m) {
    LF_CUDA(cudaMemcpy2DAsync(Qm.need((size_t)p->n_probe * ix->m), sizeof(float) * ix->m, Qp.p,
                              sizeof(float) * ix->mp, sizeof(float) * ix->m, (size_t)p->n_probe,
                              cudaMemcpyDeviceToDevice, ix->stream));
    dQ = Qm.p;
  }
  DBuf<int64_t> oi;
  DBuf<float> od;
  oi.need((size_t)p->n_probe * p->k);
  od.need((size_t)p->n_probe * p->k);
  std::vector<int32_t> kq(p->n_probe, p->k);
  std::vector<double> tg(p->n_probe, leafi_mode ? p->target : 1.0);
  // LeaFi mode: the wave-independent half of Alg. 4, from the kept queries
  CalibState cs;
  int fitted_w = ix->wave;
  if (leafi_mode) {
    const std::vector<int32_t> kc(ix->kclasses, ix->kclasses + ix->nk);
    calib_prepare(ix, ix->calib_q.p, ix->nc, kc.data(), ix->nk, cs);
  }
  int& wave = leafi_mode ? ix->wave : ix->wave_exact;
  const int w0 = wave, i0 = ix->items_per_sm;
  auto install = [&](int w, int ips) {
    if (w != wave || ips != ix->items_per_sm) ix->drop_graphs();
    wave = w;
    ix->items_per_sm = ips;
    if (leafi_mode && fitted_w != w) {
      calib_simulate(ix, cs, w);
      fitted_w = w;
    }
  };
  auto time_it = [&](int w, int ips) {
    install(w, ips);
    search_impl(ix, dQ, p->n_probe, kq, tg, p->k, oi.p, od.p, nullptr);  // warm-up
    double best = std::numeric_limits<double>::infinity();
    for (int r = 0; r < p->reps; ++r) {
      const auto t0 = std::chrono::steady_clock::now();
      search_impl(ix, dQ, p->n_probe, kq, tg, p->k, oi.p, od.p, nullptr);
      best = std::min(best, seconds_since(t0) * 1e3);
    }
    return best;
  };
  leafi_tune_report r{};
  try {
    r.ms_before = time_it(w0, i0);
    int bw = w0, bi = i0;
    double bms = r.ms_before;
    for (int w : waves)
      for (int v : items) {
        const double ms = time_it(w, v);
        if (r.n_tried < 32) {
          r.tried_wave[r.n_tried] = w;
          r.tried_items[r.n_tried] = v;
          r.tried_ms[r.n_tried] = ms;
          ++r.n_tried;
        }
        if (ms < bms) {
          bms = ms;
          bw = w;
          bi = v;
        }
      }
    install(bw, bi);
    // exact mode on an index without tables sets the width of every call
    if (!leafi_mode && ix->nc == 0) ix->wave = bw;
    r.wave = bw;
    r.items_per_sm = bi;
    r.ms_best = bms;
  } catch (...) {
    ix->drop_graphs();
    ix->items_per_sm = i0;
    wave = w0;
    if (leafi_mode && fitted_w != w0) calib_simulate(ix, cs, w0);
    throw;
  }
  if (rep) *rep = r;
}

leafi_tune_params default_tune_params(uint64_t seed) {
  leafi_tune_params t{};
  t.n_probe = 8192;
  t.k = 1;
  t.noise_lo = 0.1;
  t.noise_hi = 0.4;
  t.seed = seed;
  t.reps = 3;
  t.target = 1.0;
  return t;
}

}  // namespace
}  // namespace leafi

extern "C" {

leafi_status leafi_train_filters(leafi_index* index, const leafi_train_params* p,
                                 int32_t* epochs_run, double* best_val,
                                 leafi_train_report* report) {
  return guarded([&] {
    require_device(index);
    if (!p) fail(LEAFI_EINVAL, "params is NULL");
    const Alg1Counts c = alg1_counts(p);
    leafi_sgd_params sp{c.n_gtrain, c.n_gval, c.n_ltrain, c.n_lval, p->batch, p->max_epochs,
                        p->patience, p->lr0, p->lr_min};
    check_sgd_params(&sp);
    check_kclasses(p->kclasses, p->n_kclasses);
    if (!(p->confidence >= 0.0 && p->confidence < 1.0)) fail(LEAFI_EINVAL, "confidence must be in [0, 1)");
    if (c.n_gval > calib_max_sort())
      fail(LEAFI_EINVAL, "calibration set of %d queries exceeds %d", c.n_gval, calib_max_sort());
    const int L = index->tree.n_leaves;
    if (p->n_filters == 0 || p->n_filters < -1 || p->n_filters > L)
      fail(LEAFI_EINVAL, "n_filters must be -1 or in [1, %d]", L);
    const int h = p->hidden > 0 ? p->hidden : index->m;
    if (p->model != LEAFI_FILTER_MLP && p->model != LEAFI_FILTER_CNN)
      fail(LEAFI_EINVAL, "unknown filter model %d", p->model);
    if (p->calib_mode != LEAFI_CALIB_STEP && p->calib_mode != LEAFI_CALIB_STEFFEN)
      fail(LEAFI_EINVAL, "unknown calibration mode %d", p->calib_mode);
    if (p->model == LEAFI_FILTER_CNN && !cnn_fits(index->m, h, index->smem_optin))
      fail(LEAFI_EINVAL, "CNN filters of %d channels at m = %d exceed shared memory", h, index->m);
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    cudaStream_t s = index->stream;
    leafi_train_report rep{};
    auto t0 = std::chrono::steady_clock::now();
    // SelectLeafNodes
    std::vector<int32_t> fl;
    if (p->n_filters > 0) {
      std::vector<int32_t> idx(L);
      std::iota(idx.begin(), idx.end(), 0);
      const HostTree& t = index->tree;
      std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
        return (t.leaf_off[x + 1] - t.leaf_off[x]) > (t.leaf_off[y + 1] - t.leaf_off[y]);
      });
      fl.assign(idx.begin(), idx.begin() + p->n_filters);
    } else {
      if (!(p->a > 0.0) || p->mem_cap < 0) fail(LEAFI_EINVAL, "bad Alg. 3 parameters");
      leafi_select_params sel{p->a, p->mem_cap, h, p->model};
      leafi_select_report sr{};
      std::vector<int32_t> all(L);
      select_auto_core(index, &sel, all.data(), &sr);
      if (sr.n_selected < 1) fail(LEAFI_EINVAL, "Alg. 3 selected no leaf (threshold %.1f)", sr.threshold);
      fl.assign(all.begin(), all.begin() + sr.n_selected);
      rep.select_threshold = sr.threshold;
    }
    rep.seconds_select = seconds_since(t0);
    t0 = std::chrono::steady_clock::now();
    install_filters(index, fl, h, p->model);
    const int F = (int)fl.size();
    if (p->model == LEAFI_FILTER_CNN)
      launch_gen_cnn_weights(F, h, p->seed, index->cnn.p, s);
    else
      launch_gen_weights(F, h, index->m, p->seed, index->W1t.p, index->b1.p, index->w2.p,
                         index->b2.p, s);
    // GenerateGlobalQueries / GenerateLocalQueries
    DBuf<float> Q;
    generate_training_queries(index, p, c, fl, Q, nullptr, nullptr);
    std::vector<int32_t> hperm((size_t)p->max_epochs * (c.n_gtrain + c.n_ltrain));
    gen_epoch_perms(p->max_epochs, c.n_gtrain + c.n_ltrain, p->seed, hperm.data());
    rep.seconds_generate = seconds_since(t0);
    t0 = std::chrono::steady_clock::now();
    // targets and training
    const float* dQg = Q.p;
    const float* dQl = Q.p + (size_t)c.ng * index->mp;
    std::vector<int32_t> ep(F);
    std::vector<double> bv(F);
    train_core(index, &sp, dQg, dQl, hperm, ep.data(), bv.data());
    rep.seconds_train = seconds_since(t0);
    t0 = std::chrono::steady_clock::now();
    // the exact searches' schedule
    if (p->tune_search) {
      const leafi_tune_params tp = default_tune_params(p->seed);
      tune_core(index, &tp, nullptr);
    }
    // auto-tuners on the calibration set (the global validation queries)
    index->calib_confidence = p->confidence;
    index->calib_mode = p->calib_mode;
    fit_core(index, dQg + (size_t)c.n_gtrain * index->mp, c.n_gval, p->kclasses, p->n_kclasses);
    // the LeaFi searches' schedule (the tables are refitted for each candidate)
    if (p->tune_search) {
      leafi_tune_params tp = default_tune_params(p->seed);
      tp.target = 0.99;
      tune_core(index, &tp, nullptr);
    }
    index->rq_cache.clear();
    rep.seconds_calibrate = seconds_since(t0);
    rep.n_filters = F;
    rep.n_gtrain = c.n_gtrain;
    rep.n_gval = c.n_gval;
    rep.n_ltrain = c.n_ltrain;
    rep.n_lval = c.n_lval;
    if (epochs_run) std::memcpy(epochs_run, ep.data(), sizeof(int32_t) * F);
    if (best_val) std::memcpy(best_val, bv.data(), sizeof(double) * F);
    if (report) *report = rep;
  });
}

leafi_status leafi_tune_search(leafi_index* index, const leafi_tune_params* params,
                               leafi_tune_report* report) {
  return guarded([&] {
    require_device(index);
    if (!params) fail(LEAFI_EINVAL, "params is NULL");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    tune_core(index, params, report);
  });
}

leafi_status leafi_training_queries(leafi_index* index, const leafi_train_params* p,
                                    const int32_t* filter_leaf, int32_t F, float* Qg, float* Ql,
                                    int64_t* gpick, int64_t* lpick) {
  return guarded([&] {
    require_device(index);
    if (!p || !Qg || (F > 0 && (!filter_leaf || !Ql))) fail(LEAFI_EINVAL, "NULL argument");
    const Alg1Counts c = alg1_counts(p);
    if (F < 0 || F > index->tree.n_leaves) fail(LEAFI_EINVAL, "F out of range");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    cudaStream_t s = index->stream;
    std::vector<int32_t> fl;
    to_host(fl, filter_leaf, F, s);
    for (int32_t l : fl)
      if (l < 0 || l >= index->tree.n_leaves) fail(LEAFI_EINVAL, "filter leaf out of range");
    DBuf<float> Q;
    std::vector<int64_t> gp, lp;
    generate_training_queries(index, p, c, fl, Q, &gp, &lp);
    const int m = index->m, mp = index->mp;
    LF_CUDA(cudaMemcpy2DAsync(Qg, sizeof(float) * m, Q.p, sizeof(float) * mp, sizeof(float) * m,
                              (size_t)c.ng, on_device(Qg) ? cudaMemcpyDeviceToDevice
                                                          : cudaMemcpyDeviceToHost, s));
    if (F > 0 && c.nl > 0)
      LF_CUDA(cudaMemcpy2DAsync(Ql, sizeof(float) * m, Q.p + (size_t)c.ng * mp, sizeof(float) * mp,
                                sizeof(float) * m, (size_t)F * c.nl,
                                on_device(Ql) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                s));
    LF_CUDA(cudaStreamSynchronize(s));
    if (gpick) std::memcpy(gpick, gp.data(), sizeof(int64_t) * gp.size());
    if (lpick && !lp.empty()) std::memcpy(lpick, lp.data(), sizeof(int64_t) * lp.size());
  });
}

leafi_status leafi_initial_weights(leafi_index* index, int32_t F, int32_t h, uint64_t seed,
                                   float* W1, float* b1, float* w2, float* b2) {
  return guarded([&] {
    require_device(index);
    if (F < 1 || h < 1 || h > 4096) fail(LEAFI_EINVAL, "F / h out of range");
    if (!W1 || !b1 || !w2 || !b2) fail(LEAFI_EINVAL, "NULL output");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    cudaStream_t s = index->stream;
    const int m = index->m;
    const size_t tot = (size_t)F * h * m;
    DBuf<float> wt, w, bb1, ww2, bb2;
    launch_gen_weights(F, h, m, seed, wt.need(tot), bb1.need((size_t)F * h),
                       ww2.need((size_t)F * h), bb2.need(F), s);
    transpose_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(wt.p, w.need(tot), F, m, h);
    LF_CHECK_LAUNCH();
    deliver(W1, w.p, tot, s);
    deliver(b1, bb1.p, (size_t)F * h, s);
    deliver(w2, ww2.p, (size_t)F * h, s);
    deliver(b2, bb2.p, (size_t)F, s);
    LF_CUDA(cudaStreamSynchronize(s));
  });
}

leafi_status leafi_epoch_permutations(int32_t epochs, int32_t n, uint64_t seed, int32_t* perms) {
  return guarded([&] {
    if (epochs < 0 || n < 0 || (epochs > 0 && n > 0 && !perms)) fail(LEAFI_EINVAL, "bad arguments");
    if (on_device(perms)) fail(LEAFI_EINVAL, "perms must be host memory");
    gen_epoch_perms(epochs, n, seed, perms);
  });
}

leafi_status leafi_znormalize(const float* x, int64_t n, int32_t m, float* out, int32_t device) {
  return guarded([&] {
    if (n < 0 || m < 1 || (n > 0 && (!x || !out))) fail(LEAFI_EINVAL, "bad arguments");
    int ndev = 0;
    LF_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) fail(LEAFI_EINVAL, "device %d out of range", device);
    if (n == 0) return;
    DeviceGuard dg(device);
    cudaStream_t s = nullptr;
    LF_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct St {
      cudaStream_t s;
      ~St() { cudaStreamDestroy(s); }
    } st{s};
    // host rows go through the device in slabs of up to 256 MiB
    const int64_t per = std::max<int64_t>(1, (int64_t)(256 << 20) / ((int64_t)m * 8));
    DBuf<float> a, b;
    const bool din = on_device(x), dout = on_device(out);
    for (int64_t r0 = 0; r0 < n; r0 += per) {
      const int64_t nb = std::min(per, n - r0);
      const float* src = x + r0 * m;
      if (!din) {
        a.upload(src, (size_t)nb * m, s);
        src = a.p;
      }
      float* dst = dout ? out + r0 * m : b.need((size_t)nb * m);
      launch_znorm(src, m, nb, m, dst, m, s);
      if (!dout)
        LF_CUDA(cudaMemcpyAsync(out + r0 * m, dst, sizeof(float) * nb * m, cudaMemcpyDeviceToHost,
                                s));
      LF_CUDA(cudaStreamSynchronize(s));
    }
  });
}

leafi_status leafi_set_search_lanes(leafi_index* index, int32_t lanes) {
  return guarded([&] {
    require_device(index);
    if (lanes < 1 || lanes > kSearchLanes) fail(LEAFI_EINVAL, "lanes must be in [1, %d]", kSearchLanes);
    std::lock_guard<std::mutex> lk(index->mu);
    index->search_lanes = lanes;
  });
}

leafi_status leafi_set_scan_part(leafi_index* index, int32_t rows, int32_t items_per_sm,
                                 int32_t min_rows, int32_t blocks) {
  return guarded([&] {
    require_device(index);
    if (rows < 128 || rows > 8192 || rows % 128) fail(LEAFI_EINVAL, "rows must be a multiple of 128 in [128, 8192]");
    if (items_per_sm < 0 || items_per_sm > 64) fail(LEAFI_EINVAL, "items_per_sm must be in [0, 64]");
    if (min_rows < 128 || min_rows > 8192 || min_rows % 128)
      fail(LEAFI_EINVAL, "min_rows must be a multiple of 128 in [128, 8192]");
    if (blocks < 0 || blocks > 4096) fail(LEAFI_EINVAL, "blocks must be in [0, 4096]");
    std::lock_guard<std::mutex> lk(index->mu);
    index->drop_graphs();
    index->part = rows;
    index->items_per_sm = items_per_sm;
    index->min_part = min_rows;
    index->scan_blocks = blocks;
  });
}

leafi_status leafi_set_search_batch(leafi_index* index, int32_t queries) {
  return guarded([&] {
    require_device(index);
    if (queries < 1 || queries > kMaxBatch) fail(LEAFI_EINVAL, "queries must be in [1, %d]", kMaxBatch);
    std::lock_guard<std::mutex> lk(index->mu);
    index->drop_graphs();
    index->search_batch = queries;
  });
}

leafi_status leafi_set_query_schedule(leafi_index* index, int32_t on) {
  return guarded([&] {
    require_device(index);
    std::lock_guard<std::mutex> lk(index->mu);
    index->schedule = on != 0;
  });
}

leafi_status leafi_set_calibration_confidence(leafi_index* index, double confidence) {
  return guarded([&] {
    require_device(index);
    if (!(confidence >= 0.0 && confidence < 1.0)) fail(LEAFI_EINVAL, "confidence must be in [0, 1)");
    std::lock_guard<std::mutex> lk(index->mu);
    index->calib_confidence = confidence;
    index->rq_cache.clear();
  });
}

leafi_status leafi_set_calibration_mode(leafi_index* index, int32_t mode) {
  return guarded([&] {
    require_device(index);
    if (mode != LEAFI_CALIB_STEP && mode != LEAFI_CALIB_STEFFEN)
      fail(LEAFI_EINVAL, "unknown calibration mode %d", mode);
    std::lock_guard<std::mutex> lk(index->mu);
    index->drop_graphs();
    index->calib_mode = mode;
  });
}

leafi_status leafi_calibration_offsets(leafi_index* index, int32_t k, double recall_target,
                                       double* offsets, int32_t* uses_filters) {
  return guarded([&] {
    require_device(index);
    if (index->nc == 0 || index->F == 0) fail(LEAFI_ENOTTRAINED, "no auto-tuners fitted");
    if (!offsets) fail(LEAFI_EINVAL, "NULL output");
    if (k < 1 || k > LEAFI_MAX_K) fail(LEAFI_EINVAL, "k must be in [1, %d]", LEAFI_MAX_K);
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    std::vector<double> rq;
    required_qualities(index, 1, &k, &recall_target, true, rq);
    const int F = index->F;
    int use = 0;
    std::vector<double> col(F);
    if (rq[0] < 0.0) {
      // STEFFEN: the query's column of the offset table
      const int c = (int)(-rq[0]) - 1;
      LF_CUDA(cudaMemcpy2DAsync(col.data(), sizeof(double), index->offs.p + c,
                                sizeof(double) * index->offs_stride, sizeof(double), (size_t)F,
                                cudaMemcpyDeviceToHost, index->stream));
      LF_CUDA(cudaStreamSynchronize(index->stream));
      use = 1;
    } else if (rq[0] <= 1.0) {
      // STEP: the last position whose quality reaches rq, as the position kernel takes it
      int c = -1;
      for (int z = 0; z < index->nk; ++z)
        if (index->kclasses[z] >= k) {
          c = z;
          break;
        }
      const int nc = index->nc;
      std::vector<double> qp(nc), a((size_t)F * nc);
      LF_CUDA(cudaMemcpyAsync(qp.data(), index->qprime.p + (size_t)c * nc, sizeof(double) * nc,
                              cudaMemcpyDeviceToHost, index->stream));
      LF_CUDA(cudaMemcpyAsync(a.data(), index->alpha.p, sizeof(double) * F * nc,
                              cudaMemcpyDeviceToHost, index->stream));
      LF_CUDA(cudaStreamSynchronize(index->stream));
      int j = nc - 1;
      for (int i = 0; i < nc; ++i)
        if (!(qp[i] >= rq[0])) {
          j = i - 1;
          break;
        }
      if (j >= 0) {
        for (int f = 0; f < F; ++f) col[f] = a[(size_t)f * nc + j];
        use = 1;
      }
    }
    if (use) std::memcpy(offsets, col.data(), sizeof(double) * F);
    if (uses_filters) *uses_filters = use;
  });
}

leafi_status leafi_get_autotuners(leafi_index* index, double* alpha_sorted, double* qprime) {
  return guarded([&] {
    require_device(index);
    if (index->nc == 0) fail(LEAFI_ENOTTRAINED, "no auto-tuners fitted");
    if (!alpha_sorted || !qprime) fail(LEAFI_EINVAL, "NULL output");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    deliver(alpha_sorted, index->alpha.p, (size_t)index->F * index->nc, index->stream);
    deliver(qprime, index->qprime.p, (size_t)index->nk * index->nc, index->stream);
    LF_CUDA(cudaStreamSynchronize(index->stream));
  });
}

leafi_status leafi_set_autotuners(leafi_index* index, const double* alpha_sorted,
                                  const double* qprime, int64_t nc, const int32_t* kclasses,
                                  int32_t nk) {
  return guarded([&] {
    require_device(index);
    if (index->F == 0) fail(LEAFI_ENOTTRAINED, "no filters installed");
    if (!alpha_sorted || !qprime || !kclasses) fail(LEAFI_EINVAL, "NULL argument");
    if (nc < 1 || nc > (1 << 24)) fail(LEAFI_EINVAL, "nc out of range");
    if (nk < 1 || nk > LEAFI_MAX_KCLASSES) fail(LEAFI_EINVAL, "bad k-classes");
    std::vector<int32_t> kc;
    to_host(kc, kclasses, nk, index->stream);
    for (int i = 0; i < nk; ++i)
      if (kc[i] < 1 || kc[i] > LEAFI_MAX_K || (i && kc[i] <= kc[i - 1])) fail(LEAFI_EINVAL, "bad k-classes");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    index->drop_graphs();
    cudaStream_t s = index->stream;
    DBuf<double> t1, t2;
    const double* da = to_device(alpha_sorted, (size_t)index->F * nc, t1, s);
    const double* dq = to_device(qprime, (size_t)nk * nc, t2, s);
    LF_CUDA(cudaMemcpyAsync(index->alpha.need((size_t)index->F * nc), da,
                            sizeof(double) * index->F * nc, cudaMemcpyDeviceToDevice, s));
    LF_CUDA(cudaMemcpyAsync(index->qprime.need((size_t)nk * nc), dq, sizeof(double) * nk * nc,
                            cudaMemcpyDeviceToDevice, s));
    index->d_kclasses.upload(kc, s);
    LF_CUDA(cudaStreamSynchronize(s));
    index->nc = (int)nc;
    index->nk = nk;
    for (int i = 0; i < LEAFI_MAX_KCLASSES; ++i) index->kclasses[i] = i < nk ? kc[i] : 0;
    index->calib_q.release();  // these tables come without their calibration queries
    index->rq_cache.clear();
    index->tables_gen += 1;
  });
}

leafi_status leafi_search(leafi_index* index, const float* queries, int64_t nq, int32_t k,
                          double recall_target, int64_t* ids, float* dists,
                          leafi_search_stats* stats) {
  return guarded([&] {
    require_device(index);
    check_queries(index, queries, nq);
    if (k < 1 || k > LEAFI_MAX_K) fail(LEAFI_EINVAL, "k must be in [1, %d]", LEAFI_MAX_K);
    if (!(recall_target > 0.0)) fail(LEAFI_EINVAL, "recall_target must be > 0");
    if (nq > 0 && (!ids || !dists)) fail(LEAFI_EINVAL, "NULL output");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    std::vector<int32_t> kq(nq, k);
    std::vector<double> tg(nq, recall_target);
    search_impl(index, queries, nq, kq, tg, k, ids, dists, stats);
  });
}

leafi_status leafi_search_scanned(leafi_index* index, const float* queries, int64_t nq,
                                  int32_t k, double recall_target, int64_t* ids, float* dists,
                                  uint8_t* scanned) {
  return guarded([&] {
    require_device(index);
    check_queries(index, queries, nq);
    if (k < 1 || k > LEAFI_MAX_K) fail(LEAFI_EINVAL, "k must be in [1, %d]", LEAFI_MAX_K);
    if (!(recall_target > 0.0)) fail(LEAFI_EINVAL, "recall_target must be > 0");
    if (nq > 0 && (!ids || !dists || !scanned)) fail(LEAFI_EINVAL, "NULL output");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    const size_t bytes = (size_t)nq * index->tree.n_leaves;
    DBuf<unsigned char> sc;
    unsigned char* dsc = sc.need(std::max<size_t>(bytes, 1));
    std::vector<int32_t> kq(nq, k);
    std::vector<double> tg(nq, recall_target);
    search_impl(index, queries, nq, kq, tg, k, ids, dists, nullptr, dsc);
    deliver(scanned, dsc, bytes, index->stream);
    LF_CUDA(cudaStreamSynchronize(index->stream));
  });
}

leafi_status leafi_exact_search(leafi_index* index, const float* queries, int64_t nq, int32_t k,
                                int64_t* ids, float* dists, leafi_search_stats* stats) {
  return leafi_search(index, queries, nq, k, 1.0, ids, dists, stats);
}

leafi_status leafi_search_mixed(leafi_index* index, const float* queries, int64_t nq,
                                const int32_t* k, const double* recall_target, int32_t kmax,
                                int64_t* ids, float* dists, leafi_search_stats* stats) {
  return guarded([&] {
    require_device(index);
    check_queries(index, queries, nq);
    if (kmax < 1 || kmax > LEAFI_MAX_K) fail(LEAFI_EINVAL, "kmax must be in [1, %d]", LEAFI_MAX_K);
    if (nq > 0 && (!k || !recall_target || !ids || !dists)) fail(LEAFI_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(index->mu);
    DeviceGuard dg(index->device);
    std::vector<int32_t> kq;
    std::vector<double> tg;
    to_host(kq, k, nq, index->stream);
    to_host(tg, recall_target, nq, index->stream);
    for (int64_t i = 0; i < nq; ++i) {
      if (kq[i] < 1 || kq[i] > kmax) fail(LEAFI_EINVAL, "k[%lld] out of range", (long long)i);
      if (!(tg[i] > 0.0)) fail(LEAFI_EINVAL, "recall_target[%lld] must be > 0", (long long)i);
    }
    search_impl(index, queries, nq, kq, tg, kmax, ids, dists, stats);
  });
}

}  // extern "C"

// ---------------------------------------------------------------- serving
// A request loop over a resident index: pending queries of all requests form
// batches that run through a multi-lane pipeline of the server's own (the
// index's entry points keep theirs); see include/leafi.h.
struct leafi_server {
  leafi_index* ix = nullptr;
  leafi_serve_params p{};
  leafi::Scratch lanes[kServeLanes];
  leafi::Pipeline pl;
  leafi::DBuf<unsigned long long> stat;  // device counters of the server's batches
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv;       // new work or stop (the worker waits)
  std::condition_variable done_cv;  // a request finished (pollers wait)
  bool stopping = false;
  typedef std::chrono::steady_clock clock;
  struct Request {
    int nq = 0;
    std::vector<float> q;    // [nq][m]
    std::vector<int32_t> k;
    std::vector<double> t;
    std::vector<int64_t> ids;  // [nq][kmax]
    std::vector<float> d;
    int remaining = 0;
    bool done = false;
    size_t bytes = 0;
    clock::time_point t_submit, t_done;
  };
  std::map<int64_t, Request> reqs;
  std::deque<std::pair<int64_t, int>> pending;  // (ticket, query) not yet in a batch
  std::deque<clock::time_point> pending_t;      // arrival of each pending query
  int64_t next_ticket = 1;
  size_t bytes = 0;
  // per lane: the batch's members and its pinned host staging
  std::vector<std::pair<int64_t, int>> members[kServeLanes];
  float* hq[kServeLanes] = {};
  int32_t* hk[kServeLanes] = {};
  double* ht[kServeLanes] = {};
  int64_t* hi[kServeLanes] = {};
  float* hd[kServeLanes] = {};
  leafi_serve_stats counters{};
  int inflight = 0;  // batches on the GPU (worker thread, under mu)
  leafi_status failed = LEAFI_OK;
  std::string fail_msg;
};

namespace {

size_t serve_bytes_per_query(const leafi_server* sv) {
  return (size_t)sv->ix->m * sizeof(float) + sizeof(int32_t) + sizeof(double) +
         (size_t)sv->p.kmax * (sizeof(int64_t) + sizeof(float));
}

// run `fn` on the index (its mutex held, its device current); the index's
// own entry points find their lane and stream restored afterwards
template <class Fn>
void on_index(leafi_server* sv, Fn&& fn) {
  leafi_index* ix = sv->ix;
  std::lock_guard<std::mutex> lk(ix->mu);
  const cudaStream_t user = ix->stream;
  struct Restore {
    leafi_index* ix;
    cudaStream_t user;
    ~Restore() {
      ix->sc = &ix->lanes[0];
      ix->stream = user;
      ix->capturing = nullptr;
    }
  } restore{ix, user};
  fn();
}

void serve_loop(leafi_server* sv) {
  leafi_index* ix = sv->ix;
  cudaSetDevice(ix->device);
  const int kmax = sv->p.kmax;
  const auto wait = std::chrono::duration_cast<leafi_server::clock::duration>(
      std::chrono::duration<double, std::milli>(sv->p.max_wait_ms));
  int next = 0;  // lane of the next batch; batches start on the lanes in turn, so the
                 // oldest batch in flight is the first busy lane from `next` on
  auto any_busy = [&] {
    for (int i = 0; i < kServeLanes; ++i)
      if (sv->pl.busy(i)) return true;
    return false;
  };
  try {
    for (;;) {
      std::unique_lock<std::mutex> lk(sv->mu);
      const bool inflight = any_busy();
      if (!inflight)
        sv->cv.wait(lk, [&] { return sv->stopping || !sv->pending.empty(); });
      if (sv->stopping && sv->pending.empty() && !inflight) break;
      if (!sv->pending.empty() && !sv->pl.busy(next)) {
        // launch a full batch at once; a partial one when the GPU is idle or
        // its oldest query has waited long enough
        const auto deadline = sv->pending_t.front() + wait;
        if ((int)sv->pending.size() < sv->p.max_batch && inflight && !sv->stopping &&
            leafi_server::clock::now() < deadline)
          sv->cv.wait_until(lk, deadline, [&] {
            return sv->stopping || (int)sv->pending.size() >= sv->p.max_batch;
          });
        const int nb = std::min<int>((int)sv->pending.size(), sv->p.max_batch);
        sv->inflight += 1;
        auto& mem = sv->members[next];
        mem.assign(sv->pending.begin(), sv->pending.begin() + nb);
        sv->pending.erase(sv->pending.begin(), sv->pending.begin() + nb);
        sv->pending_t.erase(sv->pending_t.begin(), sv->pending_t.begin() + nb);
        bool use_f = false;
        for (int j = 0; j < nb; ++j) {
          const leafi_server::Request& r = sv->reqs.at(mem[j].first);
          const int qi = mem[j].second;
          std::memcpy(sv->hq[next] + (size_t)j * ix->m, r.q.data() + (size_t)qi * ix->m,
                      sizeof(float) * ix->m);
          sv->hk[next][j] = r.k[qi];
          sv->ht[next][j] = r.t[qi];
          use_f = use_f || r.t[qi] < 1.0;
        }
        lk.unlock();
        const int li = next;
        on_index(sv, [&] {
          leafi::DeviceGuard dg(ix->device);
          if (use_f) leafi::ensure_wsplit(ix);
          sv->pl.setup(ix, sv->lanes, kServeLanes, kmax, ix->F > 0 && ix->nc > 0, sv->stat.p,
                       sv->p.max_batch);
          sv->pl.start(li, sv->hq[li], nb, sv->hk[li], sv->ht[li], false, sv->hi[li], sv->hd[li]);
        });
        next = (next + 1) % kServeLanes;
        continue;
      }
      if (!inflight) continue;
      // collect the oldest batch in flight
      int li = next;
      while (!sv->pl.busy(li)) li = (li + 1) % kServeLanes;
      lk.unlock();
      on_index(sv, [&] {
        leafi::DeviceGuard dg(ix->device);
        sv->pl.finish(li);
        LF_CUDA(cudaStreamSynchronize(sv->lanes[li].st));
      });
      lk.lock();
      sv->inflight -= 1;
      const auto now = leafi_server::clock::now();
      const auto& mem = sv->members[li];
      for (size_t j = 0; j < mem.size(); ++j) {
        leafi_server::Request& r = sv->reqs.at(mem[j].first);
        const int qi = mem[j].second;
        std::memcpy(r.ids.data() + (size_t)qi * kmax, sv->hi[li] + j * kmax, sizeof(int64_t) * kmax);
        std::memcpy(r.d.data() + (size_t)qi * kmax, sv->hd[li] + j * kmax, sizeof(float) * kmax);
        if (--r.remaining == 0) {
          r.done = true;
          r.t_done = now;
          sv->counters.requests += 1;
          sv->counters.queries += r.nq;
        }
      }
      sv->counters.batches += 1;
      sv->done_cv.notify_all();
    }
  } catch (const Failure& e) {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->failed = e.status;
    sv->fail_msg = e.msg;
    sv->done_cv.notify_all();
  } catch (const std::exception& e) {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->failed = LEAFI_EINTERNAL;
    sv->fail_msg = e.what();
    sv->done_cv.notify_all();
  }
}

}  // namespace

extern "C" {

leafi_status leafi_serve_start(leafi_index* index, const leafi_serve_params* params,
                               leafi_server** out) {
  return guarded([&] {
    require_device(index);
    if (!out) fail(LEAFI_EINVAL, "out is NULL");
    leafi_serve_params p{256, 1, 0.2, 0};
    if (params) p = *params;
    if (p.max_batch < 1 || p.max_batch > kMaxBatch)
      fail(LEAFI_EINVAL, "max_batch must be in [1, %d]", kMaxBatch);
    if (p.kmax < 1 || p.kmax > LEAFI_MAX_K) fail(LEAFI_EINVAL, "kmax must be in [1, %d]", LEAFI_MAX_K);
    if (!(p.max_wait_ms >= 0.0)) fail(LEAFI_EINVAL, "max_wait_ms must be >= 0");
    if (p.max_bytes <= 0) p.max_bytes = (int64_t)1 << 30;
    std::unique_ptr<leafi_server> sv(new leafi_server());
    sv->ix = index;
    sv->p = p;
    {
      DeviceGuard dg(index->device);
      sv->stat.need(kPipelineStats);
      LF_CUDA(cudaMemset(sv->stat.p, 0, kPipelineStats * sizeof(unsigned long long)));
      for (int li = 0; li < kServeLanes; ++li) {
        const size_t b = (size_t)p.max_batch;
        LF_CUDA(cudaMallocHost(&sv->hq[li], sizeof(float) * b * index->m));
        LF_CUDA(cudaMallocHost(&sv->hk[li], sizeof(int32_t) * b));
        LF_CUDA(cudaMallocHost(&sv->ht[li], sizeof(double) * b));
        LF_CUDA(cudaMallocHost(&sv->hi[li], sizeof(int64_t) * b * p.kmax));
        LF_CUDA(cudaMallocHost(&sv->hd[li], sizeof(float) * b * p.kmax));
      }
    }
    sv->worker = std::thread(serve_loop, sv.get());
    *out = sv.release();
  });
}

leafi_status leafi_serve_submit(leafi_server* sv, const float* queries, int64_t nq,
                                const int32_t* k, const double* recall_target, int64_t* ticket) {
  return guarded([&] {
    if (!sv) fail(LEAFI_EINVAL, "server is NULL");
    if (nq < 1 || nq > (int64_t)1 << 24) fail(LEAFI_EINVAL, "nq out of range");
    if (!queries || !k || !recall_target || !ticket) fail(LEAFI_EINVAL, "NULL argument");
    if (on_device(queries) || on_device(k) || on_device(recall_target))
      fail(LEAFI_EINVAL, "serving takes host arrays");
    bool filtered = false;
    for (int64_t i = 0; i < nq; ++i) {
      if (k[i] < 1 || k[i] > sv->p.kmax) fail(LEAFI_EINVAL, "k[%lld] out of [1, kmax]", (long long)i);
      if (!(recall_target[i] > 0.0)) fail(LEAFI_EINVAL, "recall_target must be > 0");
      filtered = filtered || recall_target[i] < 1.0;
    }
    const leafi_index* ix = sv->ix;
    if (filtered && (ix->nc == 0 || ix->F == 0))
      fail(LEAFI_ENOTTRAINED, "recall_target < 1 needs fitted auto-tuners");
    const size_t need = (size_t)nq * serve_bytes_per_query(sv);
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->failed != LEAFI_OK) fail(sv->failed, "server stopped: %s", sv->fail_msg.c_str());
    if (sv->stopping) fail(LEAFI_EINVAL, "server is stopping");
    if (sv->bytes + need > (size_t)sv->p.max_bytes)
      fail(LEAFI_EAGAIN, "admission budget full (%zu of %lld bytes in use)", sv->bytes,
           (long long)sv->p.max_bytes);
    const int64_t t = sv->next_ticket++;
    leafi_server::Request& r = sv->reqs[t];
    r.nq = (int)nq;
    r.q.assign(queries, queries + (size_t)nq * ix->m);
    r.k.assign(k, k + nq);
    r.t.assign(recall_target, recall_target + nq);
    r.ids.assign((size_t)nq * sv->p.kmax, -1);
    r.d.assign((size_t)nq * sv->p.kmax, std::numeric_limits<float>::infinity());
    r.remaining = (int)nq;
    r.bytes = need;
    r.t_submit = leafi_server::clock::now();
    sv->bytes += need;
    if (sv->inflight > 0) sv->counters.admitted_in_flight += 1;
    for (int i = 0; i < (int)nq; ++i) {
      sv->pending.emplace_back(t, i);
      sv->pending_t.push_back(r.t_submit);
    }
    *ticket = t;
    sv->cv.notify_one();
  });
}

leafi_status leafi_serve_poll(leafi_server* sv, int64_t ticket, int64_t* ids, float* dists,
                              double wait_ms, int32_t* done, double* latency_ms) {
  return guarded([&] {
    if (!sv || !done) fail(LEAFI_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) fail(LEAFI_EINVAL, "unknown ticket %lld", (long long)ticket);
    if (!it->second.done && wait_ms > 0.0)
      sv->done_cv.wait_for(lk, std::chrono::duration<double, std::milli>(wait_ms), [&] {
        return sv->failed != LEAFI_OK || sv->reqs.at(ticket).done;
      });
    if (sv->failed != LEAFI_OK && !sv->reqs.at(ticket).done)
      fail(sv->failed, "server stopped: %s", sv->fail_msg.c_str());
    leafi_server::Request& r = sv->reqs.at(ticket);
    *done = r.done ? 1 : 0;
    if (!r.done) return;
    if (ids) std::memcpy(ids, r.ids.data(), sizeof(int64_t) * r.ids.size());
    if (dists) std::memcpy(dists, r.d.data(), sizeof(float) * r.d.size());
    if (latency_ms)
      *latency_ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
    sv->bytes -= r.bytes;
    sv->reqs.erase(ticket);
  });
}

leafi_status leafi_serve_get_stats(leafi_server* sv, leafi_serve_stats* stats) {
  return guarded([&] {
    if (!sv || !stats) fail(LEAFI_EINVAL, "NULL argument");
    leafi_serve_stats c;
    leafi_search_stats st;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      c = sv->counters;
    }
    unsigned long long h[kPipelineStats] = {};
    on_index(sv, [&] {
      DeviceGuard dg(sv->ix->device);
      LF_CUDA(cudaMemcpy(h, sv->stat.p, sizeof(h), cudaMemcpyDeviceToHost));
      st = sv->pl.st;
    });
    st.leaves_scanned = (int64_t)h[0];
    st.series_scanned = (int64_t)h[1];
    st.distinct_series = (int64_t)h[2];
    st.rechecks = (int64_t)h[3];
    st.filter_pruned = (int64_t)h[4];
    st.filter_evals += (int64_t)h[5];
    st.lb_pruned = c.queries * (int64_t)sv->ix->tree.n_leaves - st.leaves_scanned - st.filter_pruned;
    c.graph_batches = st.graph_batches;
    c.search = st;
    c.device_bytes = 0;
    for (int i = 0; i < kServeLanes; ++i) c.device_bytes += (int64_t)sv->lanes[i].bytes();
    *stats = c;
  });
}

leafi_status leafi_serve_stop(leafi_server* sv) {
  return guarded([&] {
    if (!sv) return;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->stopping = true;
    }
    sv->cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    const leafi_status failed = sv->failed;
    const std::string msg = sv->fail_msg;
    {
      DeviceGuard dg(sv->ix->device);
      for (int li = 0; li < kServeLanes; ++li) {
        if (sv->lanes[li].st) cudaStreamSynchronize(sv->lanes[li].st);
        for (auto& g : sv->lanes[li].graphs) {
          if (g.exec) cudaGraphExecDestroy(g.exec);
          for (cudaEvent_t e : g.ev) cudaEventDestroy(e);
        }
        sv->lanes[li].graphs.clear();
        sv->lanes[li].release_lane();
        cudaFreeHost(sv->hq[li]);
        cudaFreeHost(sv->hk[li]);
        cudaFreeHost(sv->ht[li]);
        cudaFreeHost(sv->hi[li]);
        cudaFreeHost(sv->hd[li]);
      }
      delete sv;
    }
    if (failed != LEAFI_OK) fail(failed, "server had stopped: %s", msg.c_str());
  });
}

}  // extern "C"
