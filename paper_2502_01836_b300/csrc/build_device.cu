// DSTree built level by level on the GPU (bulk form of the sequential build).
//
// Sequential insertion in id order splits a leaf exactly when it first holds
// more than `cap` members and a split candidate separates them; the decision
// uses those members only (min / max statistics and range-based scores do not
// depend on their order), and every later member is routed by the rule.  So
// the tree equals this top-down process: a node with S_v (its members in id
// order, |S_v| > cap) is decided on the first j members of S_v, j = cap + 1 or
// the smallest larger j that has a valid candidate; then all of S_v is
// partitioned stably by the rule and each child continues with its share.  A
// node's ranges (the synopsis) cover all members that ever pass through it,
// i.e. all of S_v.  Each level runs on the device:
//   1. member_stats_kernel: per decided node, the first j members' mean and
//      sigma on every segment and on both halves of every segment (float64
//      prefix sums in the host build's order and operations);
//   2. candidate_kernel: one block per split candidate: threshold = (min + max)
//      / 2 of the candidate's statistic, side counts, the children's ranges
//      and the score QoS(node) - (|L| QoS(L) + |R| QoS(R)) / |node|; the host
//      takes the earliest candidate with the largest score;
//   3. route_kernel: every member of a split node: its side, and the
//      children's ranges (warp minimum / maximum, then atomics on
//      order-preserving integer images of the doubles);
//   4. scatter_kernel: stable partition of the node's id-ordered members.
// Every float64 operation is the correctly rounded one the host performs (no
// contraction), so thresholds, ranges and routes are bit-identical to the
// sequential build.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "host_tree.h"
#include "internal.h"

namespace leafi {
namespace {

constexpr int kBuildThreads = 256;
constexpr int kMaxSegs = 512;  // segments of one node (each needs >= 1 point, m <= 512)
constexpr size_t kStatBudget = size_t(1) << 30;  // bytes of member statistics per pass

struct MS {
  double mu, sd;
};

__device__ __forceinline__ MS interval_ms(double p1s, double p2s, double p1e, double p2e, int len) {
  const double l = (double)len;
  const double mean = __ddiv_rn(__dsub_rn(p1e, p1s), l);
  double var = __dsub_rn(__ddiv_rn(__dsub_rn(p2e, p2s), l), __dmul_rn(mean, mean));
  if (var < 0.0) var = 0.0;
  return {mean, __dsqrt_rn(var)};
}

// running prefix sums of one row, advanced to point `to`
struct Prefix {
  const float* row;
  int i = 0;
  double a = 0.0, b = 0.0;
  __device__ __forceinline__ void advance(int to) {
    for (; i < to; ++i) {
      const double v = (double)row[i];
      a = __dadd_rn(a, v);
      b = __dadd_rn(b, __dmul_rn(v, v));
    }
  }
};

// doubles as unsigned integers of the same order (no NaN in the statistics)
__device__ __forceinline__ unsigned long long ord_key(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

struct StatJob {
  int64_t off;       // first member position in the permutation
  int j;             // members the decision uses
  int S;             // segments of the node
  int seg_off;       // its segment ends in `ends`
  int64_t stat_off;  // its first member's statistics (j x S records)
};

__global__ void member_stats_kernel(const float* __restrict__ X, int m,
                                    const int32_t* __restrict__ perm,
                                    const StatJob* __restrict__ jobs, int njobs,
                                    const int64_t* __restrict__ first, int64_t total,
                                    const int32_t* __restrict__ ends, MS* __restrict__ whole,
                                    MS* __restrict__ halves) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  int lo = 0, hi = njobs - 1;  // last job with first <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  const StatJob J = jobs[lo];
  const int64_t d = t - first[lo];
  Prefix P{X + (int64_t)perm[J.off + d] * m};
  const int32_t* e_ = ends + J.seg_off;
  double p1s = 0.0, p2s = 0.0;
  for (int r = 0; r < J.S; ++r) {
    const int s = r == 0 ? 0 : e_[r - 1], e = e_[r];
    const int mid = s + (e - s) / 2;
    const int64_t rec = J.stat_off + d * J.S + r;
    double p1m = 0.0, p2m = 0.0;
    if (e - s >= 2) {
      P.advance(mid);
      p1m = P.a;
      p2m = P.b;
    }
    P.advance(e);
    whole[rec] = interval_ms(p1s, p2s, P.a, P.b, e - s);
    if (e - s >= 2) {
      halves[2 * rec] = interval_ms(p1s, p2s, p1m, p2m, mid - s);
      halves[2 * rec + 1] = interval_ms(p1m, p2m, P.a, P.b, e - mid);
    }
    p1s = P.a;
    p2s = P.b;
  }
}

struct Cand {
  int job;
  int vertical, seg, half, sd;
};

struct CandJob {
  int j, S, seg_off;
  int64_t stat_off;
};

// statistic of member d on child segment q of candidate c
__device__ __forceinline__ MS child_ms(const Cand& c, const MS* whole, const MS* halves, int S,
                                       int64_t base, int64_t d, int q) {
  const int64_t rec = base + d * S;
  if (!c.vertical || q < c.seg) return whole[rec + q];
  if (q == c.seg) return halves[2 * (rec + c.seg)];
  if (q == c.seg + 1) return halves[2 * (rec + c.seg) + 1];
  return whole[rec + q - 1];
}

__device__ __forceinline__ double warp_min_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = v < w ? w : v;
  }
  return v;
}

// block-wide minimum / maximum of n values per thread (in place, result in v)
template <int NV>
__device__ void block_minmax(double (&v)[NV], const bool (&is_max)[NV], double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = is_max[k] ? warp_max_d(v[k]) : warp_min_d(v[k]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[warp * NV + k] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = red[k];
    for (int w = 1; w < nw; ++w) {
      const double y = red[w * NV + k];
      x = is_max[k] ? (x < y ? y : x) : (y < x ? y : x);
    }
    v[k] = x;
  }
  __syncthreads();
}

__device__ __forceinline__ int block_sum(int v, int* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = __reduce_add_sync(0xffffffffu, v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  int x = 0;
  for (int w = 0; w < nw; ++w) x += red[w];
  __syncthreads();
  return x;
}

__global__ void __launch_bounds__(kBuildThreads) candidate_kernel(
    const Cand* __restrict__ cands, const CandJob* __restrict__ jobs,
    const int32_t* __restrict__ ends, const MS* __restrict__ whole,
    const MS* __restrict__ halves, double* __restrict__ score, double* __restrict__ thresh,
    int32_t* __restrict__ valid) {
  extern __shared__ double sh[];  // [cn][12] ranges, then reduction scratch
  __shared__ double red[(kBuildThreads / 32) * 12];
  __shared__ int ired[kBuildThreads / 32];
  const Cand c = cands[blockIdx.x];
  const CandJob J = jobs[c.job];
  const int S = J.S, cn = c.vertical ? S + 1 : S;
  const int q_split = c.vertical ? c.seg + c.half : c.seg;
  const int32_t* e_ = ends + J.seg_off;
  // threshold: midpoint of the statistic's range over the j members
  double mm[2] = {__longlong_as_double(0x7ff0000000000000ll),
                  -__longlong_as_double(0x7ff0000000000000ll)};
  for (int64_t d = threadIdx.x; d < J.j; d += blockDim.x) {
    const MS st = child_ms(c, whole, halves, S, J.stat_off, d, q_split);
    const double v = c.sd ? st.sd : st.mu;
    mm[0] = v < mm[0] ? v : mm[0];
    mm[1] = mm[1] < v ? v : mm[1];
  }
  const bool mx2[2] = {false, true};
  block_minmax<2>(mm, mx2, red);
  const double th = __dmul_rn(__dadd_rn(mm[0], mm[1]), 0.5);
  int nl = 0;
  for (int64_t d = threadIdx.x; d < J.j; d += blockDim.x) {
    const MS st = child_ms(c, whole, halves, S, J.stat_off, d, q_split);
    nl += ((c.sd ? st.sd : st.mu) < th) ? 1 : 0;
  }
  nl = block_sum(nl, ired);
  const int nr = J.j - nl;
  if (nl == 0 || nr == 0) {
    if (threadIdx.x == 0) {
      valid[blockIdx.x] = 0;
      score[blockIdx.x] = 0.0;
      thresh[blockIdx.x] = th;
    }
    return;
  }
  // ranges of all members, the left side and the right side per child segment
  const double inf = __longlong_as_double(0x7ff0000000000000ll);
  const bool mx12[12] = {false, true, false, true, false, true, false, true, false, true, false, true};
  for (int q = 0; q < cn; ++q) {
    double g[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) g[k] = mx12[k] ? -inf : inf;
    for (int64_t d = threadIdx.x; d < J.j; d += blockDim.x) {
      const MS sp = child_ms(c, whole, halves, S, J.stat_off, d, q_split);
      const bool left = (c.sd ? sp.sd : sp.mu) < th;
      const MS v = child_ms(c, whole, halves, S, J.stat_off, d, q);
      const int o = left ? 4 : 8;
      g[0] = v.mu < g[0] ? v.mu : g[0];
      g[1] = g[1] < v.mu ? v.mu : g[1];
      g[2] = v.sd < g[2] ? v.sd : g[2];
      g[3] = g[3] < v.sd ? v.sd : g[3];
#pragma unroll
      for (int side = 4; side <= 8; side += 4) {
        if (side != o) continue;
        g[side + 0] = v.mu < g[side + 0] ? v.mu : g[side + 0];
        g[side + 1] = g[side + 1] < v.mu ? v.mu : g[side + 1];
        g[side + 2] = v.sd < g[side + 2] ? v.sd : g[side + 2];
        g[side + 3] = g[side + 3] < v.sd ? v.sd : g[side + 3];
      }
    }
    block_minmax<12>(g, mx12, red);
    if (threadIdx.x == 0)
      for (int k = 0; k < 12; ++k) sh[q * 12 + k] = g[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // QoS of the child segmentation: sum over segments of l ((mu_max - mu_min)^2 + sd_max^2)
    double qs[3] = {0.0, 0.0, 0.0};
    for (int q = 0; q < cn; ++q) {
      int len;
      if (!c.vertical || q < c.seg) {
        len = e_[q] - (q == 0 ? 0 : e_[q - 1]);
      } else if (q > c.seg + 1) {
        len = e_[q - 1] - (q - 1 == 0 ? 0 : e_[q - 2]);
      } else {
        const int s = c.seg == 0 ? 0 : e_[c.seg - 1];
        const int h1 = (e_[c.seg] - s) / 2;
        len = q == c.seg ? h1 : (e_[c.seg] - s) - h1;
      }
      const double l = (double)len;
      for (int k = 0; k < 3; ++k) {
        const double* r = sh + q * 12 + 4 * k;
        const double span = __dsub_rn(r[1], r[0]);
        const double term = __dmul_rn(l, __dadd_rn(__dmul_rn(span, span), __dmul_rn(r[3], r[3])));
        qs[k] = __dadd_rn(qs[k], term);
      }
    }
    const double w = __dadd_rn(__dmul_rn((double)nl, qs[1]), __dmul_rn((double)nr, qs[2]));
    score[blockIdx.x] = __dsub_rn(qs[0], __ddiv_rn(w, (double)J.j));
    thresh[blockIdx.x] = th;
    valid[blockIdx.x] = 1;
  }
}

struct RouteJob {
  int64_t off, cnt;
  int cn, seg_off;     // child segmentation (cn segments) in `ends`
  int q_split, sd;
  double th;
  int syn_left, syn_right;  // first record of each child's ranges in `syn` (4 keys per segment)
};

struct RouteBlock {
  int job;
  int64_t start;  // first member (relative to the job's offset)
};

// side of every member of a split node and the children's ranges
__global__ void __launch_bounds__(kBuildThreads) route_kernel(
    const float* __restrict__ X, int m, const int32_t* __restrict__ perm,
    const RouteJob* __restrict__ jobs, const RouteBlock* __restrict__ blocks,
    const int32_t* __restrict__ ends, unsigned char* __restrict__ left_flag,
    int32_t* __restrict__ block_left, unsigned long long* __restrict__ syn) {
  __shared__ int ired[kBuildThreads / 32];
  const RouteBlock B = blocks[blockIdx.x];
  const RouteJob J = jobs[B.job];
  const int64_t d = B.start + threadIdx.x;
  const bool live = d < J.cnt;
  const int lane = threadIdx.x & 31;
  const int32_t* e_ = ends + J.seg_off;
  const float* row = live ? X + (int64_t)perm[J.off + d] * m : X;
  // pass 1: the split statistic
  bool left = false;
  {
    Prefix P{row};
    double p1s = 0.0, p2s = 0.0;
    const int s = J.q_split == 0 ? 0 : e_[J.q_split - 1], e = e_[J.q_split];
    if (live) {
      P.advance(s);
      p1s = P.a;
      p2s = P.b;
      P.advance(e);
      const MS st = interval_ms(p1s, p2s, P.a, P.b, e - s);
      left = (J.sd ? st.sd : st.mu) < J.th;
      left_flag[J.off + d] = left ? 1 : 0;
    }
  }
  const int nl = block_sum(live && left ? 1 : 0, ired);
  if (threadIdx.x == 0) block_left[blockIdx.x] = nl;
  // pass 2: ranges of each child on its segments
  Prefix P{row};
  double p1s = 0.0, p2s = 0.0;
  for (int q = 0; q < J.cn; ++q) {
    const int s = q == 0 ? 0 : e_[q - 1], e = e_[q];
    unsigned long long kmu = 0, ksd = 0;
    if (live) {
      P.advance(e);
      const MS st = interval_ms(p1s, p2s, P.a, P.b, e - s);
      p1s = P.a;
      p2s = P.b;
      kmu = ord_key(st.mu);
      ksd = ord_key(st.sd);
    }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const bool mine = live && (left == (side == 0));
      unsigned long long v[4] = {mine ? kmu : ~0ull, mine ? kmu : 0ull, mine ? ksd : ~0ull,
                                 mine ? ksd : 0ull};
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const unsigned long long w = __shfl_xor_sync(0xffffffffu, v[k], o);
          v[k] = (k & 1) ? (w > v[k] ? w : v[k]) : (w < v[k] ? w : v[k]);
        }
      }
      const unsigned any = __ballot_sync(0xffffffffu, mine);
      if (lane == 0 && any != 0u) {
        unsigned long long* g = syn + 4 * ((size_t)(side == 0 ? J.syn_left : J.syn_right) + q);
        atomicMin(&g[0], v[0]);
        atomicMax(&g[1], v[1]);
        atomicMin(&g[2], v[2]);
        atomicMax(&g[3], v[3]);
      }
    }
  }
}

// stable partition: block b of a job writes its left members after the
// job's earlier blocks' left members, its right members after all left ones
__global__ void __launch_bounds__(kBuildThreads) scatter_kernel(
    const int32_t* __restrict__ perm_in, int32_t* __restrict__ perm_out,
    const RouteJob* __restrict__ jobs, const RouteBlock* __restrict__ blocks,
    const unsigned char* __restrict__ left_flag, const int64_t* __restrict__ left_base,
    const int64_t* __restrict__ right_base) {
  __shared__ int scan[kBuildThreads];
  const RouteBlock B = blocks[blockIdx.x];
  const RouteJob J = jobs[B.job];
  const int64_t d = B.start + threadIdx.x;
  const bool live = d < J.cnt;
  const int lf = live ? left_flag[J.off + d] : 0;
  scan[threadIdx.x] = lf;
  __syncthreads();
  for (int o = 1; o < kBuildThreads; o <<= 1) {
    const int v = threadIdx.x >= o ? scan[threadIdx.x - o] : 0;
    __syncthreads();
    scan[threadIdx.x] += v;
    __syncthreads();
  }
  if (!live) return;
  const int lrank = scan[threadIdx.x] - lf;           // left members before this one
  const int rrank = (int)threadIdx.x - lrank;           // right members before this one
  const int64_t dst = lf ? left_base[blockIdx.x] + lrank : right_base[blockIdx.x] + rrank;
  perm_out[J.off + dst] = perm_in[J.off + d];
}

__global__ void gather_rows_kernel(const float* __restrict__ X, int64_t n, int m,
                                   const int32_t* __restrict__ order, int mp,
                                   float* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * mp) return;
  const int64_t p = t / mp;
  const int i = (int)(t % mp);
  out[t] = i < m ? X[(int64_t)order[p] * m + i] : 0.0f;
}

__global__ void iota_kernel(int32_t* p, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = (int32_t)i;
}

// iSAX: full-cardinality symbols (PAA from the float64 prefix sums, then the
// number of breakpoints beta_1 .. beta_{C-1} at or below it) and root keys
__global__ void isax_symbols_kernel(const float* __restrict__ X, int64_t n, int m, int w, int l,
                                    const double* __restrict__ beta, int C, int bits,
                                    uint16_t* __restrict__ full, int32_t* __restrict__ key) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n) return;
  const float* row = X + id * m;
  double a = 0.0, ps = 0.0;
  int k = 0;
  for (int j = 0; j < w; ++j) {
    for (int i = j * l; i < (j + 1) * l; ++i) a = __dadd_rn(a, (double)row[i]);
    const double paa = __ddiv_rn(__dsub_rn(a, ps), (double)l);
    ps = a;
    int lo = 1, hi = C;  // first index in [1, C) with beta > paa
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (beta[mid] <= paa) lo = mid + 1;
      else hi = mid;
    }
    const int sym = lo - 1;
    full[id * w + j] = (uint16_t)sym;
    k = (k << 1) | (sym >> (bits - 1));
  }
  key[id] = k;
}

struct IsaxJob {
  int64_t off;
  int j;          // members the decision uses
  int bits[20];   // the node's cardinality bits per segment
};

// per node: ones among the first j members' next bit of every segment
__global__ void __launch_bounds__(kBuildThreads) isax_count_kernel(
    const uint16_t* __restrict__ full, int w, int card_bits, const int32_t* __restrict__ perm,
    const IsaxJob* __restrict__ jobs, int32_t* __restrict__ ones) {
  __shared__ int cnt[20];
  const IsaxJob J = jobs[blockIdx.x];
  if (threadIdx.x < w) cnt[threadIdx.x] = 0;
  __syncthreads();
  int loc[20];
  for (int q = 0; q < w; ++q) loc[q] = 0;
  for (int d = threadIdx.x; d < J.j; d += blockDim.x) {
    const uint16_t* fs = full + (int64_t)perm[J.off + d] * w;
    for (int q = 0; q < w; ++q)
      if (J.bits[q] < card_bits) loc[q] += (fs[q] >> (card_bits - J.bits[q] - 1)) & 1;
  }
  for (int q = 0; q < w; ++q) {
    const int v = __reduce_add_sync(0xffffffffu, loc[q]);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&cnt[q], v);
  }
  __syncthreads();
  if (threadIdx.x < w) ones[(size_t)blockIdx.x * w + threadIdx.x] = cnt[threadIdx.x];
}

struct IsaxRoute {
  int seg, have;  // refined segment and its bits before the split
};

// left (next bit 0) flags of a split node's members and the per-block counts
__global__ void __launch_bounds__(kBuildThreads) isax_flag_kernel(
    const uint16_t* __restrict__ full, int w, int card_bits, const int32_t* __restrict__ perm,
    const RouteJob* __restrict__ jobs, const IsaxRoute* __restrict__ how,
    const RouteBlock* __restrict__ blocks, unsigned char* __restrict__ left_flag,
    int32_t* __restrict__ block_left) {
  __shared__ int ired[kBuildThreads / 32];
  const RouteBlock B = blocks[blockIdx.x];
  const RouteJob J = jobs[B.job];
  const IsaxRoute H = how[B.job];
  const int64_t d = B.start + threadIdx.x;
  int left = 0;
  if (d < J.cnt) {
    const int bit = (full[(int64_t)perm[J.off + d] * w + H.seg] >> (card_bits - H.have - 1)) & 1;
    left = bit == 0;
    left_flag[J.off + d] = (unsigned char)left;
  }
  const int nl = block_sum(left, ired);
  if (threadIdx.x == 0) block_left[blockIdx.x] = nl;
}

double from_key(unsigned long long k) {
  const unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  double x;
  std::memcpy(&x, &u, sizeof(x));
  return x;
}

inline unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

struct Open {
  int node;
  int64_t off, cnt;
};

}  // namespace

HostTree build_dstree_device(const float* dX, int64_t n, int m, int leaf_cap, int init_segments,
                             void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t cap = leaf_cap;
  std::vector<DsNode> nodes(1);
  for (int r = 0; r < init_segments; ++r)
    nodes[0].ends.push_back((int)(((int64_t)(r + 1) * m) / init_segments));
  nodes[0].syn.resize(nodes[0].ends.size());

  DBuf<int32_t> permA, permB;
  int32_t* pin = permA.need((size_t)n);
  int32_t* pout = permB.need((size_t)n);
  iota_kernel<<<nblocks(n, 256), 256, 0, s>>>(pin, n);
  LF_CHECK_LAUNCH();
  DBuf<unsigned char> flags;
  flags.need((size_t)n);
  DBuf<int32_t> d_ends;
  DBuf<StatJob> d_sjobs;
  DBuf<int64_t> d_first;
  DBuf<MS> d_whole, d_halves;
  DBuf<Cand> d_cands;
  DBuf<CandJob> d_cjobs;
  DBuf<double> d_score, d_thresh;
  DBuf<int32_t> d_valid;
  DBuf<RouteJob> d_rjobs;
  DBuf<RouteBlock> d_rblocks;
  DBuf<int32_t> d_bleft;
  DBuf<int64_t> d_lbase, d_rbase;
  DBuf<unsigned long long> d_syn;

  // route + scatter of a set of splits (or, with th = +inf and one child, the
  // root's ranges); returns the left counts per job
  auto route = [&](std::vector<RouteJob>& rj, const std::vector<int32_t>& ends_h, int nsyn,
                   std::vector<unsigned long long>& syn_h, bool scatter) -> std::vector<int64_t> {
    std::vector<RouteBlock> rb;
    for (size_t i = 0; i < rj.size(); ++i)
      for (int64_t st = 0; st < rj[i].cnt; st += kBuildThreads) rb.push_back({(int)i, st});
    d_ends.upload(ends_h, s);
    d_rjobs.upload(rj, s);
    d_rblocks.upload(rb, s);
    d_bleft.need(rb.size());
    syn_h.assign((size_t)4 * nsyn, 0);
    for (int i = 0; i < nsyn; ++i) {
      syn_h[4 * i + 0] = ~0ull;
      syn_h[4 * i + 2] = ~0ull;
    }
    d_syn.upload(syn_h, s);
    if (!rb.empty()) {
      route_kernel<<<(unsigned)rb.size(), kBuildThreads, 0, s>>>(dX, m, pin, d_rjobs.p, d_rblocks.p,
                                                                d_ends.p, flags.p, d_bleft.p,
                                                                d_syn.p);
      LF_CHECK_LAUNCH();
    }
    std::vector<int32_t> bl(rb.size());
    if (!rb.empty())
      LF_CUDA(cudaMemcpyAsync(bl.data(), d_bleft.p, sizeof(int32_t) * rb.size(),
                              cudaMemcpyDeviceToHost, s));
    LF_CUDA(cudaMemcpyAsync(syn_h.data(), d_syn.p, sizeof(unsigned long long) * syn_h.size(),
                            cudaMemcpyDeviceToHost, s));
    LF_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> nl(rj.size(), 0);
    for (size_t b = 0; b < rb.size(); ++b) nl[rb[b].job] += bl[b];
    if (scatter && !rb.empty()) {
      std::vector<int64_t> lb(rb.size()), rbs(rb.size());
      std::vector<int64_t> accl(rj.size(), 0), accr(rj.size(), 0);
      for (size_t b = 0; b < rb.size(); ++b) {
        const int jb = rb[b].job;
        const int64_t live = std::min<int64_t>(kBuildThreads, rj[jb].cnt - rb[b].start);
        lb[b] = accl[jb];
        rbs[b] = nl[jb] + accr[jb];
        accl[jb] += bl[b];
        accr[jb] += live - bl[b];
      }
      d_lbase.upload(lb, s);
      d_rbase.upload(rbs, s);
      scatter_kernel<<<(unsigned)rb.size(), kBuildThreads, 0, s>>>(pin, pout, d_rjobs.p, d_rblocks.p,
                                                                  flags.p, d_lbase.p, d_rbase.p);
      LF_CHECK_LAUNCH();
    }
    return nl;
  };

  // the root's ranges: every series on the root's segments
  {
    std::vector<RouteJob> rj(1);
    rj[0] = {0, n, (int)nodes[0].ends.size(), 0, 0, 0,
             std::numeric_limits<double>::infinity(), 0, 0};
    std::vector<unsigned long long> syn_h;
    route(rj, nodes[0].ends, (int)nodes[0].ends.size(), syn_h, false);
    for (size_t r = 0; r < nodes[0].ends.size(); ++r) {
      nodes[0].syn[r].mlo = from_key(syn_h[4 * r + 0]);
      nodes[0].syn[r].mhi = from_key(syn_h[4 * r + 1]);
      nodes[0].syn[r].slo = from_key(syn_h[4 * r + 2]);
      nodes[0].syn[r].shi = from_key(syn_h[4 * r + 3]);
    }
  }

  std::vector<Open> frontier{{0, 0, n}}, leaves;
  while (!frontier.empty()) {
    // 1-2: decide the splits (first j members; j grows while no candidate separates them)
    struct Decide {
      Open o;
      int64_t j;
      int best = -1;
      Cand c{};
      double th = 0.0;
      bool done = false;
    };
    std::vector<Decide> dec;
    for (const Open& o : frontier) {
      if (o.cnt > cap) dec.push_back({o, cap + 1});
      else leaves.push_back(o);
    }
    for (;;) {
      std::vector<int> todo;
      for (size_t i = 0; i < dec.size(); ++i)
        if (!dec[i].done) todo.push_back((int)i);
      if (todo.empty()) break;
      size_t t0 = 0;
      while (t0 < todo.size()) {
        // a pass over as many nodes as the statistics budget holds
        std::vector<StatJob> sj;
        std::vector<CandJob> cj;
        std::vector<int64_t> first;
        std::vector<int32_t> ends_h;
        std::vector<Cand> cands;
        std::vector<int> cand_first;
        int64_t stat_total = 0, thr_total = 0;
        size_t t1 = t0;
        for (; t1 < todo.size(); ++t1) {
          const Decide& D = dec[todo[t1]];
          const DsNode& nd = nodes[D.o.node];
          const int S = (int)nd.ends.size();
          const int64_t recs = D.j * S;
          if (t1 > t0 && (size_t)(stat_total + recs) * 3 * sizeof(MS) > kStatBudget) break;
          StatJob J{D.o.off, (int)D.j, S, (int)ends_h.size(), stat_total};
          sj.push_back(J);
          cj.push_back({(int)D.j, S, J.seg_off, stat_total});
          first.push_back(thr_total);
          thr_total += D.j;
          stat_total += recs;
          ends_h.insert(ends_h.end(), nd.ends.begin(), nd.ends.end());
          cand_first.push_back((int)cands.size());
          const int jb = (int)sj.size() - 1;
          for (int r = 0; r < S; ++r)
            for (int sd = 0; sd < 2; ++sd) cands.push_back({jb, 0, r, 0, sd});
          for (int r = 0; r < S; ++r) {
            const int st = r == 0 ? 0 : nd.ends[r - 1];
            if (nd.ends[r] - st < 2) continue;
            for (int half = 0; half < 2; ++half)
              for (int sd = 0; sd < 2; ++sd) cands.push_back({jb, 1, r, half, sd});
          }
        }
        cand_first.push_back((int)cands.size());
        d_ends.upload(ends_h, s);
        d_sjobs.upload(sj, s);
        d_first.upload(first, s);
        MS* whole = d_whole.need((size_t)stat_total);
        MS* halves = d_halves.need((size_t)stat_total * 2);
        member_stats_kernel<<<nblocks(thr_total, 128), 128, 0, s>>>(
            dX, m, pin, d_sjobs.p, (int)sj.size(), d_first.p, thr_total, d_ends.p, whole, halves);
        LF_CHECK_LAUNCH();
        d_cands.upload(cands, s);
        d_cjobs.upload(cj, s);
        d_score.need(cands.size());
        d_thresh.need(cands.size());
        d_valid.need(cands.size());
        int max_cn = 1;
        for (const CandJob& c : cj) max_cn = std::max(max_cn, c.S + 1);
        if (max_cn > kMaxSegs + 1) fail(LEAFI_EINTERNAL, "node with more than %d segments", kMaxSegs);
        const size_t shm = (size_t)max_cn * 12 * sizeof(double);
        LF_CUDA(cudaFuncSetAttribute(candidate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)shm));
        candidate_kernel<<<(unsigned)cands.size(), kBuildThreads, shm, s>>>(
            d_cands.p, d_cjobs.p, d_ends.p, whole, halves, d_score.p, d_thresh.p, d_valid.p);
        LF_CHECK_LAUNCH();
        std::vector<double> sc(cands.size()), th(cands.size());
        std::vector<int32_t> va(cands.size());
        LF_CUDA(cudaMemcpyAsync(sc.data(), d_score.p, sizeof(double) * sc.size(),
                                cudaMemcpyDeviceToHost, s));
        LF_CUDA(cudaMemcpyAsync(th.data(), d_thresh.p, sizeof(double) * th.size(),
                                cudaMemcpyDeviceToHost, s));
        LF_CUDA(cudaMemcpyAsync(va.data(), d_valid.p, sizeof(int32_t) * va.size(),
                                cudaMemcpyDeviceToHost, s));
        LF_CUDA(cudaStreamSynchronize(s));
        for (size_t k = 0; k < sj.size(); ++k) {
          Decide& D = dec[todo[t0 + k]];
          int best = -1;
          for (int ci = cand_first[k]; ci < cand_first[k + 1]; ++ci)
            if (va[ci] && (best < 0 || sc[ci] > sc[best])) best = ci;
          if (best >= 0) {
            D.best = best;
            D.c = cands[best];
            D.th = th[best];
            D.done = true;
          } else if (D.j < D.o.cnt) {
            ++D.j;  // sequential insertion retries with one more member
          } else {
            D.done = true;  // no split separates the members: the leaf stays over capacity
          }
        }
        t0 = t1;
      }
    }
    // 3-4: route and partition the split nodes' members
    std::vector<RouteJob> rj;
    std::vector<int32_t> ends_h;
    std::vector<int> split_of;
    int nsyn = 0;
    for (size_t i = 0; i < dec.size(); ++i) {
      const Decide& D = dec[i];
      if (D.best < 0) {
        leaves.push_back(D.o);
        continue;
      }
      const DsNode& nd = nodes[D.o.node];
      std::vector<int> cends = nd.ends;
      if (D.c.vertical) {
        const int st = D.c.seg == 0 ? 0 : nd.ends[D.c.seg - 1];
        cends.insert(cends.begin() + D.c.seg, st + (nd.ends[D.c.seg] - st) / 2);
      }
      const int cn = (int)cends.size();
      RouteJob J{D.o.off, D.o.cnt, cn, (int)ends_h.size(),
                 D.c.vertical ? D.c.seg + D.c.half : D.c.seg, D.c.sd, D.th, nsyn, nsyn + cn};
      nsyn += 2 * cn;
      ends_h.insert(ends_h.end(), cends.begin(), cends.end());
      rj.push_back(J);
      split_of.push_back((int)i);
    }
    std::vector<Open> next;
    if (!rj.empty()) {
      LF_CUDA(cudaMemcpyAsync(pout, pin, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
      std::vector<unsigned long long> syn_h;
      const std::vector<int64_t> nl = route(rj, ends_h, nsyn, syn_h, true);
      std::swap(pin, pout);
      for (size_t k = 0; k < rj.size(); ++k) {
        const Decide& D = dec[split_of[k]];
        const RouteJob& J = rj[k];
        const int at = D.o.node;
        const int li = (int)nodes.size();
        std::vector<int> cends(ends_h.begin() + J.seg_off, ends_h.begin() + J.seg_off + J.cn);
        for (int side = 0; side < 2; ++side) {
          DsNode ch;
          ch.ends = cends;
          ch.syn.resize(J.cn);
          ch.parent = at;
          const int base = side == 0 ? J.syn_left : J.syn_right;
          for (int q = 0; q < J.cn; ++q) {
            ch.syn[q].mlo = from_key(syn_h[4 * (size_t)(base + q) + 0]);
            ch.syn[q].mhi = from_key(syn_h[4 * (size_t)(base + q) + 1]);
            ch.syn[q].slo = from_key(syn_h[4 * (size_t)(base + q) + 2]);
            ch.syn[q].shi = from_key(syn_h[4 * (size_t)(base + q) + 3]);
          }
          nodes.push_back(std::move(ch));
        }
        DsNode& nd = nodes[at];
        nd.leaf = false;
        nd.left = li;
        nd.right = li + 1;
        nd.child_ends = cends;
        nd.split_seg = J.q_split;
        nd.split_sd = J.sd != 0;
        nd.thresh = J.th;
        next.push_back({li, J.off, nl[k]});
        next.push_back({li + 1, J.off + nl[k], J.cnt - nl[k]});
      }
    }
    frontier.swap(next);
  }
  // leaves: their members, ascending ids (stable partitions of the id order)
  std::vector<int32_t> perm_h((size_t)n);
  LF_CUDA(cudaMemcpyAsync(perm_h.data(), pin, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
  LF_CUDA(cudaStreamSynchronize(s));
  for (const Open& o : leaves)
    nodes[o.node].members.assign(perm_h.begin() + o.off, perm_h.begin() + o.off + o.cnt);
  return dstree_from_nodes(nodes, n, m);
}

HostTree build_isax_device(const float* dX, int64_t n, int m, int leaf_cap, int w, int card_bits,
                           void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t cap = leaf_cap;
  const int C = 1 << card_bits;
  const int l = m / w;
  const std::vector<double> beta = isax_breakpoints(card_bits);
  DBuf<double> d_beta;
  d_beta.upload(beta, s);
  DBuf<uint16_t> full;
  full.need((size_t)n * w);
  DBuf<int32_t> keys;
  keys.need((size_t)n);
  isax_symbols_kernel<<<nblocks(n, 128), 128, 0, s>>>(dX, n, m, w, l, d_beta.p, C, card_bits, full.p,
                                                      keys.p);
  LF_CHECK_LAUNCH();
  // root children: ids grouped by root key, ascending within a key
  std::vector<int32_t> key_h((size_t)n);
  LF_CUDA(cudaMemcpyAsync(key_h.data(), keys.p, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
  LF_CUDA(cudaStreamSynchronize(s));
  const size_t K = size_t(1) << w;
  std::vector<int64_t> kstart(K + 1, 0);
  for (int64_t id = 0; id < n; ++id) ++kstart[(size_t)key_h[id] + 1];
  for (size_t k = 0; k < K; ++k) kstart[k + 1] += kstart[k];
  std::vector<int32_t> perm_h((size_t)n);
  {
    std::vector<int64_t> fill(kstart.begin(), kstart.end() - 1);
    for (int64_t id = 0; id < n; ++id) perm_h[(size_t)fill[(size_t)key_h[id]]++] = (int32_t)id;
  }
  std::vector<IsaxNode> nodes;
  std::vector<int> root_child(K, -1);
  std::vector<Open> frontier, leaves;
  for (size_t k = 0; k < K; ++k) {
    if (kstart[k + 1] == kstart[k]) continue;
    IsaxNode nd;
    nd.bits.assign(w, 1);
    nd.sym.resize(w);
    for (int j = 0; j < w; ++j) nd.sym[j] = (int)((k >> (w - 1 - j)) & 1);
    root_child[k] = (int)nodes.size();
    frontier.push_back({(int)nodes.size(), kstart[k], kstart[k + 1] - kstart[k]});
    nodes.push_back(std::move(nd));
  }
  DBuf<int32_t> permA, permB;
  int32_t* pin = permA.need((size_t)n);
  int32_t* pout = permB.need((size_t)n);
  LF_CUDA(cudaMemcpyAsync(pin, perm_h.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s));
  DBuf<unsigned char> flags;
  flags.need((size_t)n);
  DBuf<IsaxJob> d_jobs;
  DBuf<int32_t> d_ones, d_bleft;
  DBuf<RouteJob> d_rjobs;
  DBuf<IsaxRoute> d_how;
  DBuf<RouteBlock> d_rblocks;
  DBuf<int64_t> d_lbase, d_rbase;
  while (!frontier.empty()) {
    std::vector<Open> split;
    for (const Open& o : frontier) (o.cnt > cap ? split : leaves).push_back(o);
    std::vector<Open> next;
    if (!split.empty()) {
      // decisions on the first cap + 1 members (the insertion that overflows the leaf)
      std::vector<IsaxJob> jobs(split.size());
      for (size_t i = 0; i < split.size(); ++i) {
        jobs[i].off = split[i].off;
        jobs[i].j = (int)(cap + 1);
        for (int q = 0; q < w; ++q) jobs[i].bits[q] = nodes[split[i].node].bits[q];
      }
      d_jobs.upload(jobs, s);
      d_ones.need(split.size() * w);
      isax_count_kernel<<<(unsigned)split.size(), kBuildThreads, 0, s>>>(full.p, w, card_bits, pin,
                                                                         d_jobs.p, d_ones.p);
      LF_CHECK_LAUNCH();
      std::vector<int32_t> ones(split.size() * w);
      LF_CUDA(cudaMemcpyAsync(ones.data(), d_ones.p, sizeof(int32_t) * ones.size(),
                              cudaMemcpyDeviceToHost, s));
      LF_CUDA(cudaStreamSynchronize(s));
      std::vector<RouteJob> rj;
      std::vector<IsaxRoute> how;
      std::vector<int> of;
      for (size_t i = 0; i < split.size(); ++i) {
        const IsaxNode& nd = nodes[split[i].node];
        const int64_t total = cap + 1;
        int pick = -1, first = -1;
        int64_t pick_bal = 0;
        for (int q = 0; q < w; ++q) {
          if (nd.bits[q] >= card_bits) continue;
          if (first < 0) first = q;
          const int64_t o1 = ones[i * w + q], z = total - o1;
          if (o1 == 0 || z == 0) continue;
          const int64_t bal = o1 > z ? o1 - z : z - o1;
          if (pick < 0 || bal < pick_bal) {
            pick = q;
            pick_bal = bal;
          }
        }
        if (pick < 0) pick = first;
        if (pick < 0) {  // every segment at full cardinality: the leaf stays over capacity
          leaves.push_back(split[i]);
          continue;
        }
        RouteJob J{};
        J.off = split[i].off;
        J.cnt = split[i].cnt;
        rj.push_back(J);
        how.push_back({pick, nd.bits[pick]});
        of.push_back((int)i);
      }
      if (!rj.empty()) {
        std::vector<RouteBlock> rb;
        for (size_t i = 0; i < rj.size(); ++i)
          for (int64_t st = 0; st < rj[i].cnt; st += kBuildThreads) rb.push_back({(int)i, st});
        d_rjobs.upload(rj, s);
        d_how.upload(how, s);
        d_rblocks.upload(rb, s);
        d_bleft.need(rb.size());
        isax_flag_kernel<<<(unsigned)rb.size(), kBuildThreads, 0, s>>>(
            full.p, w, card_bits, pin, d_rjobs.p, d_how.p, d_rblocks.p, flags.p, d_bleft.p);
        LF_CHECK_LAUNCH();
        std::vector<int32_t> bl(rb.size());
        LF_CUDA(cudaMemcpyAsync(bl.data(), d_bleft.p, sizeof(int32_t) * rb.size(),
                                cudaMemcpyDeviceToHost, s));
        LF_CUDA(cudaStreamSynchronize(s));
        std::vector<int64_t> nl(rj.size(), 0), lb(rb.size()), rbs(rb.size()), accl(rj.size(), 0),
            accr(rj.size(), 0);
        for (size_t b = 0; b < rb.size(); ++b) nl[rb[b].job] += bl[b];
        for (size_t b = 0; b < rb.size(); ++b) {
          const int jb = rb[b].job;
          const int64_t live = std::min<int64_t>(kBuildThreads, rj[jb].cnt - rb[b].start);
          lb[b] = accl[jb];
          rbs[b] = nl[jb] + accr[jb];
          accl[jb] += bl[b];
          accr[jb] += live - bl[b];
        }
        d_lbase.upload(lb, s);
        d_rbase.upload(rbs, s);
        LF_CUDA(cudaMemcpyAsync(pout, pin, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
        scatter_kernel<<<(unsigned)rb.size(), kBuildThreads, 0, s>>>(pin, pout, d_rjobs.p, d_rblocks.p,
                                                                    flags.p, d_lbase.p, d_rbase.p);
        LF_CHECK_LAUNCH();
        std::swap(pin, pout);
        for (size_t k = 0; k < rj.size(); ++k) {
          const Open& o = split[of[k]];
          const int at = o.node, pick = how[k].seg;
          const int li = (int)nodes.size();
          for (int side = 0; side < 2; ++side) {
            IsaxNode ch;
            ch.bits = nodes[at].bits;
            ch.sym = nodes[at].sym;
            ch.bits[pick] += 1;
            ch.sym[pick] = nodes[at].sym[pick] * 2 + side;
            ch.parent = at;
            nodes.push_back(std::move(ch));
          }
          IsaxNode& nd = nodes[at];
          nd.leaf = false;
          nd.split = pick;
          nd.left = li;
          nd.right = li + 1;
          next.push_back({li, o.off, nl[k]});
          next.push_back({li + 1, o.off + nl[k], o.cnt - nl[k]});
        }
      }
    }
    frontier.swap(next);
  }
  LF_CUDA(cudaMemcpyAsync(perm_h.data(), pin, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
  LF_CUDA(cudaStreamSynchronize(s));
  for (const Open& o : leaves)
    nodes[o.node].members.assign(perm_h.begin() + o.off, perm_h.begin() + o.off + o.cnt);
  return isax_from_nodes(nodes, root_child, n, m, w, card_bits);
}

void launch_gather_rows(const float* X, int64_t n, int m, const int32_t* order, int mp, float* out,
                        cudaStream_t s) {
  if (n == 0) return;
  gather_rows_kernel<<<nblocks(n * mp, 256), 256, 0, s>>>(X, n, m, order, mp, out);
  LF_CHECK_LAUNCH();
}

}  // namespace leafi
