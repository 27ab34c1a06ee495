// Query preparation and summarisation lower bounds (Sec. 3; Alg. 2's bound test).
//
// Query statistics (prefix sums, segment means and sigmas, PAA values) are
// float64 and route queries exactly as the host build routed the series.  The
// bounds themselves are float32: each statistic is carried as the pair of
// floats enclosing it (conversions rounded down and up), each synopsis range
// and breakpoint is widened outward the same way, so every float32 gap is at
// most the float64 one and the bound stays a lower bound up to the relative
// rounding of the final products and sums.  Every operation is written with an
// explicit round-to-nearest intrinsic so nothing is contracted or reassociated.
#include <cfloat>

#include "internal.h"

namespace leafi {
namespace {

constexpr int kThreads = 128;

// Per query: P1[i] = sum_{t<i} q_t, P2[i] = sum_{t<i} q_t^2 (float64, sequential).
// One thread per query; the order of the additions is fixed.  The chains are
// bound by float64 latency, so the kernel uses no shared memory and few
// registers and can share SMs with a running leaf scan.
__global__ void prefix_kernel(const float* __restrict__ Q, int nq, int mp, int m,
                              double* __restrict__ P) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const float* x = Q + (size_t)q * mp;
  double* p1 = P + (size_t)q * 2 * (m + 1);
  double* p2 = p1 + m + 1;
  double a = 0.0, b = 0.0;
  p1[0] = 0.0;
  p2[0] = 0.0;
  for (int i = 0; i < m; ++i) {
    const double v = (double)x[i];
    a = __dadd_rn(a, v);
    b = __dadd_rn(b, __dmul_rn(v, v));
    p1[i + 1] = a;
    p2[i + 1] = b;
  }
}

__device__ __forceinline__ void interval_stat(const double* p1, const double* p2, int s, int e,
                                              double& mu, double& sd) {
  const double len = (double)(e - s);
  const double mean = __ddiv_rn(__dsub_rn(p1[e], p1[s]), len);
  double var = __dsub_rn(__ddiv_rn(__dsub_rn(p2[e], p2[s]), len), __dmul_rn(mean, mean));
  if (var < 0.0) var = 0.0;
  mu = mean;
  sd = __dsqrt_rn(var);
}

// gap of a value enclosed by [vd, vu] to a range [lo, hi] already widened
// outward: zero when they may overlap, else one float32 subtraction between
// the nearest ends, which is never above the gap of the value itself
__device__ __forceinline__ float gap32(float vd, float vu, float lo, float hi) {
  if (vu < lo) return __fsub_rn(lo, vu);
  if (vd > hi) return __fsub_rn(vd, hi);
  return 0.0f;
}

__device__ __forceinline__ float4 enclose(double mu, double sd) {
  return make_float4(__double2float_rd(mu), __double2float_ru(mu), __double2float_rd(sd),
                     __double2float_ru(sd));
}

// the float32 enclosures follow the float64 statistics of all nq queries
__device__ __forceinline__ float4* ivstat_enclosures(double* ivstat, int nq, int n_iv) {
  return reinterpret_cast<float4*>(ivstat + (size_t)nq * n_iv * 2);
}
__device__ __forceinline__ const float4* ivstat_enclosures(const double* ivstat, int nq,
                                                           int n_iv) {
  return reinterpret_cast<const float4*>(ivstat + (size_t)nq * n_iv * 2);
}

// one segment's term l (gap_mu^2 + gap_sigma^2) in float32, in this order
__device__ __forceinline__ float seg_term(float4 st, float4 syn, float len) {
  const float gm = gap32(st.x, st.y, syn.x, syn.y);
  const float gs = gap32(st.z, st.w, syn.z, syn.w);
  return __fmul_rn(len, __fadd_rn(__fmul_rn(gm, gm), __fmul_rn(gs, gs)));
}

// query statistics of every distinct segment interval: ivstat [nq][n_iv][2]
// float64, then their enclosures [nq][n_iv] float4
__global__ void ds_interval_kernel(DsTables T, const double* __restrict__ P, int nq, int m,
                                   double* __restrict__ ivstat) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nq * T.n_iv) return;
  const int q = (int)(t / T.n_iv), iv = (int)(t % T.n_iv);
  const double* p1 = P + (size_t)q * 2 * (m + 1);
  double mu, sd;
  interval_stat(p1, p1 + m + 1, T.iv_s[iv], T.iv_e[iv], mu, sd);
  ivstat[2 * t] = mu;
  ivstat[2 * t + 1] = sd;
  ivstat_enclosures(ivstat, nq, T.n_iv)[t] = enclose(mu, sd);
}

// Node bound: sum over the node's segments of l_r (gap_mu^2 + gap_sigma^2).
// Large trees: each thread takes one node for a tile of QT queries, so a
// node's synopses are read once per tile instead of once per query (there the
// synopses, not the arithmetic, are the traffic); every (query, node) sum runs
// over the node's segments in order, as in ds_node_leaf_kernel.
template <int QT>
__global__ void ds_node_tiled_kernel(DsTables T, const double* __restrict__ ivstat, int nq,
                                     double* __restrict__ node_lb) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int q0 = blockIdx.y * QT;
  if (v >= T.n_nodes) return;
  const int nqt = min(QT, nq - q0);
  const float4* st = ivstat_enclosures(ivstat, nq, T.n_iv);
  float acc[QT];
#pragma unroll
  for (int qq = 0; qq < QT; ++qq) acc[qq] = 0.0f;
  for (int r = T.seg_off[v]; r < T.seg_off[v + 1]; ++r) {
    const int iv = T.seg_iv[r];
    const float4 syn = T.syn32[r];
    const float len = (float)(T.iv_e[iv] - T.iv_s[iv]);
#pragma unroll
    for (int qq = 0; qq < QT; ++qq) {
      if (qq >= nqt) break;
      acc[qq] = __fadd_rn(acc[qq], seg_term(st[(size_t)(q0 + qq) * T.n_iv + iv], syn, len));
    }
  }
#pragma unroll
  for (int qq = 0; qq < QT; ++qq)
    if (qq < nqt) node_lb[(size_t)(q0 + qq) * T.n_nodes + v] = (double)acc[qq];
}

// Node and leaf bounds of one query per block (trees of fewer than 2048
// nodes): the node bounds, each the float32 sum over the node's segments in
// order, stay in shared memory, and each leaf takes the maximum over
// its root-to-leaf path from there, so no node bound goes through global
// memory and one launch replaces two.
__global__ void ds_node_leaf_kernel(DsTables T, const double* __restrict__ ivstat, int nq,
                                    double* __restrict__ leaf_lb) {
  extern __shared__ float s_node[];  // [n_nodes]
  const int q = blockIdx.x;
  const float4* st = ivstat_enclosures(ivstat, nq, T.n_iv) + (size_t)q * T.n_iv;
  for (int v = threadIdx.x; v < T.n_nodes; v += blockDim.x) {
    float acc = 0.0f;
    for (int r = T.seg_off[v]; r < T.seg_off[v + 1]; ++r) {
      const int iv = T.seg_iv[r];
      const float len = (float)(T.iv_e[iv] - T.iv_s[iv]);
      acc = __fadd_rn(acc, seg_term(st[iv], T.syn32[r], len));
    }
    s_node[v] = acc;
  }
  __syncthreads();
  for (int l = threadIdx.x; l < T.n_leaves; l += blockDim.x) {
    float best = 0.0f;
    for (int i = T.path_off[l]; i < T.path_off[l + 1]; ++i) best = fmaxf(best, s_node[T.path[i]]);
    leaf_lb[(size_t)q * T.n_leaves + l] = (double)best;
  }
}

// leaf bound = max over the root-to-leaf path
__global__ void ds_leaf_kernel(DsTables T, const double* __restrict__ node_lb, int nq,
                               double* __restrict__ leaf_lb) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nq * T.n_leaves) return;
  const int q = (int)(t / T.n_leaves), l = (int)(t % T.n_leaves);
  const double* nl = node_lb + (size_t)q * T.n_nodes;
  double best = 0.0;
  for (int i = T.path_off[l]; i < T.path_off[l + 1]; ++i) {
    const double v = nl[T.path[i]];
    if (v > best) best = v;
  }
  leaf_lb[t] = best;
}

__global__ void ds_route_kernel(DsTables T, const double* __restrict__ ivstat, int nq,
                                int32_t* __restrict__ route) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const double* st = ivstat + (size_t)q * T.n_iv * 2;
  int v = T.root;
  for (int guard = 0; guard < T.n_nodes && T.node_leaf[v] < 0; ++guard) {
    const int iv = T.split_iv[v];
    const double val = T.split_sd[v] ? st[2 * iv + 1] : st[2 * iv];
    v = (val < T.thresh[v]) ? T.left[v] : T.right[v];
  }
  route[q] = T.node_leaf[v];
}

// One block per query: the interval statistics go to global memory (for the
// node bounds) and to shared memory, where one thread then walks the tree to
// the query's route leaf without a global round trip per level.
__global__ void ds_interval_route_kernel(DsTables T, const double* __restrict__ P, int nq, int m,
                                         double* __restrict__ ivstat, int32_t* __restrict__ route) {
  extern __shared__ double st_s[];  // [n_iv][2]
  const int q = blockIdx.x;
  const double* p1 = P + (size_t)q * 2 * (m + 1);
  double* out = ivstat + (size_t)q * T.n_iv * 2;
  float4* enc = ivstat_enclosures(ivstat, nq, T.n_iv) + (size_t)q * T.n_iv;
  for (int iv = threadIdx.x; iv < T.n_iv; iv += blockDim.x) {
    double mu, sd;
    interval_stat(p1, p1 + m + 1, T.iv_s[iv], T.iv_e[iv], mu, sd);
    out[2 * iv] = mu;
    out[2 * iv + 1] = sd;
    enc[iv] = enclose(mu, sd);
    st_s[2 * iv] = mu;
    st_s[2 * iv + 1] = sd;
  }
  __syncthreads();
  if (threadIdx.x != 0 || !route) return;
  int v = T.root;
  for (int guard = 0; guard < T.n_nodes && T.node_leaf[v] < 0; ++guard) {
    const int iv = T.split_iv[v];
    const double val = T.split_sd[v] ? st_s[2 * iv + 1] : st_s[2 * iv];
    v = (val < T.thresh[v]) ? T.left[v] : T.right[v];
  }
  route[q] = T.node_leaf[v];
}

// ---------------------------------------------------------------- iSAX
// PAA values [nq][w] float64, then their enclosures [nq][w] float2 {down, up}
__global__ void isax_paa_kernel(IsaxTables T, const double* __restrict__ P, int nq, int m,
                                double* __restrict__ paa) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nq * T.w) return;
  const int q = t / T.w, j = t % T.w;
  const int l = m / T.w;
  const double* p1 = P + (size_t)q * 2 * (m + 1);
  const double a = __ddiv_rn(__dsub_rn(p1[(j + 1) * l], p1[j * l]), (double)l);
  paa[t] = a;
  reinterpret_cast<float2*>(paa + (size_t)nq * T.w)[t] =
      make_float2(__double2float_rd(a), __double2float_ru(a));
}

// MINDIST^2 of each leaf's word: sum_j l (gap(PAA_j, [beta_lo, beta_hi]))^2
__global__ void isax_leaf_kernel(IsaxTables T, const double* __restrict__ paa, int nq, int m,
                                 double* __restrict__ leaf_lb) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nq * T.n_leaves) return;
  const int q = (int)(t / T.n_leaves), lf = (int)(t % T.n_leaves);
  const float len = (float)(m / T.w);
  const float2* a = reinterpret_cast<const float2*>(paa + (size_t)nq * T.w) + (size_t)q * T.w;
  const int32_t* lo = T.lo_sym + (size_t)lf * T.w;
  const int32_t* hi = T.hi_sym + (size_t)lf * T.w;
  float acc = 0.0f;
  for (int j = 0; j < T.w; ++j) {
    const float2 v = a[j];
    const float g = gap32(v.x, v.y, T.beta32[lo[j]].x, T.beta32[hi[j]].y);
    acc = __fadd_rn(acc, __fmul_rn(len, __fmul_rn(g, g)));
  }
  leaf_lb[t] = (double)acc;
}

__device__ int sax_symbol(const double* beta, int C, double v) {
  // number of breakpoints beta_1 .. beta_{C-1} that are <= v
  int lo = 1, hi = C;  // answer in [0, C-1]
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (beta[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo - 1;
}

__global__ void isax_route_kernel(IsaxTables T, const double* __restrict__ paa,
                                  const double* __restrict__ leaf_lb, int nq,
                                  int32_t* __restrict__ route) {
  const int q = blockIdx.x;
  if (q >= nq) return;
  __shared__ int s_leaf;
  __shared__ int s_sym[32];
  const int C = 1 << T.bits;
  if (threadIdx.x < T.w) s_sym[threadIdx.x] = sax_symbol(T.beta, C, paa[(size_t)q * T.w + threadIdx.x]);
  __syncthreads();
  if (threadIdx.x == 0) {
    int key = 0;
    for (int j = 0; j < T.w; ++j) key = (key << 1) | (s_sym[j] >> (T.bits - 1));
    int v = T.root_child[key];
    for (int guard = 0; v >= 0 && guard < T.n_nodes && T.isplit[v] >= 0; ++guard) {
      const int j = T.isplit[v];
      const int have = T.node_bits[(size_t)v * T.w + j];
      v = ((s_sym[j] >> (T.bits - have - 1)) & 1) ? T.right[v] : T.left[v];
    }
    s_leaf = (v >= 0) ? T.node_leaf[v] : -1;
  }
  __syncthreads();
  if (s_leaf >= 0) {
    if (threadIdx.x == 0) route[q] = s_leaf;
    return;
  }
  // no leaf on the query's own path: the leaf of smallest (LB^2, id)
  __shared__ double s_lb[kThreads];
  __shared__ int s_id[kThreads];
  double best = DBL_MAX;
  int bid = 0x7fffffff;
  const double* row = leaf_lb + (size_t)q * T.n_leaves;
  for (int l = threadIdx.x; l < T.n_leaves; l += blockDim.x) {
    const double v = row[l];
    if (v < best || (v == best && l < bid)) {
      best = v;
      bid = l;
    }
  }
  s_lb[threadIdx.x] = best;
  s_id[threadIdx.x] = bid;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      const double o = s_lb[threadIdx.x + off];
      const int oi = s_id[threadIdx.x + off];
      if (o < s_lb[threadIdx.x] || (o == s_lb[threadIdx.x] && oi < s_id[threadIdx.x])) {
        s_lb[threadIdx.x] = o;
        s_id[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) route[q] = s_id[0];
}

// Scheduling keys: the route leaf of every query from its prefix sums, one
// thread per query walking the tree (no per-interval or per-leaf tables).  An
// iSAX query whose own path ends at no leaf gets key n_leaves (the search
// itself then routes it to its smallest-bound leaf).
__global__ void ds_route_key_kernel(DsTables T, const double* __restrict__ P, int nq, int m,
                                    int32_t* __restrict__ key) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const double* p1 = P + (size_t)q * 2 * (m + 1);
  int v = T.root;
  for (int guard = 0; guard < T.n_nodes && T.node_leaf[v] < 0; ++guard) {
    const int iv = T.split_iv[v];
    double mu, sd;
    interval_stat(p1, p1 + m + 1, T.iv_s[iv], T.iv_e[iv], mu, sd);
    const double val = T.split_sd[v] ? sd : mu;
    v = (val < T.thresh[v]) ? T.left[v] : T.right[v];
  }
  key[q] = T.node_leaf[v];
}

__global__ void isax_route_key_kernel(IsaxTables T, const double* __restrict__ P, int nq, int m,
                                      int32_t* __restrict__ key) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const double* p1 = P + (size_t)q * 2 * (m + 1);
  const int l = m / T.w, C = 1 << T.bits;
  int sym[32];
  int rk = 0;
  for (int j = 0; j < T.w; ++j) {
    const double a = __ddiv_rn(__dsub_rn(p1[(j + 1) * l], p1[j * l]), (double)l);
    sym[j] = sax_symbol(T.beta, C, a);
    rk = (rk << 1) | (sym[j] >> (T.bits - 1));
  }
  int v = T.root_child[rk];
  for (int guard = 0; v >= 0 && guard < T.n_nodes && T.isplit[v] >= 0; ++guard) {
    const int j = T.isplit[v];
    const int have = T.node_bits[(size_t)v * T.w + j];
    v = ((sym[j] >> (T.bits - have - 1)) & 1) ? T.right[v] : T.left[v];
  }
  key[q] = (v >= 0 && T.node_leaf[v] >= 0) ? T.node_leaf[v] : T.n_leaves;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void launch_prefix(const float* Q, int nq, int mp, int m, double* P, cudaStream_t s) {
  if (nq <= 0) return;
  prefix_kernel<<<blocks_for(nq, 64), 64, 0, s>>>(Q, nq, mp, m, P);
  LF_CHECK_LAUNCH();
}

void launch_ds_bounds(const DsTables& T, const double* P, int nq, int m, double* ivstat,
                      double* node_lb, double* leaf_lb, int32_t* route, cudaStream_t s) {
  if (nq <= 0) return;
  const size_t st_bytes = (size_t)T.n_iv * 2 * sizeof(double);
  const bool fused = st_bytes <= 48 * 1024;
  if (fused) {
    ds_interval_route_kernel<<<nq, kThreads, st_bytes, s>>>(T, P, nq, m, ivstat, route);
  } else {
    ds_interval_kernel<<<blocks_for((int64_t)nq * T.n_iv, kThreads), kThreads, 0, s>>>(T, P, nq, m,
                                                                                      ivstat);
  }
  LF_CHECK_LAUNCH();
  if (T.n_nodes >= 2048) {
    // large trees: tiles of 8 queries per thread share each node's synopses
    dim3 grid(blocks_for(T.n_nodes, kThreads), blocks_for(nq, 8));
    ds_node_tiled_kernel<8><<<grid, kThreads, 0, s>>>(T, ivstat, nq, node_lb);
    LF_CHECK_LAUNCH();
    ds_leaf_kernel<<<blocks_for((int64_t)nq * T.n_leaves, kThreads), kThreads, 0, s>>>(
        T, node_lb, nq, leaf_lb);
  } else {
    ds_node_leaf_kernel<<<nq, 256, sizeof(float) * T.n_nodes, s>>>(T, ivstat, nq, leaf_lb);
  }
  LF_CHECK_LAUNCH();
  if (route && !fused) {
    ds_route_kernel<<<blocks_for(nq, 64), 64, 0, s>>>(T, ivstat, nq, route);
    LF_CHECK_LAUNCH();
  }
}

void launch_isax_bounds(const IsaxTables& T, const double* P, int nq, int m, double* paa,
                        double* leaf_lb, int32_t* route, cudaStream_t s) {
  if (nq <= 0) return;
  isax_paa_kernel<<<blocks_for(nq * T.w, kThreads), kThreads, 0, s>>>(T, P, nq, m, paa);
  LF_CHECK_LAUNCH();
  isax_leaf_kernel<<<blocks_for((int64_t)nq * T.n_leaves, kThreads), kThreads, 0, s>>>(
      T, paa, nq, m, leaf_lb);
  LF_CHECK_LAUNCH();
  if (route) {
    isax_route_kernel<<<nq, kThreads, 0, s>>>(T, paa, leaf_lb, nq, route);
    LF_CHECK_LAUNCH();
  }
}

void launch_route_keys(const leafi_index* ix, const double* P, int nq, int32_t* key,
                       cudaStream_t s) {
  if (nq <= 0) return;
  if (ix->tree.type == LEAFI_DSTREE)
    ds_route_key_kernel<<<blocks_for(nq, 64), 64, 0, s>>>(ix->ds(), P, nq, ix->m, key);
  else
    isax_route_key_kernel<<<blocks_for(nq, 64), 64, 0, s>>>(ix->isax(), P, nq, ix->m, key);
  LF_CHECK_LAUNCH();
}

}  // namespace leafi
