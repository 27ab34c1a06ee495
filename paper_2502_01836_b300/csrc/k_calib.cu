// Auto-tuner learning (Alg. 4) on the device.
//
// Inputs per calibration query c: LB^2 and the k best keys of every leaf
// (from the leaf scan), the route leaf, and the filter predictions.  Step 1:
// alpha_f,c = |d^L - d^f| sorted descending per filter.  Step 2: for every
// sorted position j (one block each) every calibration query's search is
// simulated with offsets alpha_f,(j), in the same wave schedule as the real
// search; the quality at j is the share of the true top-k that lies in
// searched leaves (any such series is in the result).  Step 3: qprime is the
// running minimum over j.
#include <cfloat>
#include <climits>

#include "internal.h"

namespace leafi {
namespace {

typedef unsigned long long u64;
constexpr double kDeflate = 1.0 - 1e-4;
constexpr int kMaxSortN = 4096;
constexpr int kMaxWave = 65536;

__device__ __forceinline__ float key_d2(u64 k) { return __uint_as_float((uint32_t)(k >> 32)); }

__global__ void alpha_kernel(int nc, int L, int F, int stride, const u64* __restrict__ lk,
                             const float* __restrict__ P, const int32_t* __restrict__ filter_leaf,
                             double* __restrict__ alpha) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= F * nc) return;
  const int f = t / nc, c = t % nc;
  const u64 key = lk[((size_t)c * L + filter_leaf[f]) * stride];
  const float dl = __fsqrt_rn(key_d2(key));
  alpha[t] = fabs(__dsub_rn((double)dl, (double)P[(size_t)c * F + f]));
}

// sort each row of n doubles in descending order (one block per row)
__global__ void sort_desc_kernel(double* __restrict__ rows, int n) {
  __shared__ double buf[kMaxSortN];
  double* row = rows + (size_t)blockIdx.x * n;
  int n2 = 2;
  while (n2 < n) n2 <<= 1;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) buf[i] = i < n ? row[i] : -DBL_MAX;
  __syncthreads();
  for (int size = 2; size <= n2; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < (n2 >> 1); i += blockDim.x) {
        const int pos = 2 * i - (i & (stride - 1));
        const int partner = pos + stride;
        const bool desc = (pos & size) == 0;
        const double x = buf[pos], y = buf[partner];
        if ((x < y) == desc) {
          buf[pos] = y;
          buf[partner] = x;
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < n; i += blockDim.x) row[i] = buf[i];
}

// visiting order: leaves by ascending (LB^2, leaf id), one block per query
__global__ void order_kernel(int L, const double* __restrict__ lb2, int32_t* __restrict__ ord) {
  extern __shared__ double sbuf[];
  double* key = sbuf;
  int* id = reinterpret_cast<int*>(sbuf + kMaxSortN);
  const double* row = lb2 + (size_t)blockIdx.x * L;
  int n2 = 2;
  while (n2 < L) n2 <<= 1;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    key[i] = i < L ? row[i] : DBL_MAX;
    id[i] = i < L ? i : INT_MAX;
  }
  __syncthreads();
  for (int size = 2; size <= n2; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < (n2 >> 1); i += blockDim.x) {
        const int pos = 2 * i - (i & (stride - 1));
        const int partner = pos + stride;
        const bool asc = (pos & size) == 0;
        const double x = key[pos], y = key[partner];
        const int xi = id[pos], yi = id[partner];
        const bool gt = x > y || (x == y && xi > yi);
        if (gt == asc) {
          key[pos] = y;
          key[partner] = x;
          id[pos] = yi;
          id[partner] = xi;
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < L; i += blockDim.x) ord[(size_t)blockIdx.x * L + i] = id[i];
}

// Visiting order for more than kMaxSortN leaves: the same bitonic network on
// n2 = next power of two >= L entries held in global scratch (one block per
// query); compare-exchange stages with a stride of at least one tile run on
// the global arrays, the rest of each stage group tile by tile in shared memory.
constexpr int kOrderThreads = 1024;

__device__ __forceinline__ void cx_pair(double* key, int* id, int pos, int partner, bool asc) {
  const double x = key[pos], y = key[partner];
  const int xi = id[pos], yi = id[partner];
  const bool gt = x > y || (x == y && xi > yi);
  if (gt == asc) {
    key[pos] = y;
    key[partner] = x;
    id[pos] = yi;
    id[partner] = xi;
  }
}

// strides s_hi .. 1 of bitonic stage group `size` on one tile in shared memory
__device__ void tile_stages(double* gkey, int* gid, double* tk, int* ti, int t0, int size, int s_hi) {
  for (int i = threadIdx.x; i < kMaxSortN; i += blockDim.x) {
    tk[i] = gkey[t0 + i];
    ti[i] = gid[t0 + i];
  }
  __syncthreads();
  for (int stride = s_hi; stride > 0; stride >>= 1) {
    for (int t = threadIdx.x; t < kMaxSortN / 2; t += blockDim.x) {
      const int pos = 2 * t - (t & (stride - 1));
      cx_pair(tk, ti, pos, pos + stride, ((t0 + pos) & size) == 0);
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < kMaxSortN; i += blockDim.x) {
    gkey[t0 + i] = tk[i];
    gid[t0 + i] = ti[i];
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kOrderThreads) order_global_kernel(
    int L, int n2, const double* __restrict__ lb2, double* __restrict__ kbuf,
    int* __restrict__ ibuf, int32_t* __restrict__ ord) {
  extern __shared__ double tsm[];
  double* tk = tsm;
  int* ti = reinterpret_cast<int*>(tsm + kMaxSortN);
  const int q = blockIdx.x;
  double* key = kbuf + (size_t)q * n2;
  int* id = ibuf + (size_t)q * n2;
  const double* row = lb2 + (size_t)q * L;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    key[i] = i < L ? row[i] : DBL_MAX;
    id[i] = i < L ? i : INT_MAX;
  }
  __syncthreads();
  // stage groups up to one tile: every tile sorted in shared memory
  for (int size = 2; size <= kMaxSortN; size <<= 1)
    for (int t0 = 0; t0 < n2; t0 += kMaxSortN) tile_stages(key, id, tk, ti, t0, size, size >> 1);
  for (int size = 2 * kMaxSortN; size <= n2; size <<= 1) {
    for (int stride = size >> 1; stride >= kMaxSortN; stride >>= 1) {
      for (int t = threadIdx.x; t < n2 / 2; t += blockDim.x) {
        const int pos = 2 * t - (t & (stride - 1));
        cx_pair(key, id, pos, pos + stride, (pos & size) == 0);
      }
      __syncthreads();
    }
    for (int t0 = 0; t0 < n2; t0 += kMaxSortN) tile_stages(key, id, tk, ti, t0, size, kMaxSortN >> 1);
  }
  for (int i = threadIdx.x; i < L; i += blockDim.x) ord[(size_t)q * L + i] = id[i];
}

// where the true top-k of each calibration query lies: cnt_true [nc][L]
__global__ void truth_kernel(int nc, int L, int kc, int stride, const u64* __restrict__ lk,
                             int32_t* __restrict__ heads, int32_t* __restrict__ cnt_true) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  int32_t* h = heads + (size_t)c * L;
  int32_t* ct = cnt_true + (size_t)c * L;
  for (int l = 0; l < L; ++l) {
    h[l] = 0;
    ct[l] = 0;
  }
  const u64* base = lk + (size_t)c * L * stride;
  for (int z = 0; z < kc; ++z) {
    u64 best = kNoKey;
    int bl = -1;
    for (int l = 0; l < L; ++l) {
      if (h[l] >= kc) continue;
      const u64 v = base[(size_t)l * stride + h[l]];
      if (v < best) {
        best = v;
        bl = l;
      }
    }
    if (bl < 0) break;
    ct[bl] += 1;
    h[bl] += 1;
  }
}

__device__ void merge_list(u64* w, int& cnt, int kc, const u64* src) {
  for (int z = 0; z < kc; ++z) {
    const u64 e = src[z];
    if (e == kNoKey) break;
    if (cnt == kc && e >= w[kc - 1]) break;
    int p = cnt < kc ? cnt : kc - 1;
    while (p > 0 && w[p - 1] > e) {
      w[p] = w[p - 1];
      --p;
    }
    w[p] = e;
    if (cnt < kc) ++cnt;
  }
}

constexpr int kSimThreads = 128;

__global__ void __launch_bounds__(kSimThreads) sim_kernel(CalibArgs a, long long* __restrict__ hits_j) {
  const int j = blockIdx.x;
  const int L = a.L, kc = a.kc;
  long long hits = 0;
  for (int c = threadIdx.x; c < a.nc; c += blockDim.x) {
    u64* w = a.work + ((size_t)j * a.nc + c) * kc;
    int cnt = 0;
    const int route = a.route[c];
    const u64* lists = a.lk + (size_t)c * L * a.lk_stride;
    const int32_t* ct = a.cnt_true + (size_t)c * L;
    const int32_t* ord = a.ord + (size_t)c * L;
    const double* lb = a.lb2 + (size_t)c * L;
    merge_list(w, cnt, kc, lists + (size_t)route * a.lk_stride);
    long long h = ct[route];
    float bsf2 = (cnt == kc) ? key_d2(w[kc - 1]) : __int_as_float(0x7f800000);
    int cursor = 0;
    for (int guard = 0; guard <= L; ++guard) {
      // pick the wave with the bound of its start, then walk the same range
      // again to merge the picked leaves (no per-thread pick list)
      const int c0 = cursor;
      const double bsf = (double)__fsqrt_rn(bsf2);
      int np = 0;
      while (cursor < L && np < a.W) {
        const int leaf = ord[cursor];
        if (leaf == route) {
          ++cursor;
          continue;
        }
        if (__dmul_rn(lb[leaf], kDeflate) > (double)bsf2) {
          cursor = L;
          break;
        }
        const int f = a.leaf_filter[leaf];
        if (f >= 0) {
          const double df = __dsub_rn((double)a.P[(size_t)c * a.F + f], a.alpha[(size_t)f * a.nc + j]);
          if (df > bsf) {
            ++cursor;
            continue;
          }
        }
        ++np;
        ++cursor;
      }
      if (np == 0) break;
      int taken = 0;
      for (int p = c0; taken < np; ++p) {
        const int leaf = ord[p];
        if (leaf == route) continue;
        const int f = a.leaf_filter[leaf];
        if (f >= 0 &&
            __dsub_rn((double)a.P[(size_t)c * a.F + f], a.alpha[(size_t)f * a.nc + j]) > bsf)
          continue;
        merge_list(w, cnt, kc, lists + (size_t)leaf * a.lk_stride);
        h += ct[leaf];
        ++taken;
      }
      bsf2 = (cnt == kc) ? key_d2(w[kc - 1]) : __int_as_float(0x7f800000);
    }
    hits += h;
  }
  __shared__ long long red[kSimThreads];
  red[threadIdx.x] = hits;
  __syncthreads();
  for (int off = kSimThreads / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) hits_j[j] = red[0];
}

__global__ void qprime_kernel(int nc, int kk, const long long* __restrict__ hits,
                              double* __restrict__ qprime) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double run = __longlong_as_double(0x7ff0000000000000ll);
  const double denom = __dmul_rn((double)kk, (double)nc);
  for (int j = 0; j < nc; ++j) {
    const double q = __ddiv_rn((double)hits[j], denom);
    if (q < run) run = q;
    qprime[j] = run;
  }
}

}  // namespace

int calib_max_sort() { return kMaxSortN; }

size_t leaf_order_scratch(int nq, int L) {
  if (L <= kMaxSortN) return 0;
  size_t n2 = kMaxSortN;
  while (n2 < (size_t)L) n2 <<= 1;
  return (size_t)nq * n2 * (sizeof(double) + sizeof(int));
}

void launch_leaf_order(int nq, int L, const double* lb2, int32_t* ord, cudaStream_t s,
                       void* scratch) {
  if (nq <= 0) return;
  const size_t smem = kMaxSortN * (sizeof(double) + sizeof(int));
  if (L <= kMaxSortN) {
    LF_CUDA(cudaFuncSetAttribute(order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    order_kernel<<<nq, 256, smem, s>>>(L, lb2, ord);
    LF_CHECK_LAUNCH();
    return;
  }
  if (!scratch) fail(LEAFI_EINTERNAL, "visiting order of %d leaves needs scratch", L);
  int n2 = kMaxSortN;
  while (n2 < L) n2 <<= 1;
  double* kbuf = static_cast<double*>(scratch);
  int* ibuf = reinterpret_cast<int*>(kbuf + (size_t)nq * n2);
  LF_CUDA(cudaFuncSetAttribute(order_global_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem));
  order_global_kernel<<<nq, kOrderThreads, smem, s>>>(L, n2, lb2, kbuf, ibuf, ord);
  LF_CHECK_LAUNCH();
}
int calib_max_wave() { return kMaxWave; }

void launch_calib_alpha(const CalibArgs& a, cudaStream_t s) {
  if (a.F <= 0) return;
  if (a.nc > kMaxSortN) fail(LEAFI_EINVAL, "at most %d calibration queries", kMaxSortN);
  alpha_kernel<<<(a.F * a.nc + 255) / 256, 256, 0, s>>>(a.nc, a.L, a.F, a.lk_stride, a.lk, a.P,
                                                        a.filter_leaf, a.alpha);
  LF_CHECK_LAUNCH();
  sort_desc_kernel<<<a.F, 256, 0, s>>>(a.alpha, a.nc);
  LF_CHECK_LAUNCH();
}

void launch_calib_sim(const CalibArgs& a, cudaStream_t s) {
  if (a.W > kMaxWave) fail(LEAFI_EINVAL, "wave > %d", kMaxWave);
  launch_leaf_order(a.nc, a.L, a.lb2, a.ord, s, a.order_scratch);
  // `work` doubles as the truth kernel's per-leaf head pointers (nc * L ints)
  truth_kernel<<<(a.nc + 63) / 64, 64, 0, s>>>(a.nc, a.L, a.kc, a.lk_stride, a.lk,
                                               reinterpret_cast<int32_t*>(a.work), a.cnt_true);
  LF_CHECK_LAUNCH();
  sim_kernel<<<a.nc, kSimThreads, 0, s>>>(a, a.hits);
  LF_CHECK_LAUNCH();
  qprime_kernel<<<1, 32, 0, s>>>(a.nc, a.kk, a.hits, a.qprime);
  LF_CHECK_LAUNCH();
}

}  // namespace leafi
