// Leaf search (SearchNode of Alg. 2), candidate merging, and the wave
// scheduler's select step.
//
// A scan round takes (slot, query, leaf) pairs, groups them by leaf and cuts
// each leaf into work items of (series part) x (group of up to kG queries).
// One block per item streams the part's series through shared memory in
// chunks of kRows rows; thread (row, octet) computes the canonical squared
// distance of its row to kQPT queries:  acc = fmaf(q_i - x_i, q_i - x_i, acc)
// for i = 0 .. m-1 in order, so every distance equals the oracle's bit for
// bit and no re-check is needed.  Each query keeps its k best (d^2, id) keys
// of the part in shared memory (warp-cooperative sorted insertion); the part's
// list is appended to the slot's candidate buffer and a merge kernel folds all
// candidates into the slot's running top-k.
#include <cfloat>
#include <climits>

#include "internal.h"

namespace leafi {
namespace {

typedef unsigned long long u64;

constexpr int kRows = 64;                  // series rows per chunk
constexpr int kQPT = 8;                    // queries per thread
constexpr int kOct = 2;                    // query octets per block
constexpr int kG = kQPT * kOct;            // queries per work item
constexpr int kScanThreads = kRows * kOct; // one thread per (row, octet)
constexpr int kMergeThreads = 256;
constexpr int kMergeCap = 2048;
constexpr double kDeflate = 1.0 - 1e-4;    // LB^2 (1 - 1e-4) > bsf^2 prunes

__device__ __forceinline__ u64 make_key(float d2, uint32_t id) {
  return ((u64)__float_as_uint(d2) << 32) | (u64)id;
}

__device__ __forceinline__ float key_d2(u64 k) { return __uint_as_float((uint32_t)(k >> 32)); }

// Insert `key` into the ascending list (cnt entries, capacity k <= 128);
// every lane of the warp calls it with the same arguments.
__device__ int warp_insert(u64* list, int cnt, int k, u64 key, int lane) {
  int less = 0;
  for (int p = lane; p < cnt; p += 32) less += (list[p] < key) ? 1 : 0;
  const int pos = (int)__reduce_add_sync(0xffffffffu, (unsigned)less);
  const int newcnt = cnt + 1 < k ? cnt + 1 : k;
  u64 v[LEAFI_MAX_K / 32];
#pragma unroll
  for (int j = 0; j < LEAFI_MAX_K / 32; ++j) {
    const int p = pos + lane + 32 * j;
    v[j] = (p < newcnt - 1) ? list[p] : 0ull;
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < LEAFI_MAX_K / 32; ++j) {
    const int p = pos + lane + 32 * j;
    if (p < newcnt - 1) list[p + 1] = v[j];
  }
  if (lane == 0 && pos < k) list[pos] = key;
  __syncwarp();
  return newcnt;
}

__device__ __forceinline__ u64 warp_min_u64(u64 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const u64 w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}

__global__ void __launch_bounds__(kScanThreads) scan_kernel(ScanArgs a,
                                                            const int32_t* __restrict__ n_items_dev,
                                                            const int32_t* __restrict__ slot_k) {
  extern __shared__ float4 sm4[];
  const int rs = a.mp + 4;  // padded row stride in floats (16-byte multiple)
  const int r4 = rs / 4, m4 = a.mp / 4;
  float4* Xs = sm4;                                                  // [kRows][rs]
  float4* Qs = Xs + kRows * r4;                                      // [kG][rs]
  u64* lists = reinterpret_cast<u64*>(Qs + kG * r4);                 // [kG][a.k]
  u64* stage = lists + kG * a.k;                                     // [kG][kRows]
  __shared__ int s_cnt[kG], s_nst[kG], s_slot[kG], s_k[kG];
  __shared__ u64 s_thr[kG];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = kScanThreads / 32;
  const int n_items = *n_items_dev;
  const float4* X4 = reinterpret_cast<const float4*>(a.X);
  const float4* Q4 = reinterpret_cast<const float4*>(a.Q);
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    // leaf of this item: largest l with item_off[l] <= item
    int lo = 0, hi = a.L - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.item_off[mid] <= item) lo = mid; else hi = mid - 1;
    }
    const int leaf = lo;
    const int cnt = a.grp_off[leaf + 1] - a.grp_off[leaf];
    const int ngroups = (cnt + kG - 1) / kG;
    const int local = item - a.item_off[leaf];
    const int part = local / ngroups, grp = local % ngroups;
    const int64_t p0 = a.leaf_off[leaf] + (int64_t)part * a.part;
    const int64_t p1 = min(p0 + (int64_t)a.part, a.leaf_off[leaf + 1]);
    const int nqg = min(kG, cnt - grp * kG);
    const Pair* pr = a.pairs + a.grp_off[leaf] + grp * kG;
    if (tid < kG) {
      s_cnt[tid] = 0;
      if (tid < nqg) {
        const int slot = pr[tid].slot;
        s_slot[tid] = slot;
        s_thr[tid] = __ldcg(&a.thr[slot]);  // as finished items of the round lowered it
        s_k[tid] = slot_k ? slot_k[slot] : a.k;
      }
    }
    for (int idx = tid; idx < nqg * m4; idx += kScanThreads) {
      const int qq = idx / m4, c = idx % m4;
      Qs[qq * r4 + c] = Q4[(size_t)pr[qq].q * m4 + c];
    }
    const int row = tid % kRows, oct = tid / kRows;
    for (int64_t c0 = p0; c0 < p1; c0 += kRows) {
      const int ns = (int)min((int64_t)kRows, p1 - c0);
      for (int idx = tid; idx < ns * m4; idx += kScanThreads) {
        const int r = idx / m4, c = idx % m4;
        Xs[r * r4 + c] = X4[(size_t)(c0 + r) * m4 + c];
      }
      if (tid < kG) s_nst[tid] = 0;
      __syncthreads();
      if (row < ns && oct * kQPT < nqg) {
        float acc[kQPT];
#pragma unroll
        for (int j = 0; j < kQPT; ++j) acc[j] = 0.0f;
        const float4* xr = Xs + row * r4;
        const float4* qb = Qs + oct * kQPT * r4;
        for (int c = 0; c < m4; ++c) {
          const float4 x = xr[c];
#pragma unroll
          for (int j = 0; j < kQPT; ++j) {
            const float4 q = qb[j * r4 + c];
            float t = __fsub_rn(q.x, x.x);
            acc[j] = __fmaf_rn(t, t, acc[j]);
            t = __fsub_rn(q.y, x.y);
            acc[j] = __fmaf_rn(t, t, acc[j]);
            t = __fsub_rn(q.z, x.z);
            acc[j] = __fmaf_rn(t, t, acc[j]);
            t = __fsub_rn(q.w, x.w);
            acc[j] = __fmaf_rn(t, t, acc[j]);
          }
        }
        const uint32_t id = (uint32_t)a.ids[c0 + row];
#pragma unroll
        for (int j = 0; j < kQPT; ++j) {
          const int q = oct * kQPT + j;
          if (q < nqg) {
            const u64 key = make_key(acc[j], id);
            const int kq = s_k[q];
            const u64 kth = (s_cnt[q] == kq) ? lists[q * a.k + kq - 1] : s_thr[q];
            if (key < kth) stage[q * kRows + atomicAdd(&s_nst[q], 1)] = key;
          }
        }
      }
      __syncthreads();
      for (int q = warp; q < nqg; q += nwarps) {
        const int nst = s_nst[q];
        if (nst == 0) continue;
        const int kq = s_k[q];
        u64* list = lists + q * a.k;
        int c = s_cnt[q];
        if (kq == 1) {
          u64 best = kNoKey;
          for (int e = lane; e < nst; e += 32) {
            const u64 v = stage[q * kRows + e];
            best = v < best ? v : best;
          }
          best = warp_min_u64(best);
          const u64 kth = (c == 1) ? list[0] : s_thr[q];
          if (best < kth) {
            if (lane == 0) list[0] = best;
            c = 1;
          }
        } else {
          for (int e = 0; e < nst; ++e) {
            const u64 key = stage[q * kRows + e];
            const u64 kth = (c == kq) ? list[kq - 1] : s_thr[q];
            if (key < kth) c = warp_insert(list, c, kq, key, lane);
          }
        }
        if (lane == 0) s_cnt[q] = c;
      }
      __syncthreads();
    }
    // append this part's list to the slot's candidates
    for (int q = warp; q < nqg; q += nwarps) {
      const int c = s_cnt[q];
      if (c == 0) continue;
      const int slot = s_slot[q];
      int base = 0;
      if (lane == 0) {
        base = atomicAdd(&a.cand_cnt[slot], c);
        // a full list's k-th key bounds the slot's final k-th key (each pair is
        // in one item only), so later items of the round may admit against it
        if (c == s_k[q]) atomicMin(&a.thr[slot], lists[q * a.k + c - 1]);
      }
      base = __shfl_sync(0xffffffffu, base, 0);
      if (base + c > a.cand_cap) {
        if (lane == 0) atomicOr(a.err, 1);
        continue;
      }
      for (int e = lane; e < c; e += 32) a.cand[(size_t)slot * a.cand_cap + base + e] = lists[q * a.k + e];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- grouping
__global__ void count_kernel(const Pair* __restrict__ pairs, const int32_t* __restrict__ npairs,
                             int32_t* __restrict__ cnt) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < *npairs) atomicAdd(&cnt[pairs[p].leaf], 1);
}

// Small-leaf packing (tensor-core scan only): the leaves are cut into windows
// of kPackWin consecutive ids; a window whose series fit one 128-row chunk,
// with at least two searched leaves whose pairs fit one query group, becomes a
// single work item (every pair only meets the rows of its own leaf);
// otherwise each searched leaf gives parts x groups items.
constexpr int kPackWin = 8;
constexpr int kPackRows = 128;

template <class CountT>
__device__ __forceinline__ bool window_packs(const CountT* cnt, const int64_t* __restrict__ leaf_off,
                                             int w0, int w1, int g) {
  if (leaf_off[w1] - leaf_off[w0] > kPackRows) return false;
  int picked = 0, pairs = 0;
  for (int l = w0; l < w1; ++l) {
    picked += cnt[l] > 0;
    pairs += cnt[l];
  }
  return picked >= 2 && pairs <= g;
}

__device__ __forceinline__ int leaf_items(int c, const int64_t* __restrict__ leaf_off, int l, int part,
                                          int g) {
  if (c == 0) return 0;
  const int64_t size = leaf_off[l + 1] - leaf_off[l];
  return (int)((size + part - 1) / part) * ((c + g - 1) / g);
}

// Work-item size of a round (tensor-core scan): candidate parts part_max,
// part_max / 2, ... (multiples of 128 rows, none below min_part); the largest
// whose item count reaches `target` (a few items per SM, so that a launch's
// items balance) is taken, else the smallest allowed.  target 0 keeps
// part_max.  The floor keeps small rounds (a batch's route leaves) from being
// cut into one-chunk items, whose fixed costs would dominate; such a round
// occupies fewer SMs and the other lanes' work takes the rest.
constexpr int kPartLevels = 5;

__device__ __forceinline__ int part_level(int part_max, int c) {
  const int p = part_max >> c;
  return p >= 128 ? (p / 128) * 128 : 128;
}

// thread's item counts per level have been added to tot[]; returns the level
__device__ __forceinline__ int pick_part_level(const int* tot, int target, int part_max,
                                                int min_part) {
  int c = 0;
  while (c + 1 < kPartLevels && tot[c] < target && part_level(part_max, c + 1) >= min_part) ++c;
  return c;
}

// exclusive scans of per-leaf pair counts and work-item counts (one block)
__global__ void offsets_kernel(int L, const int64_t* __restrict__ leaf_off, int part_max, int g,
                               int32_t* __restrict__ cnt, int32_t* __restrict__ grp_off,
                               int32_t* __restrict__ item_off, int32_t* __restrict__ n_items,
                               unsigned long long* __restrict__ stat,
                               int32_t* __restrict__ item_leaf, bool pack_small, int target,
                               int min_part, int32_t* __restrict__ part_out) {
  __shared__ int s_a[1024], s_b[1024];
  __shared__ int tot[kPartLevels];
  const int T = blockDim.x;
  const bool pack = item_leaf != nullptr && pack_small;
  // whole windows per thread when packing
  const int win = pack ? kPackWin : 1;
  const int per = ((L + T - 1) / T + win - 1) / win * win;
  const int l0 = min(L, (int)threadIdx.x * per), l1 = min(L, l0 + per);
  if (threadIdx.x < kPartLevels) tot[threadIdx.x] = 0;
  __syncthreads();
  int sa = 0, sbl[kPartLevels] = {0, 0, 0, 0, 0};
  unsigned long long distinct = 0;
  for (int w0 = l0; w0 < l1; w0 += win) {
    const int w1 = min(l1, w0 + win);
    for (int l = w0; l < w1; ++l) {
      sa += cnt[l];
      if (cnt[l] > 0) distinct += (unsigned long long)(leaf_off[l + 1] - leaf_off[l]);
    }
    if (pack && window_packs(cnt, leaf_off, w0, w1, g)) {
#pragma unroll
      for (int c = 0; c < kPartLevels; ++c) sbl[c] += 1;
    } else {
      for (int l = w0; l < w1; ++l)
#pragma unroll
        for (int c = 0; c < kPartLevels; ++c)
          sbl[c] += leaf_items(cnt[l], leaf_off, l, part_level(part_max, c), g);
    }
  }
  if (stat && distinct) atomicAdd(stat, distinct);
#pragma unroll
  for (int c = 0; c < kPartLevels; ++c)
    if (sbl[c]) atomicAdd(&tot[c], sbl[c]);
  __syncthreads();
  const int lev = pick_part_level(tot, target, part_max, min_part);
  const int part = part_level(part_max, lev);
  int sb = 0;
#pragma unroll
  for (int c = 0; c < kPartLevels; ++c)
    if (c == lev) sb = sbl[c];
  if (threadIdx.x == 0 && part_out) *part_out = part;
  s_a[threadIdx.x] = sa;
  s_b[threadIdx.x] = sb;
  __syncthreads();
  // Hillis-Steele inclusive scan over the per-thread sums
  for (int off = 1; off < T; off <<= 1) {
    const int va = threadIdx.x >= off ? s_a[threadIdx.x - off] : 0;
    const int vb = threadIdx.x >= off ? s_b[threadIdx.x - off] : 0;
    __syncthreads();
    s_a[threadIdx.x] += va;
    s_b[threadIdx.x] += vb;
    __syncthreads();
  }
  int ra = s_a[threadIdx.x] - sa, rb = s_b[threadIdx.x] - sb;
  for (int w0 = l0; w0 < l1; w0 += win) {
    const int w1 = min(l1, w0 + win);
    const bool packed = pack && window_packs(cnt, leaf_off, w0, w1, g);
    for (int l = w0; l < w1; ++l) {
      const int c = cnt[l];
      grp_off[l] = ra;
      item_off[l] = rb;
      ra += c;
      if (!packed) {
        const int ni = leaf_items(c, leaf_off, l, part, g);
        if (item_leaf)
          for (int i = 0; i < ni; ++i) item_leaf[rb + i] = l;
        rb += ni;
      }
    }
    if (packed) {
      item_leaf[rb] = -1 - w0;  // a packed window [w0, w0 + kPackWin)
      rb += 1;
    }
    for (int l = w0; l < w1; ++l) cnt[l] = 0;  // reused as the scatter fill counter
  }
  if (threadIdx.x == T - 1) {
    grp_off[L] = s_a[T - 1];
    item_off[L] = s_b[T - 1];
    *n_items = s_b[T - 1];
  }
}

// count + offsets + scatter in one block for indexes of up to kFuseLeaves
// leaves (the per-leaf counters live in shared memory)
constexpr int kFuseLeaves = 8192;

__global__ void __launch_bounds__(1024) group_fused_kernel(
    const Pair* __restrict__ pairs, const int32_t* __restrict__ npairs, int L,
    const int64_t* __restrict__ leaf_off, int part_max, int g, int32_t* __restrict__ grp_off,
    int32_t* __restrict__ item_off, int32_t* __restrict__ n_items, Pair* __restrict__ grouped,
    unsigned long long* __restrict__ stat, int32_t* __restrict__ item_leaf, bool pack_small,
    int target, int min_part, int32_t* __restrict__ part_out, RoundPrep rp) {
  __shared__ int cnt[kFuseLeaves];
  if (rp.topk) {
    // the following scan round's prep: lists padded past their counts, locks
    // released, shared upper bounds reset, work counter zeroed
    const int64_t tot = (int64_t)rp.nslots * rp.kstride;
    for (int64_t t = threadIdx.x; t < tot; t += blockDim.x) {
      const int slot = (int)(t / rp.kstride), z = (int)(t % rp.kstride);
      if (z >= rp.topk_cnt[slot]) rp.topk[t] = kNoKey;
      if (z == 0) {
        rp.glock[slot] = 0;
        if (rp.ub) rp.ub[slot] = __int_as_float(0x7f800000);
      }
    }
    if (threadIdx.x == 0) *rp.work = 0;
  }
  __shared__ int s_a[1024], s_b[1024];
  __shared__ int tot[kPartLevels];
  const int T = blockDim.x;
  const int np = *npairs;
  for (int l = threadIdx.x; l < L; l += T) cnt[l] = 0;
  if (threadIdx.x < kPartLevels) tot[threadIdx.x] = 0;
  __syncthreads();
  for (int p = threadIdx.x; p < np; p += T) atomicAdd(&cnt[pairs[p].leaf], 1);
  __syncthreads();
  const bool pack = item_leaf != nullptr && pack_small;
  // whole windows per thread when packing
  const int win = pack ? kPackWin : 1;
  const int per = ((L + T - 1) / T + win - 1) / win * win;
  const int l0 = min(L, (int)threadIdx.x * per), l1 = min(L, l0 + per);
  int sa = 0, sbl[kPartLevels] = {0, 0, 0, 0, 0};
  unsigned long long distinct = 0;
  for (int w0 = l0; w0 < l1; w0 += win) {
    const int w1 = min(l1, w0 + win);
    for (int l = w0; l < w1; ++l) {
      sa += cnt[l];
      if (cnt[l] > 0) distinct += (unsigned long long)(leaf_off[l + 1] - leaf_off[l]);
    }
    if (pack && window_packs(cnt, leaf_off, w0, w1, g)) {
#pragma unroll
      for (int c = 0; c < kPartLevels; ++c) sbl[c] += 1;
    } else {
      for (int l = w0; l < w1; ++l)
#pragma unroll
        for (int c = 0; c < kPartLevels; ++c)
          sbl[c] += leaf_items(cnt[l], leaf_off, l, part_level(part_max, c), g);
    }
  }
  if (stat && distinct) atomicAdd(stat, distinct);
#pragma unroll
  for (int c = 0; c < kPartLevels; ++c)
    if (sbl[c]) atomicAdd(&tot[c], sbl[c]);
  __syncthreads();
  const int lev = pick_part_level(tot, target, part_max, min_part);
  const int part = part_level(part_max, lev);
  int sb = 0;
#pragma unroll
  for (int c = 0; c < kPartLevels; ++c)
    if (c == lev) sb = sbl[c];
  if (threadIdx.x == 0 && part_out) *part_out = part;
  s_a[threadIdx.x] = sa;
  s_b[threadIdx.x] = sb;
  __syncthreads();
  for (int off = 1; off < T; off <<= 1) {
    const int va = threadIdx.x >= off ? s_a[threadIdx.x - off] : 0;
    const int vb = threadIdx.x >= off ? s_b[threadIdx.x - off] : 0;
    __syncthreads();
    s_a[threadIdx.x] += va;
    s_b[threadIdx.x] += vb;
    __syncthreads();
  }
  int ra = s_a[threadIdx.x] - sa, rb = s_b[threadIdx.x] - sb;
  for (int w0 = l0; w0 < l1; w0 += win) {
    const int w1 = min(l1, w0 + win);
    const bool packed = pack && window_packs(cnt, leaf_off, w0, w1, g);
    for (int l = w0; l < w1; ++l) {
      const int c = cnt[l];
      grp_off[l] = ra;
      item_off[l] = rb;
      if (!packed) {
        const int ni = leaf_items(c, leaf_off, l, part, g);
        if (item_leaf)
          for (int i = 0; i < ni; ++i) item_leaf[rb + i] = l;
        rb += ni;
      }
      cnt[l] = ra;  // becomes the leaf's fill cursor (the window's test already ran)
      ra += c;
    }
    if (packed) {
      item_leaf[rb] = -1 - w0;  // a packed window [w0, w0 + kPackWin)
      rb += 1;
    }
  }
  if (threadIdx.x == T - 1) {
    grp_off[L] = s_a[T - 1];
    item_off[L] = s_b[T - 1];
    *n_items = s_b[T - 1];
  }
  __syncthreads();
  for (int p = threadIdx.x; p < np; p += T) {
    const Pair pr = pairs[p];
    grouped[atomicAdd(&cnt[pr.leaf], 1)] = pr;
  }
}

// ------------------------------------------------ query groups sized by k
// For k > 1 the tensor-core scan keeps one top-k list per query and lane
// quarter in shared memory, so a work item's group of queries is bounded by
// the sum of their k (`budget` keys) as well as by 64 (the MMA's N).  Each
// leaf's pairs are cut greedily, in their grouped order, into such groups;
// the items of a leaf are (part, group) as before.
__device__ __forceinline__ int pair_k(const Pair& p, const int32_t* slot_k, int kstride) {
  return slot_k ? slot_k[p.slot] : kstride;
}

__global__ void vgroup_count_kernel(int L, const int32_t* __restrict__ grp_off,
                                    const Pair* __restrict__ grouped,
                                    const int32_t* __restrict__ slot_k, int kstride, int budget,
                                    int32_t* __restrict__ ngroups) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L) return;
  int n = 0, sum = 0, g = 0;
  for (int p = grp_off[l]; p < grp_off[l + 1]; ++p) {
    const int k = pair_k(grouped[p], slot_k, kstride);
    if (n == 64 || sum + k > budget) {
      ++g;
      n = 0;
      sum = 0;
    }
    ++n;
    sum += k;
  }
  ngroups[l] = g + (n > 0 ? 1 : 0);
}

// exclusive scans of per-leaf group counts and work-item counts (one block)
__global__ void vgroup_offsets_kernel(int L, const int64_t* __restrict__ leaf_off, int part_max,
                                      const int32_t* __restrict__ ngroups,
                                      int32_t* __restrict__ gfirst, int32_t* __restrict__ item_off,
                                      int32_t* __restrict__ n_items, int target, int min_part,
                                      int32_t* __restrict__ part_out) {
  __shared__ int s_a[1024], s_b[1024];
  __shared__ int tot[kPartLevels];
  const int T = blockDim.x;
  const int per = (L + T - 1) / T;
  const int l0 = min(L, (int)threadIdx.x * per), l1 = min(L, l0 + per);
  if (threadIdx.x < kPartLevels) tot[threadIdx.x] = 0;
  __syncthreads();
  int sa = 0, sbl[kPartLevels] = {0, 0, 0, 0, 0};
  for (int l = l0; l < l1; ++l) {
    const int64_t size = leaf_off[l + 1] - leaf_off[l];
    sa += ngroups[l];
#pragma unroll
    for (int c = 0; c < kPartLevels; ++c) {
      const int p = part_level(part_max, c);
      sbl[c] += ngroups[l] * (int)((size + p - 1) / p);
    }
  }
#pragma unroll
  for (int c = 0; c < kPartLevels; ++c)
    if (sbl[c]) atomicAdd(&tot[c], sbl[c]);
  __syncthreads();
  const int lev = pick_part_level(tot, target, part_max, min_part);
  const int part = part_level(part_max, lev);
  int sb = 0;
#pragma unroll
  for (int c = 0; c < kPartLevels; ++c)
    if (c == lev) sb = sbl[c];
  if (threadIdx.x == 0 && part_out) *part_out = part;
  s_a[threadIdx.x] = sa;
  s_b[threadIdx.x] = sb;
  __syncthreads();
  for (int off = 1; off < T; off <<= 1) {
    const int va = threadIdx.x >= off ? s_a[threadIdx.x - off] : 0;
    const int vb = threadIdx.x >= off ? s_b[threadIdx.x - off] : 0;
    __syncthreads();
    s_a[threadIdx.x] += va;
    s_b[threadIdx.x] += vb;
    __syncthreads();
  }
  int ra = s_a[threadIdx.x] - sa, rb = s_b[threadIdx.x] - sb;
  for (int l = l0; l < l1; ++l) {
    const int64_t size = leaf_off[l + 1] - leaf_off[l];
    gfirst[l] = ra;
    item_off[l] = rb;
    ra += ngroups[l];
    rb += ngroups[l] * (int)((size + part - 1) / part);
  }
  if (threadIdx.x == T - 1) {
    gfirst[L] = s_a[T - 1];
    item_off[L] = s_b[T - 1];
    *n_items = s_b[T - 1];
  }
}

// group starts (gbound[gfirst[l] + g], with gbound[gfirst[L]] = all pairs)
// and the item -> leaf table
__global__ void vgroup_fill_kernel(int L, const int64_t* __restrict__ leaf_off, int part,
                                   const int32_t* __restrict__ grp_off,
                                   const Pair* __restrict__ grouped,
                                   const int32_t* __restrict__ slot_k, int kstride, int budget,
                                   const int32_t* __restrict__ gfirst,
                                   const int32_t* __restrict__ item_off,
                                   int32_t* __restrict__ gbound, int32_t* __restrict__ item_leaf) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l == 0) gbound[gfirst[L]] = grp_off[L];
  if (l >= L) return;
  int n = 0, sum = 0, g = gfirst[l];
  for (int p = grp_off[l]; p < grp_off[l + 1]; ++p) {
    const int k = pair_k(grouped[p], slot_k, kstride);
    if (n == 0 || n == 64 || sum + k > budget) {
      gbound[g++] = p;
      n = 0;
      sum = 0;
    }
    ++n;
    sum += k;
  }
  for (int i = item_off[l]; i < item_off[l + 1]; ++i) item_leaf[i] = l;
}

__global__ void scatter_kernel(const Pair* __restrict__ pairs, const int32_t* __restrict__ npairs,
                               const int32_t* __restrict__ grp_off, int32_t* __restrict__ fill,
                               Pair* __restrict__ grouped) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= *npairs) return;
  const Pair pr = pairs[p];
  grouped[grp_off[pr.leaf] + atomicAdd(&fill[pr.leaf], 1)] = pr;
}

// ---------------------------------------------------------------- merge
__device__ void bitonic_sort_u64(u64* buf, int n2) {
  for (int size = 2; size <= n2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < (n2 >> 1); i += blockDim.x) {
        const int pos = 2 * i - (i & (stride - 1));
        const int partner = pos + stride;
        const bool asc = (pos & size) == 0;
        const u64 x = buf[pos], y = buf[partner];
        if ((x > y) == asc) {
          buf[pos] = y;
          buf[partner] = x;
        }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kMergeThreads) merge_kernel(
    int nslots, int kstride, const int32_t* __restrict__ slot_k, u64* __restrict__ topk,
    int32_t* __restrict__ topk_cnt, u64* __restrict__ thr, const u64* __restrict__ cand,
    int32_t* __restrict__ cand_cnt, int cap) {
  __shared__ u64 buf[kMergeCap];
  for (int slot = blockIdx.x; slot < nslots; slot += gridDim.x) {
    int cc = cand_cnt[slot];
    if (cc == 0) continue;
    if (cc > cap) cc = cap;
    const int kq = slot_k ? slot_k[slot] : kstride;
    int tk = topk_cnt[slot];
    u64* top = topk + (size_t)slot * kstride;
    int done = 0;
    while (done < cc) {
      const int chunk = min(cc - done, kMergeCap - kq);
      const int n = tk + chunk;
      int n2 = 2;
      while (n2 < n) n2 <<= 1;
      for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        u64 v = kNoKey;
        if (i < tk) v = top[i];
        else if (i < n) v = cand[(size_t)slot * cap + done + (i - tk)];
        buf[i] = v;
      }
      __syncthreads();
      bitonic_sort_u64(buf, n2);
      tk = min(kq, n);
      for (int i = threadIdx.x; i < tk; i += blockDim.x) top[i] = buf[i];
      __syncthreads();
      done += chunk;
    }
    if (threadIdx.x == 0) {
      topk_cnt[slot] = tk;
      thr[slot] = (tk == kq) ? top[kq - 1] : kNoKey;
      cand_cnt[slot] = 0;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- select
// One block per query: the next W leaves of the wave, i.e. the W smallest
// (LB^2, leaf) keys beyond the query's cursor among leaves that are neither
// searched, nor pruned by the bound test of Alg. 2, nor by its filter
// test, against the best-so-far of the wave's start.
constexpr int kSelThreads = 128;

// Walk of the precomputed visiting order from the query's cursor: the next W
// positions that are neither searched nor filter-pruned, stopping at the first
// bound-pruned leaf (the order ascends in LB^2, so every later leaf is pruned
// too).  One block of 128 threads per query examines 128 positions per step
// with a block-wide prefix count.
__global__ void __launch_bounds__(kSelThreads) select_walk_kernel(SelectArgs a,
                                                                 const int32_t* __restrict__ ord,
                                                                 int32_t* __restrict__ cursor) {
  const int q = blockIdx.x;
  if (a.done[q]) return;
  __shared__ int s_warp[kSelThreads / 32];
  __shared__ int s_stop, s_newcur;
  const int L = a.L;
  const u64 thr = a.thr[q];
  const float bsf2 = (thr == kNoKey) ? __int_as_float(0x7f800000) : key_d2(thr);
  const double bsf2d = (double)bsf2;
  const double bsf = (double)__fsqrt_rn(bsf2);
  const bool filt = a.P != nullptr && a.jpos != nullptr && a.jpos[q] >= 0;
  const int jp = filt ? a.jpos[q] : 0;
  const double* lb = a.lb2 + (size_t)q * L;
  const int32_t* od = ord + (size_t)q * L;
  unsigned char* sc = a.scanned + (size_t)q * L;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int pos0 = cursor[q];
  int picked = 0;
  bool finished = false;  // reached the end or a bound-pruned leaf
  while (pos0 < L && picked < a.W) {
    const int p = pos0 + (int)threadIdx.x;
    int leaf = -1, elig = 0, stop = 0, fpruned = 0;
    if (p < L) {
      leaf = od[p];
      if (__dmul_rn(lb[leaf], kDeflate) > bsf2d) {
        stop = 1;
      } else if (!sc[leaf]) {
        elig = 1;
        if (filt) {
          const int f = a.leaf_filter[leaf];
          if (f >= 0) {
            const double df =
                __dsub_rn((double)a.P[(size_t)q * a.F + f], a.alpha[(size_t)f * a.nc + jp]);
            if (df > bsf) {
              elig = 0;
              fpruned = 1;
            }
          }
        }
      }
    }
    if (threadIdx.x == 0) s_stop = INT_MAX;
    __syncthreads();
    if (stop) atomicMin(&s_stop, p);
    __syncthreads();
    const int first_stop = s_stop;
    if (p >= first_stop) elig = 0;
    // block exclusive prefix count of eligible positions
    const unsigned bal = __ballot_sync(0xffffffffu, elig);
    const int in_warp = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) s_warp[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < kSelThreads / 32; ++w) {
      if (w < warp) before += s_warp[w];
      total += s_warp[w];
    }
    const int rank = picked + before + in_warp;
    if (threadIdx.x == 0) s_newcur = -1;
    __syncthreads();
    if (elig && rank < a.W) {
      sc[leaf] = 1;
      const int idx = atomicAdd(a.npairs, 1);
      a.pairs[idx] = Pair{q, q, leaf, 0};
      atomicAdd(&a.stat[0], 1ull);
      atomicAdd(&a.stat[1], (u64)(a.leaf_off[leaf + 1] - a.leaf_off[leaf]));
      if (rank == a.W - 1) s_newcur = p + 1;
    }
    __syncthreads();
    // filter-pruned positions the cursor passes for good (Alg. 2's filter test); a
    // position at or after the next wave's start is examined again then
    const int cut = picked + total >= a.W ? s_newcur : first_stop;
    {
      const unsigned fb = __ballot_sync(0xffffffffu, fpruned && p < cut);
      if (lane == 0 && fb && a.stat) atomicAdd(&a.stat[4], (u64)__popc(fb));
    }
    if (picked + total >= a.W) {
      pos0 = s_newcur;
      picked = a.W;
      break;
    }
    picked += total;
    if (first_stop != INT_MAX || pos0 + kSelThreads >= L) {
      finished = true;
      pos0 = L;
      break;
    }
    pos0 += kSelThreads;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    cursor[q] = (finished || pos0 >= L) ? L : pos0;
    if (picked < a.W) a.done[q] = 1;
  }
}

// A wave at least as wide as the index (W >= L) takes every leaf that the
// walk of the visiting order would reach: the order ascends in LB^2 and the
// walk stops at the first bound-pruned leaf, so its picks are exactly the
// leaves that are not searched, not bound-pruned and not filter-pruned - a
// set that needs no order.  One thread per (query, leaf); the caller marks
// the queries done afterwards (no second wave can pick anything).
__global__ void select_all_kernel(SelectArgs a) {
  const int q = blockIdx.y;
  const int leaf = blockIdx.x * blockDim.x + threadIdx.x;
  if (leaf >= a.L || a.done[q]) return;
  unsigned char* sc = a.scanned + (size_t)q * a.L;
  if (sc[leaf]) return;
  const u64 thr = a.thr[q];
  const float bsf2 = (thr == kNoKey) ? __int_as_float(0x7f800000) : key_d2(thr);
  if (__dmul_rn(a.lb2[(size_t)q * a.L + leaf], kDeflate) > (double)bsf2) return;
  if (a.P != nullptr && a.jpos != nullptr && a.jpos[q] >= 0) {
    const int f = a.leaf_filter[leaf];
    if (f >= 0) {
      const double bsf = (double)__fsqrt_rn(bsf2);
      const double df =
          __dsub_rn((double)a.P[(size_t)q * a.F + f], a.alpha[(size_t)f * a.nc + a.jpos[q]]);
      if (df > bsf) {
        atomicAdd(&a.stat[4], 1ull);  // filter-pruned (Alg. 2's filter test)
        return;
      }
    }
  }
  sc[leaf] = 1;
  const int idx = atomicAdd(a.npairs, 1);
  a.pairs[idx] = Pair{q, q, leaf, 0};
  atomicAdd(&a.stat[0], 1ull);
  atomicAdd(&a.stat[1], (u64)(a.leaf_off[leaf + 1] - a.leaf_off[leaf]));
}

// The wave select reads the filter prediction of a (query, leaf) pair only
// when the leaf is not searched and passes the bound test against the wave's
// best-so-far; the best-so-far never rises, so after the route leaves' round a
// pair failing the same test (or of a query without filters, or of a searched
// leaf) is never read.  One thread per (query, filter); each filter's list of
// queries comes out in any order (a prediction does not depend on its row).
__global__ void filter_need_kernel(int nq, int F, int L, const int32_t* __restrict__ filter_leaf,
                                   const double* __restrict__ lb2, const u64* __restrict__ thr,
                                   const unsigned char* __restrict__ scanned,
                                   const int32_t* __restrict__ jpos, int32_t* __restrict__ rows_of,
                                   int32_t* __restrict__ cnt) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nq * F) return;
  const int q = (int)(t / F), f = (int)(t % F);
  if (jpos[q] < 0) return;
  const int leaf = filter_leaf[f];
  if (scanned[(size_t)q * L + leaf]) return;
  const u64 th = thr[q];
  const float bsf2 = (th == kNoKey) ? __int_as_float(0x7f800000) : key_d2(th);
  if (__dmul_rn(lb2[(size_t)q * L + leaf], kDeflate) > (double)bsf2) return;
  rows_of[(size_t)f * nq + atomicAdd(&cnt[f], 1)] = q;
}

__global__ void done_all_kernel(int nq, int32_t* __restrict__ done) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nq) done[q] = 1;
}

__global__ void leafknn_pairs_kernel(int nq, int nl, const int32_t* __restrict__ leaves, int L,
                                     Pair* __restrict__ pairs, int32_t* __restrict__ npairs) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nq * nl) return;
  const int leaf = leaves[t];
  if (leaf < 0 || leaf >= L) return;
  pairs[atomicAdd(npairs, 1)] = Pair{t, t / nl, leaf, 0};
}

__global__ void fill_u64_kernel(u64* p, u64 v, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// sorted position per query (Sec. 4.4.2 with the STEP reading): the query's
// k picks the smallest calibrated class >= k; the position is the largest j
// whose calibrated quality qprime[class][j] still reaches rq, the quality
// that certifies the query's recall target (computed on the host from the
// binomial tail of the calibration misses); rq > 1 leaves no position (exact).
// Computed by a whole warp (every lane gets the result): the table is read 32
// entries at a time and the position is the entry before the first one below
// the target.
__device__ __forceinline__ int jpos_of(int kq, double r, int nk, const int32_t* __restrict__ kclasses,
                                       const double* __restrict__ qprime, int nc, int lane) {
  int c = -1;
  for (int i = 0; i < nk; ++i)
    if (kclasses[i] >= kq) {
      c = i;
      break;
    }
  int j = -1;
  if (r < 0.0) {
    // interpolated offsets (STEFFEN mode): r = -(column + 1) of the offset table
    j = (int)(-r) - 1;
  } else if (c >= 0 && r <= 1.0) {
    const double* qp = qprime + (size_t)c * nc;
    j = nc - 1;
    for (int base = 0; base < nc; base += 32) {
      const int i = base + lane;
      const unsigned below = __ballot_sync(0xffffffffu, i < nc && !(qp[i] >= r));
      if (below) {
        j = base + __ffs(below) - 2;
        break;
      }
    }
  }
  return j;
}

// A batch's per-query state before its first wave, one warp per query: the
// searched flags cleared and the route leaf marked, the route leaf's pair
// (wave 0 of Alg. 2), the wave cursor, list counts, thresholds and done flags,
// and (jpos non-null) the sorted offset position.
__global__ void batch_init_kernel(int nq, int L, const int32_t* __restrict__ route,
                                  unsigned char* __restrict__ scanned,
                                  const int64_t* __restrict__ leaf_off, Pair* __restrict__ pairs,
                                  int32_t* __restrict__ npairs, u64* __restrict__ stat,
                                  int32_t* __restrict__ cursor, int32_t* __restrict__ topk_cnt,
                                  u64* __restrict__ thr, int32_t* __restrict__ cand_cnt,
                                  int32_t* __restrict__ done, const int32_t* __restrict__ k,
                                  const double* __restrict__ rq, int nk,
                                  const int32_t* __restrict__ kclasses,
                                  const double* __restrict__ qprime, int nc,
                                  int32_t* __restrict__ jpos) {
  const int q = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (q == 0 && lane == 0) *npairs = nq;
  if (q >= nq) return;
  const int leaf = route[q];
  unsigned char* sc = scanned + (size_t)q * L;
  for (int l = lane; l < L; l += 32) sc[l] = l == leaf ? 1 : 0;
  if (jpos) {
    const int j = jpos_of(k[q], rq[q], nk, kclasses, qprime, nc, lane);
    if (lane == 0) jpos[q] = j;
  }
  if (lane == 0) {
    pairs[q] = Pair{q, q, leaf, 0};
    atomicAdd(&stat[0], 1ull);
    atomicAdd(&stat[1], (u64)(leaf_off[leaf + 1] - leaf_off[leaf]));
    cursor[q] = 0;
    topk_cnt[q] = 0;
    thr[q] = kNoKey;
    cand_cnt[q] = 0;
    done[q] = 0;
  }
}

// results of batch query q go to row rows[q] of ids / dists (row q without rows)
__global__ void write_results_kernel(int nq, int kmax, const int32_t* __restrict__ kq,
                                     const u64* __restrict__ topk, int kstride,
                                     const int32_t* __restrict__ topk_cnt,
                                     const int32_t* __restrict__ rows, int64_t* __restrict__ ids,
                                     float* __restrict__ dists) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nq * kmax) return;
  const int q = t / kmax, z = t % kmax;
  const size_t o = (size_t)(rows ? rows[q] : q) * kmax + z;
  const int lim = min(kq ? kq[q] : kmax, topk_cnt[q]);
  if (z < lim) {
    const u64 key = topk[(size_t)q * kstride + z];
    ids[o] = (int64_t)(uint32_t)(key & 0xffffffffull);
    dists[o] = __fsqrt_rn(key_d2(key));
  } else {
    ids[o] = -1;
    dists[o] = __int_as_float(0x7f800000);
  }
}

__global__ void leafknn_out_kernel(int nslots, int k, const u64* __restrict__ topk,
                                   const int32_t* __restrict__ topk_cnt, float* __restrict__ d2,
                                   int64_t* __restrict__ ids) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nslots * k) return;
  const int s = t / k, z = t % k;
  if (z < topk_cnt[s]) {
    const u64 key = topk[t];
    d2[t] = key_d2(key);
    ids[t] = (int64_t)(uint32_t)(key & 0xffffffffull);
  } else {
    d2[t] = __int_as_float(0x7f800000);
    ids[t] = -1;
  }
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

size_t scan_smem_bytes(int mp, int k) {
  const size_t rs = (size_t)mp + 4;
  return (kRows + kG) * rs * sizeof(float) + (size_t)kG * k * 8 + (size_t)kG * kRows * 8;
}

int scan_group_size() { return kG; }

void launch_scan(const ScanArgs& a, const int32_t* n_items_dev, const int32_t* slot_k, int grid,
                 cudaStream_t s) {
  const size_t smem = scan_smem_bytes(a.mp, a.k);
  LF_CUDA(cudaFuncSetAttribute(scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  scan_kernel<<<grid, kScanThreads, smem, s>>>(a, n_items_dev, slot_k);
  LF_CHECK_LAUNCH();
}

bool launch_group(const Pair* pairs, const int32_t* npairs_dev, int npairs_max, int L,
                  const int64_t* leaf_off, int part, int g, int32_t* cnt, int32_t* grp_off,
                  int32_t* item_off, Pair* grouped, int32_t* n_items_dev,
                  unsigned long long* stat, cudaStream_t s, int32_t* item_leaf,
                  bool pack_small, int target_items, int32_t* part_out, int min_part,
                  const RoundPrep* rp) {
  if (L <= kFuseLeaves) {
    // the one-block kernel also preps the round while that is at most 16
    // entries per thread
    const bool fuse = rp && rp->topk && (int64_t)rp->nslots * rp->kstride <= 16 * 1024;
    group_fused_kernel<<<1, 1024, 0, s>>>(pairs, npairs_dev, L, leaf_off, part, g, grp_off,
                                          item_off, n_items_dev, grouped, stat, item_leaf,
                                          pack_small, target_items, min_part, part_out,
                                          fuse ? *rp : RoundPrep());
    LF_CHECK_LAUNCH();
    return fuse;
  }
  LF_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * L, s));
  if (npairs_max > 0) {
    count_kernel<<<nblk(npairs_max, 256), 256, 0, s>>>(pairs, npairs_dev, cnt);
    LF_CHECK_LAUNCH();
  }
  offsets_kernel<<<1, 1024, 0, s>>>(L, leaf_off, part, g, cnt, grp_off, item_off, n_items_dev,
                                    stat, item_leaf, pack_small, target_items, min_part, part_out);
  LF_CHECK_LAUNCH();
  if (npairs_max > 0) {
    scatter_kernel<<<nblk(npairs_max, 256), 256, 0, s>>>(pairs, npairs_dev, grp_off, cnt, grouped);
    LF_CHECK_LAUNCH();
  }
  return false;
}

void launch_var_groups(int L, const int64_t* leaf_off, int part, const int32_t* grp_off,
                       const Pair* grouped, const int32_t* slot_k, int kstride, int budget,
                       int32_t* ngroups, int32_t* gfirst, int32_t* gbound, int32_t* item_off,
                       int32_t* item_leaf, int32_t* n_items_dev, cudaStream_t s,
                       int target_items, int32_t* part_out, int min_part) {
  if (L <= 0) return;
  vgroup_count_kernel<<<nblk(L, 256), 256, 0, s>>>(L, grp_off, grouped, slot_k, kstride, budget,
                                                   ngroups);
  LF_CHECK_LAUNCH();
  vgroup_offsets_kernel<<<1, 1024, 0, s>>>(L, leaf_off, part, ngroups, gfirst, item_off, n_items_dev,
                                           target_items, min_part, part_out);
  LF_CHECK_LAUNCH();
  vgroup_fill_kernel<<<nblk(L, 256), 256, 0, s>>>(L, leaf_off, part, grp_off, grouped, slot_k,
                                                  kstride, budget, gfirst, item_off, gbound,
                                                  item_leaf);
  LF_CHECK_LAUNCH();
}

void launch_merge(int nslots, int kstride, const int32_t* slot_k, unsigned long long* topk,
                  int32_t* topk_cnt, unsigned long long* thr, const unsigned long long* cand,
                  int32_t* cand_cnt, int cand_cap, cudaStream_t s) {
  if (nslots <= 0) return;
  const int grid = nslots < 4096 ? nslots : 4096;
  merge_kernel<<<grid, kMergeThreads, 0, s>>>(nslots, kstride, slot_k, topk, topk_cnt, thr, cand,
                                              cand_cnt, cand_cap);
  LF_CHECK_LAUNCH();
}


void launch_select_all(const SelectArgs& a, cudaStream_t s) {
  if (a.nq <= 0 || a.L <= 0) return;
  select_all_kernel<<<dim3(nblk(a.L, 256), a.nq), 256, 0, s>>>(a);
  LF_CHECK_LAUNCH();
  done_all_kernel<<<nblk(a.nq, 256), 256, 0, s>>>(a.nq, a.done);
  LF_CHECK_LAUNCH();
}

void launch_filter_need(int nq, int F, int L, const int32_t* filter_leaf, const double* lb2,
                        const unsigned long long* thr, const unsigned char* scanned,
                        const int32_t* jpos, int32_t* rows_of, int32_t* cnt, cudaStream_t s) {
  if (nq <= 0 || F <= 0) return;
  LF_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)F, s));
  const int64_t tot = (int64_t)nq * F;
  filter_need_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(nq, F, L, filter_leaf, lb2, thr,
                                                                   scanned, jpos, rows_of, cnt);
  LF_CHECK_LAUNCH();
}

void launch_select_walk(const SelectArgs& a, const int32_t* ord, int32_t* cursor, cudaStream_t s) {
  if (a.nq <= 0) return;
  select_walk_kernel<<<a.nq, kSelThreads, 0, s>>>(a, ord, cursor);
  LF_CHECK_LAUNCH();
}

void launch_leafknn_pairs(int nq, int nl, const int32_t* leaves, int L, Pair* pairs,
                          int32_t* npairs, cudaStream_t s) {
  LF_CUDA(cudaMemsetAsync(npairs, 0, sizeof(int32_t), s));
  if (nq * nl == 0) return;
  leafknn_pairs_kernel<<<nblk((int64_t)nq * nl, 256), 256, 0, s>>>(nq, nl, leaves, L, pairs, npairs);
  LF_CHECK_LAUNCH();
}

void launch_fill_u64(unsigned long long* p, unsigned long long v, size_t n, cudaStream_t s) {
  if (!n) return;
  fill_u64_kernel<<<nblk((int64_t)n, 256), 256, 0, s>>>(p, v, n);
  LF_CHECK_LAUNCH();
}

void launch_batch_init(int nq, int L, const int32_t* route, unsigned char* scanned,
                       const int64_t* leaf_off, Pair* pairs, int32_t* npairs,
                       unsigned long long* stat, int32_t* cursor, int32_t* topk_cnt,
                       unsigned long long* thr, int32_t* cand_cnt, int32_t* done,
                       const int32_t* k, const double* target, int nk, const int32_t* kclasses,
                       const double* qprime, int nc, int32_t* jpos, cudaStream_t s) {
  batch_init_kernel<<<nblk((int64_t)(nq > 0 ? nq : 1) * 32, 256), 256, 0, s>>>(
      nq, L, route, scanned, leaf_off, pairs, npairs, stat, cursor, topk_cnt, thr, cand_cnt, done,
      k, target, nk, kclasses, qprime, nc, jpos);
  LF_CHECK_LAUNCH();
}

void launch_write_results(int nq, int kmax, const int32_t* kq, const unsigned long long* topk,
                          int kstride, const int32_t* topk_cnt, int64_t* ids, float* dists,
                          cudaStream_t s, const int32_t* rows) {
  if (nq * kmax == 0) return;
  write_results_kernel<<<nblk((int64_t)nq * kmax, 256), 256, 0, s>>>(nq, kmax, kq, topk, kstride,
                                                                     topk_cnt, rows, ids, dists);
  LF_CHECK_LAUNCH();
}

void launch_leafknn_out(int nslots, int k, const unsigned long long* topk, const int32_t* topk_cnt,
                        float* d2, int64_t* ids, cudaStream_t s) {
  if (nslots * k == 0) return;
  leafknn_out_kernel<<<nblk((int64_t)nslots * k, 256), 256, 0, s>>>(nslots, k, topk, topk_cnt, d2,
                                                                    ids);
  LF_CHECK_LAUNCH();
}

}  // namespace leafi
