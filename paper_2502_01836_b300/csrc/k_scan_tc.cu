// Tensor-core leaf scan (SearchNode of Alg. 2 on tcgen05).
//
// A work item is (leaf, part of the leaf, group of up to kTcG queries).  The
// part's series stream through shared memory in chunks of 128 rows of an
// fp16 copy of the data: one 2-D TMA per 64-column block (128-byte rows,
// 128-byte swizzle) lands each chunk directly in the K-major layout the MMA
// reads (two stages).  A loader warp gathers the item's query rows (fp16,
// prepared once per batch) into one of two query tiles while the previous item
// is still being scanned.  One thread issues tcgen05.mma (M = 128 series,
// N = the query group rounded to 16, K = the padded length) into one of four
// TMEM accumulators; the epilogue warps read them back with tcgen05.ld (one
// series row per thread).  The dot products give approximate squared distances
//     a = |q|^2 + |x|^2 - 2 <q~, x~>
// whose error against the canonical float32 distance is bounded per pair by
//     band = 2 (c |q| |x| + 2^-24 sqrt(m) (|q| + |x|)) + 1e-4 (|q|^2 + |x|^2),
// c = 2^-10 + 2^-22 + K 2^-23 (fp16 rounding of both operands, products,
// float32 accumulation of K terms with truncation, norm and canonical-sum
// rounding).  A series is re-checked with the canonical float32 distance
// (identical to the oracle's) whenever a - band <= T, where T is the query's
// admission bound: its k-th best exact distance so far, and for k = 1 also
// the smallest a + band seen in the part (an upper bound of the part's
// minimum).  No series whose canonical distance could enter the top-k is
// skipped, so results are bit-exact while almost all arithmetic runs on the
// tensor cores.
//
// Roles (352 threads): warps 0-7 epilogue, warp 8 lane 0 TMA producer, warp 9
// lane 0 MMA issuer, warp 10 query-tile loader.  For k = 1 the epilogue warps
// split into two halves that take alternate accumulators (warps 0-3 even
// chunks, 4-7 odd chunks), so all eight warps work even for small query
// groups; the re-checks are deferred to the end of the item.  For k > 1 all
// eight warps read every chunk; each TMEM lane quarter keeps its own top-k
// list per query (the quarter's two warps split the columns), re-checks run
// at once, and the quarter lists merge at the end of the item.
//
// The operands may instead be float8 e4m3 with a power-of-two scale per
// series and per query (x ~ s_x x^, q ~ s_q q^, kind::f8f6f4 MMAs of K = 32):
// the dot product is s_q s_x <q^, x^> and the band widens to
// c8 = 2^-3 + 2^-7 + 2^-8 (e4m3 rounding of both operands, |e| <= 2^-4 |v| in
// the normal range) plus the subnormal and accumulation terms (see
// tc_query_prep8_kernel); everything else, re-check included, is the same.
//
// Work items merge their results straight into each query's top-k list (an
// atomic minimum for k = 1; for k > 1 a warp-wide merge under the slot's
// lock), and every item admits against the list's current k-th key, read
// when it starts and again every other chunk.  Every (query, series) pair
// belongs to exactly one item, so a series of the final top-k has a smaller
// key than the k-th key of any list that does not contain it and is never
// dropped; the final lists do not depend on the order of items.
#include <cuda_fp8.h>

#include <algorithm>
#include <cfloat>

#include "device_util.cuh"

namespace leafi {
namespace {

using dev::u64;

constexpr int kTcRows = 128;      // MMA M: series per chunk
constexpr int kTcG = 64;          // queries per work item (MMA N <= 64)
constexpr int kEpi = 256;         // epilogue threads: warps 0-7, two per TMEM lane quarter
constexpr int kEpiWarps = kEpi / 32;
constexpr int kLoadWarp = kEpiWarps;      // lane 0 issues the TMA loads
constexpr int kMmaWarp = kEpiWarps + 1;   // lane 0 issues the MMAs
constexpr int kQueryWarp = kEpiWarps + 2; // gathers the query tiles
constexpr int kTcThreads = kEpi + 96;
constexpr int kAcc = 4;                   // TMEM accumulators of kTcG columns
constexpr int kTmemCols = kAcc * kTcG;
constexpr long long kWaitLimit = 1ll << 26;
constexpr int kCandCap = 2048;    // deferred re-check buffer (k = 1 rounds)
constexpr int kRing = 4;          // work items handed from the TMA thread to the other roles

struct TcShared {
  u64 full[2];      // TMA of stage s landed (1 arrival + bytes)
  u64 empty[2];     // MMAs reading stage s finished (tcgen05.commit)
  u64 tfull[kAcc];  // accumulator t written (tcgen05.commit)
  u64 tempty[kAcc]; // accumulator t read back by the epilogue threads
  u64 bready[2];    // query tile b gathered (32 arrivals of the loader warp)
  u64 bempty[2];    // MMAs reading query tile b finished (tcgen05.commit)
  u64 iready[kRing];  // ring slot holds the next work item (TMA thread)
  u64 ifree[kRing];   // ring slot read by the loader, the MMA thread and the epilogue
  int ring[kRing];    // work item index, -1 = no more work
  int eitem;          // epilogue's current item (broadcast through shared memory)
  uint32_t tmem_base;
  int abort;
  int stop;            // epilogue warps' uniform snapshot of `abort`
  u64 thr[kTcG];       // slot's k-th best key at the start of the round
  float thrd[kTcG];    // its squared distance (inf if fewer than k)
  float H[kTcG];       // k = 1: running admission bound (thrd, smallest a + band so far)
  float4 qb[kTcG];     // per query: U_lo, U_hi, alpha, |q|^2 (see the epilogue)
  float qm[kTcG];      // |q|
  float qs[kTcG];      // e4m3 operands: the query's scale s_q (1 for fp16)
  int slot[kTcG], kq[kTcG], cnt[kTcG], qrow[kTcG], wide[kTcG];
  int cnt4[4][kTcG];   // k > 1: entries of each TMEM lane quarter's list per query
  int loff[kTcG];      // k > 1: offset of each query's list in a quarter's lists (sum of earlier k)
  float Tq[kTcG];      // k > 1: admission bound (thrd, any full quarter list's k-th, refreshed threshold)
  int rs[kTcG], re[kTcG];  // packed item: the chunk rows of each pair's own leaf
  int ncb;             // buffered candidates of the current item
  unsigned long long rechecks;
};

// optional per-phase cycle counters (TcScanArgs::prof, 24 entries; 16-19 are
// the launch timeline totals in ns, 20-23 the current launch's, see
// tc_timeline_kernel):
// epilogue warp 0 lane 0: 0 item set-up, 1 wait accumulator, 2 epilogue, 3 flush+emit;
// MMA thread: 5 wait query tile, 6 wait TMA, 7 wait accumulator free, 14 MMA issue, 8 commits;
// load thread: 4 wait stage free, 11 TMA issue; 9 items, 10 chunks (of warp 0);
// query loader lane 0: 12 wait tile free, 13 gather; 15 epilogue warp 0 from kernel entry to exit
#define PROF_T0() long long _pt = clock64()
#define PROF_ADD(i)                                              \
  do {                                                           \
    const long long _nw = clock64();                             \
    if (prof_on) pr[i] += (unsigned long long)(_nw - _pt);       \
    _pt = _nw;                                                   \
  } while (0)

struct Item {
  int64_t p0, p1;
  int nqg, N, nchunks;
  bool packed;       // several small leaves in one chunk (pairs meet their own leaf's rows)
  const Pair* pr;
};

constexpr int kPackWin = 8;  // leaves per packed window (the grouping pass's windows)

template <bool kVarGroups>
__device__ __forceinline__ Item decode_item(const TcScanArgs& a, int item, int part_rows) {
  const int lf = a.item_leaf[item];
  Item it;
  if (lf < 0) {
    // a packed window of consecutive leaves [w0, w1): one chunk, one group
    const int w0 = -1 - lf, w1 = min(w0 + kPackWin, a.L);
    it.p0 = a.leaf_off[w0];
    it.p1 = a.leaf_off[w1];
    it.nqg = a.grp_off[w1] - a.grp_off[w0];
    it.N = ((it.nqg + 15) / 16) * 16;
    it.pr = a.pairs + a.grp_off[w0];
    it.nchunks = 1;
    it.packed = true;
    return it;
  }
  const int leaf = lf;
  const int local = item - a.item_off[leaf];
  int part;
  if (kVarGroups) {
    // groups bounded by the sum of their queries' k (launch_var_groups)
    const int gf = a.gfirst[leaf], ng = a.gfirst[leaf + 1] - gf;
    part = local / ng;
    const int grp = gf + local % ng;
    it.nqg = a.gbound[grp + 1] - a.gbound[grp];
    it.pr = a.pairs + a.gbound[grp];
  } else {
    const int cnt = a.grp_off[leaf + 1] - a.grp_off[leaf];
    const int G = a.G;
    const int ngroups = (cnt + G - 1) / G;
    part = local / ngroups;
    const int grp = local % ngroups;
    it.nqg = min(G, cnt - grp * G);
    it.pr = a.pairs + a.grp_off[leaf] + grp * G;
  }
  it.p0 = a.leaf_off[leaf] + (int64_t)part * part_rows;
  it.p1 = min(it.p0 + (int64_t)part_rows, a.leaf_off[leaf + 1]);
  it.N = ((it.nqg + 15) / 16) * 16;
  it.nchunks = (int)((it.p1 - it.p0 + kTcRows - 1) / kTcRows);
  it.packed = false;
  return it;
}

// One chunk's MMAs (KS steps of K = 16), fully unrolled: the descriptors'
// upper words are fixed, the lower words advance by constants (start address
// in 16-byte units: +32 bytes per step inside a 128-byte swizzled row of A and
// +16 KB per 64-column block; +256 bytes per step of the no-swizzle B), so the
// issuing thread spends a few instructions per MMA.
// A K step is 32 bytes of both operands for either kind: 16 fp16 or 32 e4m3
// values (the instruction descriptor's operand formats are 0 in both cases:
// F16 for kind::f16, E4M3 for kind::f8f6f4).
template <int KS, bool kFp8>
__device__ __forceinline__ void issue_chunk(uint32_t dt, uint32_t a_lo, uint32_t a_hi,
                                            uint32_t b_lo, uint32_t b_hi, uint32_t idesc) {
#pragma unroll
  for (int kk = 0; kk < KS; ++kk) {
    const uint32_t ao = a_lo + (uint32_t)((kk >> 2) * 1024 + (kk & 3) * 2);
    const uint32_t bo = b_lo + (uint32_t)(kk * 16);
    const uint32_t acc = kk > 0 ? 1u : 0u;
    if (kFp8)
      asm volatile(
          "{\n.reg .b64 ad, bd;\n.reg .pred p;\nmov.b64 ad, {%1, %2};\nmov.b64 bd, {%3, %4};\n"
          "setp.ne.b32 p, %6, 0;\ntcgen05.mma.cta_group::1.kind::f8f6f4 [%0], ad, bd, %5, p;\n}\n" ::"r"(dt),
          "r"(ao), "r"(a_hi), "r"(bo), "r"(b_hi), "r"(idesc), "r"(acc)
          : "memory");
    else
      asm volatile(
          "{\n.reg .b64 ad, bd;\n.reg .pred p;\nmov.b64 ad, {%1, %2};\nmov.b64 bd, {%3, %4};\n"
          "setp.ne.b32 p, %6, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], ad, bd, %5, p;\n}\n" ::"r"(dt),
          "r"(ao), "r"(a_hi), "r"(bo), "r"(b_hi), "r"(idesc), "r"(acc)
          : "memory");
  }
}

__device__ __forceinline__ void atomic_min_float_nonneg(float* p, float v) {
  // non-negative floats order like their bit patterns
  atomicMin(reinterpret_cast<unsigned int*>(p), __float_as_uint(v));
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(u64* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(dev::smem_addr(mbar)) : "memory");
}

// bounded wait that also gives up once another role has aborted
__device__ __forceinline__ bool wait_phase(u64* mbar, uint32_t parity, volatile int* abort) {
  if (*abort) return false;
  for (int round = 0; round < 64; ++round) {
    if (dev::mbar_wait(mbar, parity, kWaitLimit >> 6)) return true;
    if (*abort) return false;
  }
  return false;
}

// Canonical squared distance (the same operations in the same order as
// dev::canonical_d2) computed by a whole warp: lane l loads float4 words l and
// l + 32 of both rows, the differences are broadcast in order by shuffles.
// Rows of up to 64 float4 words (m <= 256, the tensor-core scan's limit).
__device__ __forceinline__ float warp_canonical_d2(const float4* __restrict__ q,
                                                   const float4* __restrict__ x, int m4, int lane) {
  float4 t[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int c = lane + 32 * h;
    t[h] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (c < m4) {
      const float4 a = q[c], b = x[c];
      t[h] = make_float4(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z),
                         __fsub_rn(a.w, b.w));
    }
  }
  float acc = 0.0f;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int cnt = min(32, m4 - 32 * h);
    for (int u = 0; u < cnt; ++u) {
      const float tx = __shfl_sync(0xffffffffu, t[h].x, u);
      const float ty = __shfl_sync(0xffffffffu, t[h].y, u);
      const float tz = __shfl_sync(0xffffffffu, t[h].z, u);
      const float tw = __shfl_sync(0xffffffffu, t[h].w, u);
      acc = __fmaf_rn(tx, tx, acc);
      acc = __fmaf_rn(ty, ty, acc);
      acc = __fmaf_rn(tz, tz, acc);
      acc = __fmaf_rn(tw, tw, acc);
    }
  }
  return acc;
}

constexpr int kIlp = 4;
constexpr int kCoopRechecks = 2;  // k > 1: columns with at most this many candidates re-check warp-wide

// Canonical squared distance by one thread (the operations and order of
// dev::canonical_d2) with the row loads issued eight float4 words at a time,
// so a re-check waits for a few memory round trips instead of one per word.
__device__ __forceinline__ float canonical_d2_ilp(const float4* __restrict__ q,
                                                  const float4* __restrict__ x, int m4) {
  float acc = 0.0f;
  for (int c0 = 0; c0 < m4; c0 += kIlp) {
    float4 xa[kIlp], qa[kIlp];
#pragma unroll
    for (int u = 0; u < kIlp; ++u)
      if (c0 + u < m4) {
        xa[u] = x[c0 + u];
        qa[u] = q[c0 + u];
      }
#pragma unroll
    for (int u = 0; u < kIlp; ++u)
      if (c0 + u < m4) {
        float t = __fsub_rn(qa[u].x, xa[u].x);
        acc = __fmaf_rn(t, t, acc);
        t = __fsub_rn(qa[u].y, xa[u].y);
        acc = __fmaf_rn(t, t, acc);
        t = __fsub_rn(qa[u].z, xa[u].z);
        acc = __fmaf_rn(t, t, acc);
        t = __fsub_rn(qa[u].w, xa[u].w);
        acc = __fmaf_rn(t, t, acc);
      }
  }
  return acc;
}

// Merge the keys held one per lane (kNoKey: none) that lie below `bound`
// into the ascending list L (cc entries, capacity kq): the warp sorts the
// keys (bitonic exchange over shuffles), every key and list entry finds its
// merged position by binary search in the other sequence, and the first kq
// are written back.  All lanes call it; keys are distinct from the list's.
__device__ __forceinline__ int warp_merge_keys(u64* L, int cc, int kq, u64 key, u64 bound,
                                               int lane) {
  u64 v = key < bound ? key : kNoKey;
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const u64 o = __shfl_xor_sync(0xffffffffu, v, stride);
      const bool keep_min = ((lane & stride) == 0) == ((lane & size) == 0);
      v = keep_min ? (o < v ? o : v) : (o < v ? v : o);
    }
  }
  const int nnew = __popc(__ballot_sync(0xffffffffu, v != kNoKey));
  if (nnew == 0) return cc;
  int rv = kq;
  if (lane < nnew) {
    int lo = 0, hi = cc;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (L[mid] < v) lo = mid + 1;
      else hi = mid;
    }
    rv = lane + lo;
  }
  u64 xv[LEAFI_MAX_K / 32];
  int rx[LEAFI_MAX_K / 32];
#pragma unroll
  for (int u = 0; u < LEAFI_MAX_K / 32; ++u) {
    xv[u] = kNoKey;
    rx[u] = kq;
    if (32 * u < cc) {  // warp-uniform
      const int p = lane + 32 * u;
      const u64 x = p < cc ? L[p] : kNoKey;
      int pos = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        const u64 pv = __shfl_sync(0xffffffffu, v, pos + step - 1);
        if (pv < x) pos += step;
      }
      const u64 last = __shfl_sync(0xffffffffu, v, 31);
      if (pos == 31 && last < x) pos = 32;
      xv[u] = x;
      if (p < cc) rx[u] = p + pos;
    }
  }
  __syncwarp();
#pragma unroll
  for (int u = 0; u < LEAFI_MAX_K / 32; ++u)
    if (rx[u] < kq) L[rx[u]] = xv[u];
  if (rv < kq) L[rv] = v;
  __syncwarp();
  return min(kq, cc + nnew);
}

// Attempts at a slot's lock before a work item reports a timeout come in
// TcScanArgs::lock_tries (kDefaultLockTries).  The lock is held for one
// warp-wide merge of at most 2k keys, so the default (tens of milliseconds
// with the back-off) is only reached if something is broken.

// Merge an item's ascending list B (cb entries) into the slot's top-k list gl
// (kq entries, ascending, kNoKey padded; keys of other items and of earlier
// rounds) under the slot's lock.  Readers take gl[kq - 1] without the lock:
// it is written once per merge, and both its old and its new value are the
// k-th key of k distinct scanned series (or kNoKey).  Returns false if the
// lock could not be taken (the list is then left unchanged).
__device__ __forceinline__ bool share_list(u64* gl, int32_t* lock, const u64* B, int cb, int kq,
                                           u64* scratch, int lane, int tries) {
  const u64 gk = __ldcg(&gl[kq - 1]);
  if (!(B[0] < gk)) return true;  // nothing of this item enters the list
  int got = 0;
  if (lane == 0) {
    unsigned ns = 32;
    for (int t = 0; t < tries && !got; ++t) {
      got = atomicCAS(lock, 0, 1) == 0 ? 1 : 0;
      if (!got) {
        __nanosleep(ns);
        ns = ns < 1024 ? 2 * ns : ns;
      }
    }
  }
  got = __shfl_sync(0xffffffffu, got, 0);
  if (!got) return false;
  __threadfence();
  for (int p = lane; p < kq; p += 32) scratch[p] = __ldcg(&gl[p]);
  __syncwarp();
  for (int p = lane; p < kq; p += 32) {
    const u64 x = scratch[p];
    int lo = 0, hi = cb;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (B[mid] < x) lo = mid + 1;
      else hi = mid;
    }
    if (p + lo < kq) gl[p + lo] = x;
  }
  for (int p = lane; p < cb; p += 32) {
    const u64 x = B[p];
    int lo = 0, hi = kq;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (scratch[mid] < x) lo = mid + 1;
      else hi = mid;
    }
    if (p + lo < kq) gl[p + lo] = x;
  }
  __threadfence();
  __syncwarp();
  if (lane == 0) atomicExch(lock, 0);
  return true;
}

// Work items are claimed dynamically: the TMA thread takes the next index
// from a global counter (one item ahead of the one it is loading) and hands
// it to the other roles through a ring of kRing slots, so every role of the
// CTA walks the same sequence and CTAs that finish early take more work.
__device__ __forceinline__ int ring_take(TcShared& S, int n, volatile int* abort) {
  const int s = n % kRing;
  const bool ok = wait_phase(&S.iready[s], (uint32_t)((n / kRing) & 1), abort);
  const int item = ok ? *reinterpret_cast<volatile int*>(&S.ring[s]) : -1;
  mbar_arrive(&S.ifree[s]);
  return item;
}

// Band constants of one query (fp16 operands over Kp columns, mp-float rows):
// alpha = 2 (c |q| + s), beta = 2 s |q| + 1e-4 |q|^2 with c = 2^-10 + 2^-22 +
// Kp 2^-23 and s = sqrt(mp) 2^-24, so that for any series x
//   lo = (|q|^2 - beta) + |x|^2 (1 - 1e-4) - alpha |x| - 2 <q~, x~>
//   hi = (|q|^2 + beta) + |x|^2 (1 + 1e-4) + alpha |x| - 2 <q~, x~>
// bracket the canonical squared distance.
__device__ __forceinline__ float band_c(int Kp) {
  return 9.7656250e-4f + 2.3841858e-7f + (float)Kp * 1.1920929e-7f;
}
__device__ __forceinline__ float band_s(int mp) { return sqrtf((float)mp) * 5.9604645e-8f; }

// fp16 query rows and band constants, one warp per query:
// Qk[2q] = (U_lo, U_hi, alpha, |q|^2), Qk[2q+1] = (|q|, wide, 0, 0), where
// U_lo = |q|^2 - beta (-inf for a query outside the safe fp16 range, whose
// series are then all re-checked) and U_hi = |q|^2 + beta
__global__ void tc_query_prep_kernel(const float* __restrict__ Q, int nq, int mp, int Kp,
                                     __half* __restrict__ Qh, float4* __restrict__ Qk) {
  const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= nq) return;
  float ss = 0.0f, mx = 0.0f;
  for (int piece = lane; piece < Kp / 8; piece += 32) {
    __align__(16) __half hv[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int i = piece * 8 + e;
      const float v = i < mp ? Q[(size_t)q * mp + i] : 0.0f;
      ss = fmaf(v, v, ss);
      mx = fmaxf(mx, fabsf(v));
      hv[e] = __float2half_rn(v);
    }
    *reinterpret_cast<uint4*>(Qh + (size_t)q * Kp + piece * 8) = *reinterpret_cast<const uint4*>(hv);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (lane == 0) {
    const float qm = sqrtf(ss);
    const float sm = band_s(mp);
    const float alpha = 2.0f * (band_c(Kp) * qm + sm);
    const float beta = 2.0f * sm * qm + 1e-4f * ss;
    const bool wide = mx >= 30000.0f;
    Qk[2 * (size_t)q] = make_float4(wide ? -__int_as_float(0x7f800000) : ss - beta, ss + beta, alpha, ss);
    Qk[2 * (size_t)q + 1] = make_float4(qm, wide ? 1.0f : 0.0f, 0.0f, 0.0f);
  }
}

// e4m3 query rows (Kp bytes, zero padded) with a power-of-two scale s_q
// (max |q_i| / s_q <= 448, the largest finite e4m3 value; s_q < max |q_i| / 224)
// and band constants, one warp per query: Qk[2q] = (U_lo, U_hi, alpha, |q|^2),
// Qk[2q+1] = (|q|, 0, s_q, 0).  Rounding to e4m3 moves a value v by at most
// 2^-4 |v| in the normal range and 2^-10 s in the subnormal one, so for the
// scaled dot product
//   |<q, x> - s_q s_x <q^, x^>| <= c1 |q||x| + c2 sqrt(m) (s_x |q| + s_q |x|)
//                                  + c3 m s_q s_x
// with c1 = 2 (1 + 2^-4) 2^-4 + 2^-8, c2 = (1 + 2^-4) 2^-10 + 2^-13 + 2^-14,
// c3 = 3 2^-20; with s < |v| / 224 every term is a multiple of |q||x|, and the
// float32 accumulation of K exact products adds K 2^-23 (1 + 2^-4)^2 |q||x|.
// The band then has the fp16 form with c8 in place of c.
__global__ void tc_query_prep8_kernel(const float* __restrict__ Q, int nq, int mp, int Kp,
                                      unsigned char* __restrict__ Q8, float4* __restrict__ Qk) {
  const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= nq) return;
  float ss = 0.0f, mx = 0.0f;
  for (int i = lane; i < mp; i += 32) {
    const float v = Q[(size_t)q * mp + i];
    ss = fmaf(v, v, ss);
    mx = fmaxf(mx, fabsf(v));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  int e = 0;
  if (mx > 0.0f) frexpf(mx / 448.0f, &e);
  const float sc = mx > 0.0f ? ldexpf(1.0f, e) : 1.0f;
  for (int piece = lane; piece < Kp / 16; piece += 32) {
    __align__(16) unsigned char b[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int i = piece * 16 + u;
      const float v = i < mp ? Q[(size_t)q * mp + i] : 0.0f;
      b[u] = (unsigned char)__nv_cvt_float_to_fp8(v / sc, __NV_SATFINITE, __NV_E4M3);
    }
    *reinterpret_cast<uint4*>(Q8 + (size_t)q * Kp + piece * 16) = *reinterpret_cast<const uint4*>(b);
  }
  if (lane == 0) {
    const float qm = sqrtf(ss);
    const float sm = band_s(mp);
    const float rm = sqrtf((float)mp);
    const float c8 = 0.13671875f + 2.0f * 0.0011596680f * rm / 224.0f +
                     2.8610229e-6f * (float)mp / 50176.0f + (float)Kp * 1.1920929e-7f * 1.1289063f +
                     9.5367432e-7f;
    const float alpha = 2.0f * (c8 * qm + sm);
    const float beta = 2.0f * sm * qm + 1e-4f * ss;
    Qk[2 * (size_t)q] = make_float4(ss - beta, ss + beta, alpha, ss);
    Qk[2 * (size_t)q + 1] = make_float4(qm, 0.0f, sc, 0.0f);
  }
}

// kSplit: k = 1 (one best key per query, fixed groups of 64); otherwise top-k
// lists per lane quarter and groups sized by k.  Two instantiations, so each
// path is compiled and scheduled on its own.
template <bool kSplit, bool kFp8>
__global__ void __launch_bounds__(kTcThreads, 1) tc_scan_kernel(
    const __grid_constant__ CUtensorMap tmap, TcScanArgs a, const int32_t* __restrict__ n_items_dev,
    const int32_t* __restrict__ slot_k) {
  const long long t_enter = clock64();
  if (a.prof && threadIdx.x == 0) {
    // launch timeline (ns): first and last block start
    unsigned long long g;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g));
    atomicMin(&a.prof[20], g);
    atomicMax(&a.prof[21], g);
  }
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ TcShared S;
  // 128-byte swizzled tiles need 1024-byte aligned bases
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int Kp = a.kp;                       // operand row length (fp16: multiple of 64,
                                             // e4m3: multiple of 128)
  const int RB = kFp8 ? Kp : 2 * Kp;         // operand bytes per row
  const int tileA = kTcRows * RB;            // bytes per A stage
  const int G = a.G;                         // queries per work item (64, or 16 for large k)
  const int tileB = G * RB;                  // bytes per query tile
  const int nbuf = a.nbuf;                   // query tiles (1 or 2)
  unsigned char* A0 = smem;
  unsigned char* A1 = smem + tileA;
  unsigned char* B0 = smem + 2 * tileA;      // G x Kp operands, no swizzle
  unsigned char* B1 = B0 + (nbuf - 1) * tileB;
  // k = 1: [G] best keys; k > 1: four quarters of a.qkeys keys, query j's list at S.loff[j]
  u64* lists = reinterpret_cast<u64*>(B0 + nbuf * tileB);
  int* cb_pos = reinterpret_cast<int*>(lists + G * a.k);
  int* cb_j = cb_pos + kCandCap;
  float* cb_lo = reinterpret_cast<float*>(cb_j + kCandCap);
  constexpr bool split = kSplit;             // k = 1: halves on alternate accumulators, deferred re-checks
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t sbo = 8u * RB;              // B: bytes between 8-row groups
  const int m4 = a.mp / 4;
  volatile int* abort = &S.abort;

  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      dev::mbar_init(&S.full[i], 1);
      dev::mbar_init(&S.empty[i], 1);
      dev::mbar_init(&S.bready[i], 32);
      dev::mbar_init(&S.bempty[i], 1);
    }
    for (int i = 0; i < kRing; ++i) {
      dev::mbar_init(&S.iready[i], 1);
      dev::mbar_init(&S.ifree[i], 3);
    }
    for (int i = 0; i < kAcc; ++i) {
      dev::mbar_init(&S.tfull[i], 1);
      dev::mbar_init(&S.tempty[i], split ? kEpi / 2 : kEpi);
    }
    S.abort = 0;
    S.stop = 0;
    S.ncb = 0;
    S.rechecks = 0;
  }
  if (warp == 0) dev::tmem_alloc(&S.tmem_base, kTmemCols);
  dev::tc_fence_before();
  __syncthreads();
  dev::tc_fence_after();
  const uint32_t tmem = S.tmem_base;
  const int n_items = *n_items_dev;
  const int part_rows = a.part_dev ? *a.part_dev : a.part;  // this round's work-item rows
  unsigned long long pr[16];
  for (int i = 0; i < 16; ++i) pr[i] = 0;
  const bool prof_on = a.prof != nullptr &&
                       (tid == 0 || tid == kLoadWarp * 32 || tid == kMmaWarp * 32 || tid == kQueryWarp * 32);

  if (warp == kLoadWarp) {
    // ------------------------------------------------ TMA producer + item scheduler
    if (lane == 0) {
      PROF_T0();
      long long g_ld = 0;
      long long ld_cnt[2] = {0, 0};  // loads issued per stage
      uint32_t empty_ph[2] = {0u, 0u};
      bool alive = true;
      auto publish = [&](int n) -> int {
        const int sl = n % kRing;
        if (n >= kRing && !wait_phase(&S.ifree[sl], (uint32_t)((n / kRing - 1) & 1), abort)) {
          atomicOr(a.err, 2);
          S.abort = 1;
          alive = false;
          return -1;
        }
        int item = atomicAdd(a.work, 1);
        if (item >= n_items) item = -1;
        S.ring[sl] = item;
        mbar_arrive(&S.iready[sl]);
        return item;
      };
      int cur = publish(0);
      for (int n = 0; cur >= 0 && alive && !*abort; ++n) {
        const int nxt = publish(n + 1);
        const Item I = decode_item<!kSplit>(a, cur, part_rows);
        for (int c = 0; c < I.nchunks; ++c) {
          const int st = (int)(g_ld & 1);
          if (g_ld >= 2) {
            PROF_ADD(11);
            const bool ok = wait_phase(&S.empty[st], empty_ph[st], abort);
            empty_ph[st] ^= 1u;
            PROF_ADD(4);
            if (!ok) {
              atomicOr(a.err, 2);
              S.abort = 1;
              break;
            }
          }
          unsigned char* dst = st ? A1 : A0;
          const int r0 = (int)(I.p0 + (int64_t)c * kTcRows);
          dev::mbar_expect_tx(&S.full[st], (uint32_t)tileA);
          // one 128-byte swizzled box (64 fp16 or 128 e4m3 columns) per block
          for (int kb = 0; kb < RB / 128; ++kb)
            dev::tma_load_2d(dst + kb * 16384, &tmap, kb * (kFp8 ? 128 : 64), r0, &S.full[st]);
          ++g_ld;
          ++ld_cnt[st];
        }
        cur = nxt;
      }
      PROF_ADD(11);
      // after a timeout the loads already issued may still be landing: wait
      // (bounded) until the last one of each stage has, so that no copy writes
      // shared memory after the block exits
      if (*abort)
        for (int st = 0; st < 2; ++st)
          if (ld_cnt[st] > 0)
            dev::mbar_wait(&S.full[st], (uint32_t)((ld_cnt[st] - 1) & 1), kWaitLimit);
    }
  } else if (warp == kQueryWarp) {
    // ------------------------------------------------ query-tile loader
    // (lane 0 takes every decision and broadcasts it, so the warp stays converged)
    PROF_T0();
    uint32_t bempty_ph[2] = {0u, 0u};
    int li = 0;
    const int pieces = RB / 16;                // 16-byte pieces per query row
    const unsigned char* qops = kFp8 ? a.Q8 : reinterpret_cast<const unsigned char*>(a.Qh);
    for (;; ++li) {
      int item = -1;
      if (lane == 0) item = ring_take(S, li, abort);
      item = __shfl_sync(0xffffffffu, item, 0);
      if (item < 0) break;
      const Item I = decode_item<!kSplit>(a, item, part_rows);
      const int b = li % nbuf;
      if (li >= nbuf) {
        bool ok = true;
        if (lane == 0) ok = wait_phase(&S.bempty[b], bempty_ph[b], abort);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        bempty_ph[b] ^= 1u;
        if (!ok) {
          if (lane == 0) {
            atomicOr(a.err, 2);
            S.abort = 1;
          }
          break;
        }
      }
      PROF_ADD(12);
      unsigned char* Bt = b ? B1 : B0;
      // every 16-byte piece of the tile is an asynchronous copy (rows beyond the
      // group are zero-filled), so all of them are in flight at once; the
      // group's query rows (at most 64) are read two per lane up front and
      // broadcast, rather than one dependent load per row
      const int r_lo = lane < I.nqg ? I.pr[lane].q : -1;
      const int r_hi = lane + 32 < I.nqg ? I.pr[lane + 32].q : -1;
      for (int qq = 0; qq < I.N; ++qq) {
        const int row = __shfl_sync(0xffffffffu, qq < 32 ? r_lo : r_hi, qq & 31);
        const unsigned char* src = qops + (size_t)(row >= 0 ? row : 0) * RB;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int piece = lane + 32 * h;
          if (piece < pieces)
            dev::cp_async16_zfill(Bt + (qq / 8) * sbo + piece * 128 + (qq % 8) * 16,
                                  src + piece * 16, row >= 0 ? 16 : 0);
        }
      }
      dev::cp_async_commit();
      dev::cp_async_wait_all();
      dev::fence_async_smem();
      __syncwarp();
      mbar_arrive(&S.bready[b]);
      PROF_ADD(13);
    }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------ MMA issue
    if (lane == 0) {
      PROF_T0();
      long long g_mm = 0;
      long long bc_cnt[2] = {0, 0};  // commits to each query tile's barrier
      int last_b = -1;
      int li = 0;
      uint32_t full_ph[2] = {0u, 0u}, bready_ph[2] = {0u, 0u}, tempty_ph[kAcc] = {0u, 0u, 0u, 0u};
      const uint64_t adesc[2] = {dev::smem_desc(dev::smem_addr(A0), 16, 1024, 2),
                                 dev::smem_desc(dev::smem_addr(A1), 16, 1024, 2)};
      const uint64_t bdesc[2] = {dev::smem_desc(dev::smem_addr(B0), 128, sbo),
                                 dev::smem_desc(dev::smem_addr(B1), 128, sbo)};
      for (;; ++li) {
        const int item = ring_take(S, li, abort);
        if (item < 0) break;
        const Item I = decode_item<!kSplit>(a, item, part_rows);
        const int b = li % nbuf;
        bool ok = wait_phase(&S.bready[b], bready_ph[b], abort);
        bready_ph[b] ^= 1u;
        PROF_ADD(5);
        const uint32_t idesc = dev::idesc_f16(kTcRows, I.N);
        for (int c = 0; ok && c < I.nchunks; ++c) {
          const int st = (int)(g_mm & 1), t = (int)(g_mm & (kAcc - 1));
          ok = wait_phase(&S.full[st], full_ph[st], abort);
          full_ph[st] ^= 1u;
          PROF_ADD(6);
          if (ok && g_mm >= kAcc) {
            ok = wait_phase(&S.tempty[t], tempty_ph[t], abort);
            tempty_ph[t] ^= 1u;
            PROF_ADD(7);
          }
          if (!ok) break;
          dev::tc_fence_after();
          // descriptor start addresses advance in 16-byte units: +32 bytes per
          // K step inside a 128-byte swizzle row, +16 KB per 64-column block (A);
          // +256 bytes per K step (B, two core matrices)
          const uint64_t ad = adesc[st], bd = bdesc[b];
          const uint32_t dt = tmem + (uint32_t)(t * kTcG);
          const uint32_t alo = (uint32_t)ad, ahi = (uint32_t)(ad >> 32);
          const uint32_t blo = (uint32_t)bd, bhi = (uint32_t)(bd >> 32);
          switch (RB) {
            case 128: issue_chunk<4, kFp8>(dt, alo, ahi, blo, bhi, idesc); break;
            case 256: issue_chunk<8, kFp8>(dt, alo, ahi, blo, bhi, idesc); break;
            case 384: issue_chunk<12, kFp8>(dt, alo, ahi, blo, bhi, idesc); break;
            default: issue_chunk<16, kFp8>(dt, alo, ahi, blo, bhi, idesc); break;
          }
          PROF_ADD(14);
          dev::mma_commit(&S.empty[st]);
          dev::mma_commit(&S.tfull[t]);
          ++g_mm;
          PROF_ADD(8);
        }
        // the query tile is free once this item's MMAs have completed
        dev::mma_commit(&S.bempty[b]);
        ++bc_cnt[b];
        last_b = b;
        if (!ok) {
          atomicOr(a.err, 2);
          S.abort = 1;
        }
      }
      // after a timeout, wait (bounded) for the last commit: every MMA issued
      // before it has then finished reading shared memory and writing TMEM,
      // which the block releases on exit
      if (*abort && last_b >= 0)
        dev::mbar_wait(&S.bempty[last_b], (uint32_t)((bc_cnt[last_b] - 1) & 1), kWaitLimit);
    }
  } else {
    // ------------------------------------------------ epilogue warps 0-7
    const float4* Q4 = reinterpret_cast<const float4*>(a.Q);
    const float4* X4 = reinterpret_cast<const float4*>(a.X);
    const float kInf = __int_as_float(0x7f800000);
    const int half = warp >> 2;
    const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
    const int r = quarter * 32 + lane;
    uint32_t tfull_ph[kAcc] = {0u, 0u, 0u, 0u};
    long long g = 0;
    PROF_T0();
    for (int n = 0;; ++n) {
      if (tid == 0) S.eitem = ring_take(S, n, abort);
      epi_sync();
      const int item = S.eitem;
      if (item < 0) break;
      const Item I = decode_item<!kSplit>(a, item, part_rows);
      const int nqg = I.nqg, N = I.N;
      if (prof_on) pr[9] += 1;
      // per-query state of the item (padding columns never admit a series)
      if (tid < N) {
        const int qq = tid;
        if (qq < nqg) {
          const int slot = I.pr[qq].slot, qrow = I.pr[qq].q;
          const float4 k0 = a.Qk[2 * (size_t)qrow], k1 = a.Qk[2 * (size_t)qrow + 1];
          // the slot's k-th best key so far: earlier rounds and the work items
          // of this round that have finished (kNoKey while fewer than k)
          const int kqs = slot_k ? slot_k[slot] : a.k;
          const u64 th = __ldcg(&a.topk[(size_t)slot * a.k + kqs - 1]);
          const float thd = (th == kNoKey) ? kInf : dev::key_d2(th);
          S.slot[qq] = slot;
          S.qrow[qq] = qrow;
          S.kq[qq] = kqs;
          S.thr[qq] = th;
          S.thrd[qq] = thd;
          // k = 1: the round's shared upper bound of the query's best distance
          S.H[qq] = (split && a.ub) ? fminf(thd, __ldcg(&a.ub[slot])) : thd;
          S.cnt[qq] = 0;
          S.cnt4[0][qq] = S.cnt4[1][qq] = S.cnt4[2][qq] = S.cnt4[3][qq] = 0;
          S.Tq[qq] = thd;
          S.wide[qq] = k1.y != 0.0f ? 1 : 0;
          S.qb[qq] = k0;
          S.qm[qq] = k1.x;
          S.qs[qq] = kFp8 ? k1.z : 1.0f;
          if (I.packed) {
            const int lf = I.pr[qq].leaf;
            S.rs[qq] = (int)(a.leaf_off[lf] - I.p0);
            S.re[qq] = (int)(a.leaf_off[lf + 1] - I.p0);
          }
          if (split) lists[qq * a.k] = th;
        } else {
          S.qb[qq] = make_float4(kInf, kInf, 0.0f, 0.0f);
          S.qs[qq] = 1.0f;
          S.H[qq] = 0.0f;  // lo = inf > 0: never a candidate
          S.Tq[qq] = 0.0f;
          S.rs[qq] = S.re[qq] = 0;
        }
      }
      epi_sync();
      if (!split && warp == 0) {
        // list offsets: exclusive prefix of the group's k (64 queries, two per lane)
        int k0 = lane < nqg ? S.kq[lane] : 0, k1 = lane + 32 < nqg ? S.kq[lane + 32] : 0;
        int s0 = k0, s1 = k1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int u0 = __shfl_up_sync(0xffffffffu, s0, o), u1 = __shfl_up_sync(0xffffffffu, s1, o);
          if (lane >= o) {
            s0 += u0;
            s1 += u1;
          }
        }
        const int tot0 = __shfl_sync(0xffffffffu, s0, 31);
        S.loff[lane] = s0 - k0;
        S.loff[lane + 32] = tot0 + s1 - k1;
      }
      if (!split) epi_sync();
      PROF_ADD(0);

      for (int c = 0; c < I.nchunks; ++c, ++g) {
        const int t = (int)(g & (kAcc - 1));
        if (split && (t & 1) != half) continue;
        if (prof_on) pr[10] += 1;
        const int64_t pos = I.p0 + (int64_t)c * kTcRows + r;
        const bool valid = pos < I.p1;
        const float xn = valid ? a.xn[pos] : 0.0f;
        // e4m3 operands: the dot product of the row with column j is
        // -2 s_x s_q acc (powers of two: the scaling is exact)
        const float m2sx = kFp8 ? (valid ? -2.0f * a.sx[pos] : 0.0f) : -2.0f;
        // k = 1: bounds other work items of the round have published since
        // the item started (thread r refreshes query column r)
        const float ubr = (split && a.ub && r < nqg) ? __ldcg(&a.ub[S.slot[r]]) : kInf;
        // on a timeout every later wait returns at once; the loop still reaches
        // all arrivals and barriers, and the error word reports the failure
        const bool ok = wait_phase(&S.tfull[t], tfull_ph[t], abort);
        tfull_ph[t] ^= 1u;
        if (!ok) {
          atomicOr(a.err, 2);
          S.abort = 1;
        }
        PROF_ADD(1);
        if (ubr < S.H[r]) atomic_min_float_nonneg(&S.H[r], ubr);
        const bool okw = __all_sync(0xffffffffu, ok);  // warp-uniform for tcgen05.ld
        dev::tc_fence_after();
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(t * kTcG);
        if (split) {
          // rows past the part end never admit a series
          const float xnorm = sqrtf(xn);
          const float vlo = valid ? xn * (1.0f - 1e-4f) : kInf;
          const float vhi = valid ? xn * (1.0f + 1e-4f) : kInf;
          for (int c0 = 0; okw && c0 < N; c0 += 16) {
            float d[16];
            dev::tmem_ld16(tl + (uint32_t)c0, d);
            float lov[16], hw[16];
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
              const float4 qb = S.qb[c0 + jj];
              const float cf = kFp8 ? m2sx * S.qs[c0 + jj] : -2.0f;
              lov[jj] = fmaf(cf, d[jj], fmaf(-qb.z, xnorm, qb.x + vlo));
              hw[jj] = fmaxf(fmaf(cf, d[jj], fmaf(qb.z, xnorm, qb.y + vhi)), 0.0f);
            }
            if (I.packed) {
              // a pair only meets the rows of its own leaf
#pragma unroll
              for (int jj = 0; jj < 16; ++jj)
                if (r < S.rs[c0 + jj] || r >= S.re[c0 + jj]) {
                  lov[jj] = kInf;
                  hw[jj] = kInf;
                }
            }
            const float4* H4 = reinterpret_cast<const float4*>(&S.H[c0]);
            float T[16];
#pragma unroll
            for (int v4 = 0; v4 < 4; ++v4) {
              // re-read every 16 columns: the tcgen05.ld above carries a memory clobber
              const float4 h = H4[v4];
              T[4 * v4 + 0] = h.x;
              T[4 * v4 + 1] = h.y;
              T[4 * v4 + 2] = h.z;
              T[4 * v4 + 3] = h.w;
            }
            unsigned cand = 0;
#pragma unroll
            for (int jj = 0; jj < 16; ++jj)
              if (valid && !(lov[jj] > T[jj])) cand |= 1u << jj;
            // an upper bound a + band below T needs a - band <= T first, so the
            // warp minimum of the upper bounds (one REDUX per column) is only
            // formed for the columns where some row is admitted
            const unsigned act = __reduce_or_sync(0xffffffffu, cand);
            if (act) {
              unsigned lower = 0;
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) {
                if (!(act & (1u << jj))) continue;
                const float hm = __uint_as_float(__reduce_min_sync(0xffffffffu, __float_as_uint(hw[jj])));
                if (hm < T[jj]) {
                  lower |= 1u << jj;
                  T[jj] = hm;
                  if (lov[jj] > hm) cand &= ~(1u << jj);
                }
              }
              // a tighter upper bound is rare once the part is under way; it
              // is published to the round's other work items as well
              if (lane == 0 && lower) {
#pragma unroll
                for (int jj = 0; jj < 16; ++jj)
                  if (lower & (1u << jj)) {
                    atomic_min_float_nonneg(&S.H[c0 + jj], T[jj]);
                    if (a.ub) atomic_min_float_nonneg(&a.ub[S.slot[c0 + jj]], T[jj]);
                  }
              }
            }
            if (__any_sync(0xffffffffu, cand != 0u)) {
              while (cand) {
                const int jj = __ffs(cand) - 1;
                cand &= cand - 1;
                const int j = c0 + jj;
                const int slotc = atomicAdd(&S.ncb, 1);
                float lo_j = 0.0f;
#pragma unroll
                for (int u = 0; u < 16; ++u)
                  if (u == jj) lo_j = lov[u];
                if (slotc < kCandCap) {
                  cb_pos[slotc] = (int)pos;
                  cb_j[slotc] = j;
                  cb_lo[slotc] = lo_j;
                  // the float32 row is re-read at the end of the item: start it now
                  const char* row = reinterpret_cast<const char*>(X4 + (size_t)pos * m4);
                  for (int o = 0; o < m4 * 16; o += 128)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(row + o));
                } else {
                  const float e = dev::canonical_d2(Q4 + (size_t)S.qrow[j] * m4, X4 + (size_t)pos * m4, m4);
                  atomicMin(&lists[j * a.k], dev::make_key(e, (uint32_t)a.ids[pos]));
                  atomicAdd(&S.rechecks, 1ull);
                }
              }
            }
          }
        } else {
          // general k: every TMEM lane quarter keeps its own top-k list per query
          // (warps w and w + 4 share the quarter and split the 16-column groups),
          // so no two warps ever write the same list.  The admission bound Tq
          // of a query is shared by the quarters and by the round's other work
          // items: it falls to any quarter's k-th best distance and to the k-th
          // key of the slot's list as other items merge into it (re-read every
          // other chunk).  Admission compares distances (a - band <= Tq, ties
          // admitted); insertion compares keys against the quarter's own k-th
          // or the list's k-th read at the item's start (the item merges its
          // own series only when it ends).  32 columns
          // are tested at once, re-checks run at once (one candidate per lane),
          // and the quarter lists merge at the item's end.
          const int qd = warp & 3;
          u64* ql = lists + (size_t)qd * a.qkeys;  // this quarter's lists
          const float xnorm = sqrtf(xn);
          const float vlo = xn * (1.0f - 1e-4f);
          const bool refresh = (c & 1) == 1;
          // warp w reads columns 32 (w / 4) .. + 31 of its lane quarter in one load
          const int c0 = (warp >> 2) * 32;
          if (okw && c0 < N) {
            // the slot thresholds of these 32 columns, consumed after the tests
            u64 gth = kNoKey;
            if (refresh && c0 + lane < nqg)
              gth = __ldcg(&a.topk[(size_t)S.slot[c0 + lane] * a.k + S.kq[c0 + lane] - 1]);
            float d[32];
            dev::tmem_ld32(tl + (uint32_t)c0, d);
            const float4* T4v = reinterpret_cast<const float4*>(&S.Tq[c0]);
            unsigned cand = 0;
#pragma unroll
            for (int v4 = 0; v4 < 8; ++v4) {
              const float4 tv = T4v[v4];
              const float tt[4] = {tv.x, tv.y, tv.z, tv.w};
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int jj = 4 * v4 + u;
                const float4 qb = S.qb[c0 + jj];
                const float cf = kFp8 ? m2sx * S.qs[c0 + jj] : -2.0f;
                const float lo = fmaf(cf, d[jj], fmaf(-qb.z, xnorm, qb.x + vlo));
                if (!(lo > tt[u])) cand |= 1u << jj;
              }
            }
            // columns at or past N belong to no query of this item
            if (N - c0 < 32) cand &= (1u << (N - c0)) - 1u;
            if (!valid) cand = 0u;
            if (I.packed) {
              // a pair only meets the rows of its own leaf
#pragma unroll
              for (int jj = 0; jj < 32; ++jj)
                if (r < S.rs[c0 + jj] || r >= S.re[c0 + jj]) cand &= ~(1u << jj);
            }
            unsigned any = __reduce_or_sync(0xffffffffu, cand);
            while (any) {
              const int jj = __ffs(any) - 1;
              any &= any - 1;
              const int j = c0 + jj;
              const bool cj = (cand >> jj) & 1u;
              unsigned mask = __ballot_sync(0xffffffffu, cj);
              const int kq = S.kq[j];
              int cc = S.cnt4[qd][j];
              u64 key = kNoKey;
              const float4* qrow4 = Q4 + (size_t)S.qrow[j] * m4;
              if (__popc(mask) <= kCoopRechecks) {
                // few candidates: the whole warp loads each row at once (one
                // memory round trip) and runs the canonical chain on shuffles
                unsigned mm = mask;
                while (mm) {
                  const int src = __ffs(mm) - 1;
                  mm &= mm - 1;
                  const int64_t ps = __shfl_sync(0xffffffffu, pos, src);
                  const float e = warp_canonical_d2(qrow4, X4 + (size_t)ps * m4, m4, lane);
                  if (lane == src) key = dev::make_key(e, (uint32_t)a.ids[pos]);
                }
              } else if (cj) {
                // many: one row per lane, loads issued kIlp words at a time
                const float e = canonical_d2_ilp(qrow4, X4 + (size_t)pos * m4, m4);
                key = dev::make_key(e, (uint32_t)a.ids[pos]);
              }
              if (lane == 0) atomicAdd(&S.rechecks, (unsigned long long)__popc(mask));
              u64* lj = ql + S.loff[j];
              if (__popc(mask) > 3) {
                cc = warp_merge_keys(lj, cc, kq, key, (cc == kq) ? lj[kq - 1] : S.thr[j], lane);
              } else {
                while (mask) {
                  const int src = __ffs(mask) - 1;
                  mask &= mask - 1;
                  const u64 kk = __shfl_sync(0xffffffffu, key, src);
                  const u64 kth = (cc == kq) ? lj[kq - 1] : S.thr[j];
                  if (kk < kth) cc = dev::warp_insert(lj, cc, kq, kk, lane);
                }
              }
              if (lane == 0) {
                S.cnt4[qd][j] = cc;
                // a full quarter list's k-th bounds the item's k-th
                if (cc == kq) atomic_min_float_nonneg(&S.Tq[j], dev::key_d2(lj[kq - 1]));
              }
              __syncwarp();
            }
            if (refresh && gth != kNoKey) {
              const float g = dev::key_d2(gth);
              if (g < S.Tq[c0 + lane]) atomic_min_float_nonneg(&S.Tq[c0 + lane], g);
            }
          }
        }
        dev::tc_fence_before();
        mbar_arrive(&S.tempty[t]);
        PROF_ADD(2);
      }
      if (split && a.ub && tid < nqg) {
        const float u = __ldcg(&a.ub[S.slot[tid]]);
        if (u < S.H[tid]) atomic_min_float_nonneg(&S.H[tid], u);
      }
      epi_sync();
      if (split) {
        // deferred re-checks: only candidates whose lower bound still reaches the
        // part's final bound (round threshold, smallest upper bound, best exact)
        // one warp per candidate: the lanes load the two rows, the chain of
        // fused multiply-adds runs in the canonical order on shuffled values
        const int ncb = min(S.ncb, kCandCap);
        for (int e = warp; e < ncb; e += kEpiWarps) {
          const int j = cb_j[e];
          const float T = fminf(S.H[j], dev::key_d2(*(volatile u64*)&lists[j * a.k]));
          if (!(cb_lo[e] > T)) {
            const int64_t pos = cb_pos[e];
            const float d2 = warp_canonical_d2(Q4 + (size_t)S.qrow[j] * m4, X4 + (size_t)pos * m4, m4, lane);
            if (lane == 0) {
              atomicMin(&lists[j * a.k], dev::make_key(d2, (uint32_t)a.ids[pos]));
              atomicAdd(&S.rechecks, 1ull);
            }
          }
        }
        epi_sync();
        if (tid == 0) S.ncb = 0;
      }
      if (!split) {
        // merge the quarter lists into quarter 0's, one warp per query
        for (int q = warp; q < nqg; q += kEpiWarps) {
          const int kq = S.kq[q];
          int cc = S.cnt4[0][q];
          for (int qd = 1; qd < 4; ++qd) {
            const u64* src = lists + (size_t)qd * a.qkeys + S.loff[q];
            const int n = S.cnt4[qd][q];
            for (int e = 0; e < n; ++e) {
              const u64 kk = src[e];
              u64* l0 = lists + S.loff[q];
              const u64 kth = (cc == kq) ? l0[kq - 1] : S.thr[q];
              if (kk < kth) cc = dev::warp_insert(l0, cc, kq, kk, lane);
              else break;  // the rest of a sorted list is no better
            }
          }
          // the item's list joins the slot's top-k list, whose k-th key later
          // work items admit against
          if (cc > 0 &&
              !share_list(a.topk + (size_t)S.slot[q] * a.k, a.glock + S.slot[q], lists + S.loff[q],
                          cc, kq, lists + a.qkeys + S.loff[q], lane, a.lock_tries) &&
              lane == 0)
            atomicOr(a.err, 2);
          __syncwarp();
        }
        epi_sync();
      }
      // k = 1: the part's best key enters the slot's list if it beats it
      if (split && tid < nqg) {
        const u64 best = lists[tid * a.k];
        if (best < S.thr[tid]) atomicMin(&a.topk[S.slot[tid]], best);
      }
      // one thread snapshots the abort flag before the barrier so that every
      // epilogue thread leaves the item loop at the same item
      if (tid == 0) S.stop = *abort;
      epi_sync();
      PROF_ADD(3);
      if (S.stop) break;
    }
  }
  if (prof_on && tid == 0) pr[15] = (unsigned long long)(clock64() - t_enter);  // epilogue warp 0's span
  if (prof_on)
    for (int i = 0; i < 16; ++i)
      if (pr[i]) atomicAdd(&a.prof[i], pr[i]);
  dev::tc_fence_before();
  __syncthreads();
  dev::tc_fence_after();
  if (tid == 0 && a.stat && S.rechecks) atomicAdd(a.stat, S.rechecks);
  if (warp == 0) dev::tmem_dealloc(tmem, kTmemCols);
  if (a.prof && tid == 0) {
    // first and last block end
    unsigned long long g;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g));
    atomicMin(&a.prof[22], g);
    atomicMax(&a.prof[23], g);
  }
}

// after a profiled launch: fold its timeline into the totals (16 launch span,
// 17 start skew, 18 end skew, 19 launches) and reset it for the next one
__global__ void tc_timeline_kernel(unsigned long long* prof) {
  if (prof[21] >= prof[20] && prof[23] >= prof[22]) {
    prof[16] += prof[23] - prof[20];
    prof[17] += prof[21] - prof[20];
    prof[18] += prof[23] - prof[22];
    prof[19] += 1;
  }
  prof[20] = ~0ull;
  prof[21] = 0;
  prof[22] = ~0ull;
  prof[23] = 0;
}

}  // namespace

// queries per work item of the fixed grouping (k = 1): 64; for k > 1 the
// groups are cut by launch_var_groups with at most 64 queries
int tc_group_size(int k) {
  (void)k;
  return kTcG;
}

// rb: operand bytes per row (2 kp for fp16, kp for e4m3)
static size_t tc_dyn_smem(int rb, int k, int nbuf, int qkeys) {
  // k = 1: one key per query plus the deferred re-check buffer; k > 1: four
  // lane quarters' lists of qkeys keys each
  const size_t G = (size_t)kTcG;
  return 1024 + (size_t)2 * kTcRows * rb + (size_t)nbuf * G * rb +
         (k == 1 ? G * 8 + (size_t)kCandCap * 12 : (size_t)4 * qkeys * 8);
}

int tc_scan_plan(int rb, int k, int smem_optin, size_t* smem, int* qkeys) {
  cudaFuncAttributes fa;
  if (k == 1) LF_CUDA(cudaFuncGetAttributes(&fa, tc_scan_kernel<true, false>));
  else LF_CUDA(cudaFuncGetAttributes(&fa, tc_scan_kernel<false, false>));
  const size_t avail = (size_t)smem_optin > fa.sharedSizeBytes ? smem_optin - fa.sharedSizeBytes : 0;
  if (k == 1) {
    for (int nbuf = 2; nbuf >= 1; --nbuf) {
      const size_t dyn = tc_dyn_smem(rb, k, nbuf, 0);
      if (dyn <= avail) {
        if (smem) *smem = dyn;
        if (qkeys) *qkeys = 0;
        return nbuf;
      }
    }
    return 0;
  }
  // k > 1: lists for 64 queries of the largest k if they fit; otherwise as
  // many keys as fit (a group then holds fewer queries), preferring two query
  // tiles unless one tile leaves clearly more room for lists
  const size_t target = (size_t)kTcG * k;
  size_t q[3] = {0, 0, 0};
  for (int nbuf = 1; nbuf <= 2; ++nbuf) {
    const size_t base = tc_dyn_smem(rb, k, nbuf, 0);
    if (base < avail) q[nbuf] = std::min(target, (avail - base) / 32 / 8 * 8);
  }
  int nbuf = 0;
  if (q[2] >= (size_t)k && 5 * q[2] >= 4 * q[1]) nbuf = 2;
  else if (q[1] >= (size_t)k) nbuf = 1;
  if (nbuf == 0) return 0;
  if (smem) *smem = tc_dyn_smem(rb, k, nbuf, (int)q[nbuf]);
  if (qkeys) *qkeys = (int)q[nbuf];
  return nbuf;
}

namespace {
__global__ void round_prep_kernel(int nslots, int kstride, const int32_t* __restrict__ slot_k,
                                  u64* __restrict__ topk, const int32_t* __restrict__ topk_cnt,
                                  int32_t* __restrict__ glock, float* __restrict__ ub,
                                  int32_t* __restrict__ work) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) *work = 0;
  if (t >= (int64_t)nslots * kstride) return;
  const int slot = (int)(t / kstride), z = (int)(t % kstride);
  if (z >= topk_cnt[slot]) topk[t] = kNoKey;
  if (z == 0) {
    glock[slot] = 0;
    if (ub) ub[slot] = __int_as_float(0x7f800000);
  }
  (void)slot_k;
}

__global__ void round_finish_kernel(int nslots, int kstride, const int32_t* __restrict__ slot_k,
                                    const u64* __restrict__ topk, int32_t* __restrict__ topk_cnt,
                                    u64* __restrict__ thr) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= nslots) return;
  const int kq = slot_k ? slot_k[slot] : kstride;
  const u64* l = topk + (size_t)slot * kstride;
  int lo = 0, hi = kq;  // the list ascends, padding last: count the keys
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (l[mid] != kNoKey) lo = mid + 1;
    else hi = mid;
  }
  topk_cnt[slot] = lo;
  thr[slot] = lo == kq ? l[kq - 1] : kNoKey;
}
}  // namespace

void launch_tc_round_prep(int nslots, int kstride, const int32_t* slot_k, unsigned long long* topk,
                          const int32_t* topk_cnt, int32_t* glock, float* ub, int32_t* work,
                          cudaStream_t s) {
  const int64_t tot = std::max<int64_t>((int64_t)nslots * kstride, 1);
  round_prep_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(nslots, kstride, slot_k, topk,
                                                                   topk_cnt, glock, ub, work);
  LF_CHECK_LAUNCH();
}

void launch_tc_round_finish(int nslots, int kstride, const int32_t* slot_k,
                            const unsigned long long* topk, int32_t* topk_cnt,
                            unsigned long long* thr, cudaStream_t s) {
  if (nslots == 0) return;
  round_finish_kernel<<<(nslots + 255) / 256, 256, 0, s>>>(nslots, kstride, slot_k, topk, topk_cnt,
                                                           thr);
  LF_CHECK_LAUNCH();
}

void launch_tc_query_prep(const float* Q, int nq, int mp, int kp, __half* Qh, float4* Qk,
                          cudaStream_t s) {
  if (nq <= 0) return;
  tc_query_prep_kernel<<<(nq + 7) / 8, 256, 0, s>>>(Q, nq, mp, kp, Qh, Qk);
  LF_CHECK_LAUNCH();
}

void launch_tc_query_prep8(const float* Q, int nq, int mp, int kp, unsigned char* Q8, float4* Qk,
                           cudaStream_t s) {
  if (nq <= 0) return;
  tc_query_prep8_kernel<<<(nq + 7) / 8, 256, 0, s>>>(Q, nq, mp, kp, Q8, Qk);
  LF_CHECK_LAUNCH();
}

namespace {
template <bool kSplit, bool kFp8>
void launch_tc_scan_as(const CUtensorMap& tmap, const TcScanArgs& a, const int32_t* n_items_dev,
                       const int32_t* slot_k, int grid, size_t smem, cudaStream_t s) {
  // the opt-in shared-memory size is raised only when a launch needs more than
  // any earlier one on this device (the attribute persists)
  static std::mutex mu;
  static std::map<int, size_t> set;  // device -> bytes
  int dev = 0;
  LF_CUDA(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lk(mu);
    size_t& have = set[dev];
    if (smem > have) {
      LF_CUDA(cudaFuncSetAttribute(tc_scan_kernel<kSplit, kFp8>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      have = smem;
    }
  }
  tc_scan_kernel<kSplit, kFp8><<<grid, kTcThreads, smem, s>>>(tmap, a, n_items_dev, slot_k);
  LF_CHECK_LAUNCH();
}
}  // namespace

void launch_tc_scan(const CUtensorMap& tmap, const TcScanArgs& a, const int32_t* n_items_dev,
                    const int32_t* slot_k, int grid, cudaStream_t s) {
  const size_t smem = tc_dyn_smem(a.fp8 ? a.kp : 2 * a.kp, a.k, a.nbuf, a.qkeys);
  if (a.k == 1) {
    if (a.fp8) launch_tc_scan_as<true, true>(tmap, a, n_items_dev, slot_k, grid, smem, s);
    else launch_tc_scan_as<true, false>(tmap, a, n_items_dev, slot_k, grid, smem, s);
  } else {
    if (a.fp8) launch_tc_scan_as<false, true>(tmap, a, n_items_dev, slot_k, grid, smem, s);
    else launch_tc_scan_as<false, false>(tmap, a, n_items_dev, slot_k, grid, smem, s);
  }
  if (a.prof) {
    tc_timeline_kernel<<<1, 1, 0, s>>>(a.prof);
    LF_CHECK_LAUNCH();
  }
}

}  // namespace leafi
