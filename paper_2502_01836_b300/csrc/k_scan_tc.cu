// Tensor-core leaf scan (SearchNode of Alg. 2 on tcgen05).
//
// A work item is (leaf, part of the leaf, group of up to kTcG queries).  The
// part's series stream through shared memory in chunks of 128 rows of an
// fp16 copy of the data: one 2-D TMA per 64-column block (128-byte rows,
// 128-byte swizzle) lands each chunk directly in the K-major layout the MMA
// reads (two stages, loads run two chunks ahead); one thread issues tcgen05.mma (M = 128 series, N =
// the query group rounded to 16, K = the padded length) into one of two TMEM
// accumulators, so the MMA of chunk c+1 overlaps the epilogue of chunk c, in
// which the four warps read their 32 TMEM lanes back (one series row per
// thread) with tcgen05.ld.  The dot products give approximate squared distances
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
constexpr int kTcThreads = kEpi + 64;
constexpr int kTmemCols = 2 * kTcG;
constexpr long long kWaitLimit = 1ll << 26;
constexpr int kCandCap = 2048;    // deferred re-check buffer (k = 1 rounds)

struct TcShared {
  u64 full[2];    // TMA of stage s landed (1 arrival + bytes)
  u64 empty[2];   // MMAs reading stage s finished (tcgen05.commit)
  u64 tfull[2];   // accumulator t written (tcgen05.commit)
  u64 tempty[2];  // accumulator t read back by the epilogue threads
  u64 bready;     // the item's query tile is in shared memory (kEpi arrivals)
  uint32_t tmem_base;
  int abort;
  int stop;            // epilogue warps' uniform snapshot of `abort`
  u64 thr[kTcG];       // slot's k-th best key at the start of the round
  float thrd[kTcG];    // its squared distance (inf if fewer than k)
  float H[kTcG];       // k = 1: smallest upper bound a + band in the part
  float4 qc[kTcG];     // per query: |q|^2, |q|, k-th best d^2 (inf if none), wide flag
  float4 qb[kTcG];     // per query band terms: U_lo, U_hi, alpha (see the epilogue)
  int slot[kTcG], kq[kTcG], cnt[kTcG], qrow[kTcG], wide[kTcG];
  int ncb;             // buffered candidates of the current item
  unsigned long long rechecks;
};

// optional per-phase cycle counters (TcScanArgs::prof, 16 entries):
// epilogue warp 0 lane 0: 0 query tile, 1 wait accumulator, 2 epilogue, 3 flush+emit;
// MMA thread: 5 wait query tile, 6 wait TMA, 7 wait accumulator free, 8 MMA issue;
// load thread: 4 wait stage free, 11 TMA issue; 9 items, 10 chunks
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
  const Pair* pr;
};

__device__ __forceinline__ Item decode_item(const TcScanArgs& a, int item) {
  int lo = 0, hi = a.L - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.item_off[mid] <= item) lo = mid; else hi = mid - 1;
  }
  const int leaf = lo;
  const int cnt = a.grp_off[leaf + 1] - a.grp_off[leaf];
  const int ngroups = (cnt + kTcG - 1) / kTcG;
  const int local = item - a.item_off[leaf];
  const int part = local / ngroups, grp = local % ngroups;
  Item it;
  it.p0 = a.leaf_off[leaf] + (int64_t)part * a.part;
  it.p1 = min(it.p0 + (int64_t)a.part, a.leaf_off[leaf + 1]);
  it.nqg = min(kTcG, cnt - grp * kTcG);
  it.N = ((it.nqg + 15) / 16) * 16;
  it.pr = a.pairs + a.grp_off[leaf] + grp * kTcG;
  it.nchunks = (int)((it.p1 - it.p0 + kTcRows - 1) / kTcRows);
  return it;
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

__global__ void __launch_bounds__(kTcThreads, 1) tc_scan_kernel(
    const __grid_constant__ CUtensorMap tmap, TcScanArgs a, const int32_t* __restrict__ n_items_dev,
    const int32_t* __restrict__ slot_k) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ TcShared S;
  // 128-byte swizzled tiles need 1024-byte aligned bases
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int Kp = a.kp;                       // fp16 row length (multiple of 64)
  const int tileA = kTcRows * Kp * 2;        // bytes per A stage
  unsigned char* A0 = smem;
  unsigned char* A1 = smem + tileA;
  unsigned char* B = smem + 2 * tileA;       // kTcG x Kp fp16, no swizzle
  u64* lists = reinterpret_cast<u64*>(B + kTcG * Kp * 2);  // [kTcG][a.k]
  int* cb_pos = reinterpret_cast<int*>(lists + kTcG * a.k);
  int* cb_j = cb_pos + kCandCap;
  float* cb_lo = reinterpret_cast<float*>(cb_j + kCandCap);
  const bool defer = (a.k == 1);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t sbo = 16u * Kp;             // B: bytes between 8-row groups
  const int m4 = a.mp / 4;
  volatile int* abort = &S.abort;

  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      dev::mbar_init(&S.full[i], 1);
      dev::mbar_init(&S.empty[i], 1);
      dev::mbar_init(&S.tfull[i], 1);
      dev::mbar_init(&S.tempty[i], kEpi);
    }
    dev::mbar_init(&S.bready, kEpi);
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
  unsigned long long pr[16];
  for (int i = 0; i < 16; ++i) pr[i] = 0;
  const bool prof_on = a.prof != nullptr && (tid == 0 || tid == kLoadWarp * 32 || tid == kMmaWarp * 32);

  if (warp == kLoadWarp) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      PROF_T0();
      long long g_ld = 0;
      uint32_t empty_ph[2] = {0u, 0u};
      for (int item = blockIdx.x; item < n_items && !*abort; item += gridDim.x) {
        const Item I = decode_item(a, item);
        for (int c = 0; c < I.nchunks; ++c) {
          const int st = (int)(g_ld & 1);
          if (g_ld >= 2) {
            PROF_ADD(11);
            const bool ok = wait_phase(&S.empty[st], empty_ph[st], abort);
            empty_ph[st] ^= 1u;
            PROF_ADD(4);
            if (!ok) break;
          }
          unsigned char* dst = st ? A1 : A0;
          const int r0 = (int)(I.p0 + (int64_t)c * kTcRows);
          dev::mbar_expect_tx(&S.full[st], (uint32_t)tileA);
          for (int kb = 0; kb < Kp / 64; ++kb)
            dev::tma_load_2d(dst + kb * 16384, &tmap, kb * 64, r0, &S.full[st]);
          ++g_ld;
        }
      }
      PROF_ADD(11);
    }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------ MMA issue
    if (lane == 0) {
      PROF_T0();
      long long g_mm = 0;
      uint32_t full_ph[2] = {0u, 0u}, tempty_ph[2] = {0u, 0u};
      uint32_t bready_ph = 0;
      for (int item = blockIdx.x; item < n_items && !*abort; item += gridDim.x) {
        const Item I = decode_item(a, item);
        bool ok = wait_phase(&S.bready, bready_ph, abort);
        bready_ph ^= 1u;
        PROF_ADD(5);
        const uint32_t idesc = dev::idesc_f16(kTcRows, I.N);
        for (int c = 0; ok && c < I.nchunks; ++c) {
          const int st = (int)(g_mm & 1);
          ok = wait_phase(&S.full[st], full_ph[st], abort);
          full_ph[st] ^= 1u;
          PROF_ADD(6);
          if (ok && g_mm >= 2) {
            ok = wait_phase(&S.tempty[st], tempty_ph[st], abort);
            tempty_ph[st] ^= 1u;
            PROF_ADD(7);
          }
          if (!ok) break;
          dev::tc_fence_after();
          const uint32_t a_base = dev::smem_addr(st ? A1 : A0), b_base = dev::smem_addr(B);
          for (int kk = 0; kk < Kp / 16; ++kk)
            dev::mma_f16(tmem + (uint32_t)(st * kTcG),
                         dev::smem_desc(a_base + (kk >> 2) * 16384 + (kk & 3) * 32, 16, 1024, 2),
                         dev::smem_desc(b_base + kk * 256, 128, sbo), idesc, kk > 0 ? 1u : 0u);
          dev::mma_commit(&S.empty[st]);
          dev::mma_commit(&S.tfull[st]);
          ++g_mm;
          PROF_ADD(8);
        }
        if (!ok) {
          atomicOr(a.err, 2);
          S.abort = 1;
        }
      }
    }
  } else {
    // ------------------------------------------------ epilogue warps 0-7
    const float4* Q4 = reinterpret_cast<const float4*>(a.Q);
    const float4* X4 = reinterpret_cast<const float4*>(a.X);
    const float cK = 9.7656250e-4f + 2.3841858e-7f + (float)Kp * 1.1920929e-7f;
    const float sm = sqrtf((float)a.mp) * 5.9604645e-8f;
    uint32_t tfull_ph[2] = {0u, 0u};
    long long g = 0;
    PROF_T0();
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
      const Item I = decode_item(a, item);
      const int nqg = I.nqg, N = I.N;
      if (prof_on) pr[9] += 1;
      // the previous item's MMAs are complete (its last accumulator was read),
      // so the query tile can be replaced
      // one warp per query row: each lane converts 8 consecutive values (16 bytes)
      for (int qq = warp; qq < N; qq += kEpiWarps) {
        const int qrow = qq < nqg ? I.pr[qq].q : -1;
        float ss = 0.0f, mx = 0.0f;
        for (int piece = lane; piece < Kp / 8; piece += 32) {
          float v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int i = piece * 8 + e;
            v[e] = (qrow >= 0 && i < a.mp) ? a.Q[(size_t)qrow * a.mp + i] : 0.0f;
            ss = fmaf(v[e], v[e], ss);
            mx = fmaxf(mx, fabsf(v[e]));
          }
          __align__(16) __half hv[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) hv[e] = __float2half_rn(v[e]);
          *reinterpret_cast<uint4*>(B + (qq / 8) * sbo + piece * 128 + (qq % 8) * 16) =
              *reinterpret_cast<const uint4*>(hv);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          ss += __shfl_xor_sync(0xffffffffu, ss, o);
          mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0 && qq < nqg) {
          const int slot = I.pr[qq].slot;
          S.slot[qq] = slot;
          S.qrow[qq] = qrow;
          S.kq[qq] = slot_k ? slot_k[slot] : a.k;
          S.thr[qq] = a.thr[slot];
          S.thrd[qq] = (a.thr[slot] == kNoKey) ? __int_as_float(0x7f800000) : dev::key_d2(a.thr[slot]);
          S.H[qq] = __int_as_float(0x7f800000);
          S.cnt[qq] = 0;
          S.wide[qq] = (mx >= 30000.0f) ? 1 : 0;  // outside the safe fp16 range: re-check all
          S.qc[qq] = make_float4(ss, sqrtf(ss), S.thrd[qq], S.wide[qq] ? 1.0f : 0.0f);
          {
            // band(q, x) = alpha |x| + beta + 1e-4 |x|^2 with alpha = 2 (c |q| + s),
            // beta = 2 s |q| + 1e-4 |q|^2; the bounds are then
            //   lo = (|q|^2 - beta) + |x|^2 (1 - 1e-4) - alpha |x| - 2 <q~, x~>
            //   hi = (|q|^2 + beta) + |x|^2 (1 + 1e-4) + alpha |x| - 2 <q~, x~>
            const float qm = sqrtf(ss);
            const float alpha = 2.0f * (cK * qm + sm);
            const float beta = 2.0f * sm * qm + 1e-4f * ss;
            S.qb[qq] = make_float4(S.wide[qq] ? -__int_as_float(0x7f800000) : ss - beta, ss + beta,
                                   alpha, 0.0f);
          }
          if (S.kq[qq] == 1) lists[qq * a.k] = S.thr[qq];
        }
      }
      dev::fence_async_smem();
      mbar_arrive(&S.bready);
      epi_sync();
      PROF_ADD(0);

      const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
      const int r = quarter * 32 + lane;
      // squared norm of this thread's row in the next chunk, loaded ahead
      float xn_next = (I.p0 + r < I.p1) ? a.xn[I.p0 + r] : 0.0f;
      for (int c = 0; c < I.nchunks; ++c) {
        const int t = (int)(g & 1);
        if (prof_on) pr[10] += 1;
        const int64_t r0 = I.p0 + (int64_t)c * kTcRows;
        const bool valid = r0 + r < I.p1;
        const int64_t pos = r0 + r;
        const float xn = valid ? xn_next : 0.0f;
        xn_next = (pos + kTcRows < I.p1) ? a.xn[pos + kTcRows] : 0.0f;
        const float xnorm = sqrtf(xn);
        const float vlo = xn * (1.0f - 1e-4f), vhi = xn * (1.0f + 1e-4f);
        // on a timeout every later wait returns at once; the loop still reaches
        // all arrivals and barriers, and the error word reports the failure
        const bool ok = wait_phase(&S.tfull[t], tfull_ph[t], abort);
        tfull_ph[t] ^= 1u;
        if (!ok) {
          atomicOr(a.err, 2);
          S.abort = 1;
        }
        PROF_ADD(1);
        const bool okw = __all_sync(0xffffffffu, ok);  // warp-uniform for tcgen05.ld
        dev::tc_fence_after();
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(t * kTcG);
        if (defer) {
          // 1-NN round, one pass over this warp's column groups (warps w and w+4
          // share the rows and split the 16-column groups); 16 columns at a
          // time so the loads and warp reductions overlap
          for (int c0 = (warp >> 2) * 16; okw && c0 < N; c0 += 32) {
            float d[16];
            dev::tmem_ld16(tl + (uint32_t)c0, d);
            float lov[16], hw[16];
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
              const int j = c0 + jj;
              lov[jj] = __int_as_float(0x7f800000);
              hw[jj] = __int_as_float(0x7f800000);
              if (valid && j < nqg) {
                const float4 qb = S.qb[j];
                lov[jj] = fmaf(-2.0f, d[jj], fmaf(-qb.z, xnorm, qb.x + vlo));
                hw[jj] = fmaxf(fmaf(-2.0f, d[jj], fmaf(qb.z, xnorm, qb.y + vhi)), 0.0f);
              }
            }
            // warp minimum of the (non-negative) upper bounds: one REDUX per column
#pragma unroll
            for (int jj = 0; jj < 16; ++jj)
              hw[jj] = __uint_as_float(__reduce_min_sync(0xffffffffu, __float_as_uint(hw[jj])));
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
              const int j = c0 + jj;
              if (j < nqg) {
                const float T = fminf(fminf(S.thrd[j], fminf(S.H[j], hw[jj])),
                                      dev::key_d2(*(volatile u64*)&lists[j * a.k]));
                if (valid && !(lov[jj] > T)) {
                  const int slotc = atomicAdd(&S.ncb, 1);
                  if (slotc < kCandCap) {
                    cb_pos[slotc] = (int)pos;
                    cb_j[slotc] = j;
                    cb_lo[slotc] = lov[jj];
                  } else {
                    const float e = dev::canonical_d2(Q4 + (size_t)S.qrow[j] * m4, X4 + (size_t)pos * m4, m4);
                    atomicMin(&lists[j * a.k], dev::make_key(e, (uint32_t)a.ids[pos]));
                    atomicAdd(&S.rechecks, 1ull);
                  }
                }
              }
            }
            if (lane == 0) {
#pragma unroll
              for (int jj = 0; jj < 16; ++jj)
                if (c0 + jj < nqg) atomic_min_float_nonneg(&S.H[c0 + jj], hw[jj]);
            }
          }
        } else {
          // general k: immediate re-checks; warps 0-3 take turns inserting into
          // the lists (warps 4-7 only join the barriers)
          for (int turn = 0; turn < 4; ++turn) {
            for (int c0 = 0; okw && warp < 4 && c0 < N; c0 += 16) {
              float d[16];
              dev::tmem_ld16(tl + (uint32_t)c0, d);
#pragma unroll 1
              for (int jj = 0; jj < 16; ++jj) {
                const int j = c0 + jj;
                if (j >= nqg) break;
                const int kq = S.kq[j];
                if (kq == 1 ? (turn != 0) : (turn != warp)) continue;
                bool cand = false;
                if (valid) {
                  const float4 qc = S.qc[j];
                  const float ap = qc.x + xn - 2.0f * d[jj];
                  const float band = 2.0f * (cK * qc.y * xnorm + sm * (qc.y + xnorm)) + 1e-4f * (qc.x + xn);
                  float T = qc.z;
                  if (kq == 1)
                    T = fminf(T, dev::key_d2(*(volatile u64*)&lists[j * a.k]));
                  else if (S.cnt[j] == kq)
                    T = fminf(T, dev::key_d2(lists[j * a.k + kq - 1]));
                  cand = S.wide[j] || !(ap - band > T);
                }
                u64 key = kNoKey;
                if (cand) {
                  const float e = dev::canonical_d2(Q4 + (size_t)S.qrow[j] * m4, X4 + (size_t)pos * m4, m4);
                  key = dev::make_key(e, (uint32_t)a.ids[pos]);
                  atomicAdd(&S.rechecks, 1ull);
                }
                if (kq == 1) {
                  if (cand) atomicMin(&lists[j * a.k], key);
                } else {
                  unsigned mask = __ballot_sync(0xffffffffu, cand);
                  int cc = S.cnt[j];
                  while (mask) {
                    const int src = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const u64 kk = __shfl_sync(0xffffffffu, key, src);
                    const u64 kth = (cc == kq) ? lists[j * a.k + kq - 1] : S.thr[j];
                    if (kk < kth) cc = dev::warp_insert(lists + j * a.k, cc, kq, kk, lane);
                  }
                  if (lane == 0) S.cnt[j] = cc;
                  __syncwarp();
                }
              }
            }
            epi_sync();
          }
        }
        dev::tc_fence_before();
        mbar_arrive(&S.tempty[t]);
        ++g;
        PROF_ADD(2);
      }
      epi_sync();
      if (defer) {
        // deferred re-checks: only candidates whose lower bound still reaches the
        // part's final bound (round threshold, smallest upper bound, best exact)
        const int ncb = min(S.ncb, kCandCap);
        for (int e = tid; e < ncb; e += kEpi) {
          const int j = cb_j[e];
          const float T = fminf(fminf(S.thrd[j], S.H[j]), dev::key_d2(*(volatile u64*)&lists[j * a.k]));
          if (!(cb_lo[e] > T)) {
            const int64_t pos = cb_pos[e];
            const float d2 = dev::canonical_d2(Q4 + (size_t)S.qrow[j] * m4, X4 + (size_t)pos * m4, m4);
            atomicMin(&lists[j * a.k], dev::make_key(d2, (uint32_t)a.ids[pos]));
            atomicAdd(&S.rechecks, 1ull);
          }
        }
        epi_sync();
        if (tid == 0) S.ncb = 0;
      }
      // k = 1 lists hold the part's best key if it beat the round's threshold
      if (tid < nqg && S.kq[tid] == 1) S.cnt[tid] = (lists[tid * a.k] < S.thr[tid]) ? 1 : 0;
      epi_sync();
      for (int q = warp; q < nqg; q += kEpiWarps) {
        const int cc = S.cnt[q];
        if (cc == 0) continue;
        const int slot = S.slot[q];
        int base = 0;
        if (lane == 0) base = atomicAdd(&a.cand_cnt[slot], cc);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base + cc > a.cand_cap) {
          if (lane == 0) atomicOr(a.err, 1);
          continue;
        }
        for (int e = lane; e < cc; e += 32)
          a.cand[(size_t)slot * a.cand_cap + base + e] = lists[q * a.k + e];
      }
      // one thread snapshots the abort flag before the barrier so that every
      // epilogue thread leaves the item loop at the same item
      if (tid == 0) S.stop = *abort;
      epi_sync();
      PROF_ADD(3);
      if (S.stop) break;
    }
  }
  if (prof_on)
    for (int i = 0; i < 16; ++i)
      if (pr[i]) atomicAdd(&a.prof[i], pr[i]);
  dev::tc_fence_before();
  __syncthreads();
  dev::tc_fence_after();
  if (tid == 0 && a.stat && S.rechecks) atomicAdd(a.stat, S.rechecks);
  if (warp == 0) dev::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

int tc_group_size() { return kTcG; }

size_t tc_scan_smem_bytes(int kp, int k) {
  return 1024 + (size_t)2 * kTcRows * kp * 2 + (size_t)kTcG * kp * 2 + (size_t)kTcG * k * 8 +
         (k == 1 ? (size_t)kCandCap * 12 : 0);
}

void launch_tc_scan(const CUtensorMap& tmap, const TcScanArgs& a, const int32_t* n_items_dev,
                    const int32_t* slot_k, int grid, cudaStream_t s) {
  const size_t smem = tc_scan_smem_bytes(a.kp, a.k);
  LF_CUDA(cudaFuncSetAttribute(tc_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  tc_scan_kernel<<<grid, kTcThreads, smem, s>>>(tmap, a, n_items_dev, slot_k);
  LF_CHECK_LAUNCH();
}

}  // namespace leafi
