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

constexpr int kTcRows = 128;     // MMA M: series per chunk
constexpr int kTcG = 64;         // queries per work item (MMA N <= 64)
constexpr int kTcThreads = 128;  // 4 warps, one TMEM lane quarter each
constexpr int kTmemCols = 2 * kTcG;
constexpr long long kWaitLimit = 1ll << 26;
constexpr int kCandCap = 2048;   // deferred re-check buffer (k = 1 rounds)

struct TcShared {
  u64 mbar[2];         // MMA of stage s finished
  u64 full[2];         // TMA of stage s landed
  uint32_t tmem_base;
  int abort;
  u64 thr[kTcG];       // slot's k-th best key at the start of the round
  float thrd[kTcG];    // its squared distance (inf if fewer than k)
  float H[kTcG];       // k = 1: smallest upper bound a + band in the part
  float qn[kTcG];      // |q|^2 (float32)
  float qnorm[kTcG];   // |q|
  int slot[kTcG], kq[kTcG], cnt[kTcG], qrow[kTcG], wide[kTcG];
  int ncb;             // buffered candidates of the current item
  unsigned long long rechecks;
};

__device__ __forceinline__ void atomic_min_float_nonneg(float* p, float v) {
  // non-negative floats order like their bit patterns
  atomicMin(reinterpret_cast<unsigned int*>(p), __float_as_uint(v));
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
  unsigned char* B = smem + 2 * tileA;       // kTcG x Kp fp16
  u64* lists = reinterpret_cast<u64*>(B + kTcG * Kp * 2);  // [kTcG][a.k]
  // k = 1 rounds defer re-checks: (query, position, lower bound) of each candidate
  int* cb_pos = reinterpret_cast<int*>(lists + kTcG * a.k);
  int* cb_j = cb_pos + kCandCap;
  float* cb_lo = reinterpret_cast<float*>(cb_j + kCandCap);
  const bool defer = (a.k == 1);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t sbo = 16u * Kp;             // bytes between 8-row groups
  const int m4 = a.mp / 4;

  if (tid == 0) {
    dev::mbar_init(&S.mbar[0], 1);
    dev::mbar_init(&S.mbar[1], 1);
    dev::mbar_init(&S.full[0], 1);
    dev::mbar_init(&S.full[1], 1);
    S.abort = 0;
    S.ncb = 0;
    S.rechecks = 0;
  }
  if (warp == 0) dev::tmem_alloc(&S.tmem_base, kTmemCols);
  dev::tc_fence_before();
  __syncthreads();
  dev::tc_fence_after();
  const uint32_t tmem = S.tmem_base;
  uint32_t mma_ph[2] = {0u, 0u};   // parity of the next completion to wait for
  uint32_t full_ph[2] = {0u, 0u};  // (only thread 0 uses full_ph)
  const int n_items = *n_items_dev;
  const float4* Q4 = reinterpret_cast<const float4*>(a.Q);
  const float4* X4 = reinterpret_cast<const float4*>(a.X);

  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
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
    const int64_t p0 = a.leaf_off[leaf] + (int64_t)part * a.part;
    const int64_t p1 = min(p0 + (int64_t)a.part, a.leaf_off[leaf + 1]);
    const int nqg = min(kTcG, cnt - grp * kTcG);
    const int N = ((nqg + 15) / 16) * 16;
    const Pair* pr = a.pairs + a.grp_off[leaf] + grp * kTcG;
    const int nchunks = (int)((p1 - p0 + kTcRows - 1) / kTcRows);

    // queries of the group: fp16 into the B tile (K-major core matrices), norms
    for (int qq = warp; qq < N; qq += kTcThreads / 32) {
      const int qrow = qq < nqg ? pr[qq].q : -1;
      float ss = 0.0f, mx = 0.0f;
      for (int i = lane; i < Kp; i += 32) {
        float v = 0.0f;
        if (qrow >= 0 && i < a.mp) v = a.Q[(size_t)qrow * a.mp + i];
        ss = fmaf(v, v, ss);
        mx = fmaxf(mx, fabsf(v));
        *reinterpret_cast<__half*>(B + (qq / 8) * sbo + (i / 8) * 128 + (qq % 8) * 16 + (i % 8) * 2) =
            __float2half_rn(v);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      }
      if (lane == 0 && qq < nqg) {
        const int slot = pr[qq].slot;
        S.slot[qq] = slot;
        S.qrow[qq] = qrow;
        S.kq[qq] = slot_k ? slot_k[slot] : a.k;
        S.thr[qq] = a.thr[slot];
        S.thrd[qq] = (a.thr[slot] == kNoKey) ? __int_as_float(0x7f800000) : dev::key_d2(a.thr[slot]);
        S.H[qq] = __int_as_float(0x7f800000);
        S.qn[qq] = ss;
        S.qnorm[qq] = sqrtf(ss);
        S.cnt[qq] = 0;
        S.wide[qq] = (mx >= 30000.0f) ? 1 : 0;  // outside the safe fp16 range: re-check all
        if (S.kq[qq] == 1) lists[qq * a.k] = S.thr[qq];
      }
    }
    // A tile of chunk c: columns [64 kb, 64 kb + 64) of rows r0..r0+127 are one
    // TMA box (128-byte rows, 128-byte swizzle) landing at kb * 16 KB.
    auto issue_tma = [&](int c, int st) {
      unsigned char* dst = st ? A1 : A0;
      const int r0 = (int)(p0 + (int64_t)c * kTcRows);
      dev::mbar_expect_tx(&S.full[st], (uint32_t)tileA);
      for (int kb = 0; kb < Kp / 64; ++kb)
        dev::tma_load_2d(dst + kb * 16384, &tmap, kb * 64, r0, &S.full[st]);
    };
    auto issue_mma = [&](int c) {
      const int st = c & 1;
      if (!dev::mbar_wait(&S.full[st], full_ph[st], kWaitLimit)) {
        atomicOr(a.err, 2);
        S.abort = 1;
      }
      full_ph[st] ^= 1u;
      dev::tc_fence_after();
      const uint32_t idesc = dev::idesc_f16(kTcRows, N);
      const uint32_t a_base = dev::smem_addr(st ? A1 : A0), b_base = dev::smem_addr(B);
      for (int kk = 0; kk < Kp / 16; ++kk)
        dev::mma_f16(tmem + (uint32_t)(st * kTcG),
                     dev::smem_desc(a_base + (kk >> 2) * 16384 + (kk & 3) * 32, 16, 1024, 2),
                     dev::smem_desc(b_base + kk * 256, 128, sbo), idesc, kk > 0 ? 1u : 0u);
      dev::mma_commit(&S.mbar[st]);
    };
    dev::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      issue_tma(0, 0);
      if (nchunks > 1) issue_tma(1, 1);
      issue_mma(0);
    }

    for (int c = 0; c < nchunks; ++c) {
      const int s = c & 1;
      const bool ok = dev::mbar_wait(&S.mbar[s], mma_ph[s], kWaitLimit);
      mma_ph[s] ^= 1u;
      if (!ok && tid == 0) {
        atomicOr(a.err, 2);
        S.abort = 1;
      }
      dev::tc_fence_after();
      if (tid == 0 && ok) {
        if (c + 2 < nchunks) issue_tma(c + 2, s);  // stage s is free: MMA(c) is done
        if (c + 1 < nchunks) issue_mma(c + 1);     // overlaps this chunk's epilogue
      }

      // ---- epilogue: one series row per thread
      const int64_t r0 = p0 + (int64_t)c * kTcRows;
      const int r = warp * 32 + lane;
      const bool valid = r0 + r < p1;
      const int64_t pos = r0 + r;
      const float xn = valid ? a.xn[pos] : 0.0f;
      const float xnorm = sqrtf(xn);
      const float cK = 9.7656250e-4f + 2.3841858e-7f + (float)Kp * 1.1920929e-7f;
      const float sm = sqrtf((float)a.mp) * 5.9604645e-8f;
      const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(s * kTcG);
      if (defer) {
        // 1-NN round, one pass: the part's smallest upper bound so far (block
        // running value and this warp's rows) caps the admission bound
        for (int c0 = 0; c0 < N; c0 += 16) {
          float d[16];
          dev::tmem_ld16(tl + (uint32_t)c0, d);
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int j = c0 + jj;
            if (j < nqg) {
              float lov = __int_as_float(0x7f800000), hiv = __int_as_float(0x7f800000);
              if (valid) {
                const float ap = S.qn[j] + xn - 2.0f * d[jj];
                const float band = 2.0f * (cK * S.qnorm[j] * xnorm + sm * (S.qnorm[j] + xnorm)) +
                                   1e-4f * (S.qn[j] + xn);
                lov = ap - band;
                hiv = fmaxf(ap + band, 0.0f);
              }
              float hw = hiv;
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) hw = fminf(hw, __shfl_xor_sync(0xffffffffu, hw, o));
              const float T = fminf(fminf(S.thrd[j], fminf(S.H[j], hw)),
                                    dev::key_d2(*(volatile u64*)&lists[j * a.k]));
              if (valid && (S.wide[j] || !(lov > T))) {
                const int slotc = atomicAdd(&S.ncb, 1);
                if (slotc < kCandCap) {
                  cb_pos[slotc] = (int)pos;
                  cb_j[slotc] = j;
                  cb_lo[slotc] = S.wide[j] ? -1.0f : lov;
                } else {
                  const float e = dev::canonical_d2(Q4 + (size_t)S.qrow[j] * m4, X4 + (size_t)pos * m4, m4);
                  atomicMin(&lists[j * a.k], dev::make_key(e, (uint32_t)a.ids[pos]));
                  atomicAdd(&S.rechecks, 1ull);
                }
              }
              if (lane == 0) atomic_min_float_nonneg(&S.H[j], hw);
            }
          }
        }
      } else {
        // pass 1 (k = 1 queries): H_j = min over rows of a + band
        for (int c0 = 0; c0 < N; c0 += 16) {
          float d[16];
          dev::tmem_ld16(tl + (uint32_t)c0, d);
  #pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int j = c0 + jj;
            if (j < nqg && S.kq[j] == 1) {
              float hiv = __int_as_float(0x7f800000);
              if (valid) {
                const float ap = S.qn[j] + xn - 2.0f * d[jj];
                const float band = 2.0f * (cK * S.qnorm[j] * xnorm + sm * (S.qnorm[j] + xnorm)) +
                                   1e-4f * (S.qn[j] + xn);
                hiv = fmaxf(ap + band, 0.0f);
              }
  #pragma unroll
              for (int o = 16; o > 0; o >>= 1) hiv = fminf(hiv, __shfl_xor_sync(0xffffffffu, hiv, o));
              if (lane == 0) atomic_min_float_nonneg(&S.H[j], hiv);
            }
          }
        }
        __syncthreads();
        // pass 2: admission, canonical re-check, top-k update
        for (int turn = 0; turn < 4; ++turn) {
          for (int c0 = 0; c0 < N; c0 += 16) {
            float d[16];
            dev::tmem_ld16(tl + (uint32_t)c0, d);
  #pragma unroll 1
            for (int jj = 0; jj < 16; ++jj) {
              const int j = c0 + jj;
              if (j >= nqg) break;
              const int kq = S.kq[j];
              // k = 1 is handled by every warp in turn 0 (atomic min); k > 1 one warp per turn
              if (kq == 1 ? (turn != 0) : (turn != warp)) continue;
              bool cand = false;
              if (valid) {
                const float ap = S.qn[j] + xn - 2.0f * d[jj];
                const float band = 2.0f * (cK * S.qnorm[j] * xnorm + sm * (S.qnorm[j] + xnorm)) +
                                   1e-4f * (S.qn[j] + xn);
                float T = S.thrd[j];
                if (kq == 1) {
                  T = fminf(fminf(T, S.H[j]), dev::key_d2(*(volatile u64*)&lists[j * a.k]));
                } else if (S.cnt[j] == kq) {
                  T = fminf(T, dev::key_d2(lists[j * a.k + kq - 1]));
                }
                cand = S.wide[j] || !(ap - band > T);
              }
              u64 key = kNoKey;
              if (kq == 1) {
                if (cand) {
                  // defer: the part's final bound usually rejects it without a re-check
                  const int slotc = defer ? atomicAdd(&S.ncb, 1) : kCandCap;
                  if (slotc < kCandCap) {
                    const float ap = S.qn[j] + xn - 2.0f * d[jj];
                    const float band = 2.0f * (cK * S.qnorm[j] * xnorm + sm * (S.qnorm[j] + xnorm)) +
                                       1e-4f * (S.qn[j] + xn);
                    cb_pos[slotc] = (int)pos;
                    cb_j[slotc] = j;
                    cb_lo[slotc] = S.wide[j] ? -1.0f : ap - band;
                  } else {
                    const float e = dev::canonical_d2(Q4 + (size_t)S.qrow[j] * m4, X4 + (size_t)pos * m4, m4);
                    atomicMin(&lists[j * a.k], dev::make_key(e, (uint32_t)a.ids[pos]));
                    atomicAdd(&S.rechecks, 1ull);
                  }
                }
              } else {
                if (cand) {
                  const float e = dev::canonical_d2(Q4 + (size_t)S.qrow[j] * m4, X4 + (size_t)pos * m4, m4);
                  key = dev::make_key(e, (uint32_t)a.ids[pos]);
                  atomicAdd(&S.rechecks, 1ull);
                }
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
          __syncthreads();
        }
      }
      dev::tc_fence_before();
      __syncthreads();
      if (S.abort) break;
    }
    if (S.abort) break;
    // deferred re-checks: only candidates whose lower bound still reaches the
    // part's final bound (round threshold, smallest upper bound, best exact)
    if (defer) {
      const int ncb = min(S.ncb, kCandCap);
      for (int e = tid; e < ncb; e += kTcThreads) {
        const int j = cb_j[e];
        const float T = fminf(fminf(S.thrd[j], S.H[j]),
                              dev::key_d2(*(volatile u64*)&lists[j * a.k]));
        if (!(cb_lo[e] > T)) {
          const int64_t pos = cb_pos[e];
          const float d2 = dev::canonical_d2(Q4 + (size_t)S.qrow[j] * m4, X4 + (size_t)pos * m4, m4);
          atomicMin(&lists[j * a.k], dev::make_key(d2, (uint32_t)a.ids[pos]));
          atomicAdd(&S.rechecks, 1ull);
        }
      }
      __syncthreads();
      if (tid == 0) S.ncb = 0;
    }
    // k = 1 lists hold the part's best key if it beat the round's threshold
    if (tid < nqg && S.kq[tid] == 1) S.cnt[tid] = (lists[tid * a.k] < S.thr[tid]) ? 1 : 0;
    __syncthreads();
    for (int q = warp; q < nqg; q += kTcThreads / 32) {
      const int c = S.cnt[q];
      if (c == 0) continue;
      const int slot = S.slot[q];
      int base = 0;
      if (lane == 0) base = atomicAdd(&a.cand_cnt[slot], c);
      base = __shfl_sync(0xffffffffu, base, 0);
      if (base + c > a.cand_cap) {
        if (lane == 0) atomicOr(a.err, 1);
        continue;
      }
      for (int e = lane; e < c; e += 32)
        a.cand[(size_t)slot * a.cand_cap + base + e] = lists[q * a.k + e];
    }
    __syncthreads();
  }
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
