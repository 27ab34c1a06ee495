// Learned-filter forward on the tensor cores (Sec. 4, Sec. 5.1; Alg. 2's filter inference):
//   out[q][f] = b2_f + sum_j w2_fj relu(b1_fj + sum_i W1_fji q_i)
// for a whole query batch against every filter.
//
// The hidden layer is a (queries x m) . (m x h) product per filter, run with
// tcgen05.mma kind::tf32 at float32 accuracy by the three-term split
//   a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi,
// a_hi = a rounded to tf32 (10-bit mantissa), a_lo = a - a_hi rounded to tf32;
// the dropped a_lo b_lo term and the rounding of the low parts are below
// 2^-21 |a b|, the float32 accumulation is the same order as a CUDA-core dot
// product.  One CTA per (filter, 128-query tile): the K dimension streams in
// 32-column slices through two stages (the weight planes as 128-byte swizzled
// TMA boxes; the query planes gathered row by row with cp.async into the same
// swizzled layout, so a tile can hold any set of queries: in a search, the
// queries whose prediction of that filter a wave select can read); one thread
// issues TMA and MMA, the accumulator (128 queries x h hidden units) sits in
// TMEM and four warps read it back for the ReLU and output layer.
#include <cfloat>

#include "device_util.cuh"

namespace leafi {
namespace {

using dev::u64;

constexpr int kFRows = kFilterTile;  // queries per CTA (MMA M)
static_assert(kFRows == 128, "one MMA of M = 128 per query tile");
constexpr int kFThreads = 128;
constexpr int kSlice = 32;           // K columns per stage (128 bytes of float32)
constexpr int kAPlane = kFRows * kSlice * 4;   // 16 KB
constexpr int kBPlane = 256 * kSlice * 4;      // 32 KB (h <= 256)
constexpr int kStage = 2 * kAPlane + 2 * kBPlane;
// two stages of 96 KB: the loads of one slice overlap the MMAs of the other
constexpr int kFStages = 2;
constexpr long long kFWait = 1ll << 26;

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// instruction descriptor: kind::tf32, f32 accumulator, both operands K-major
__device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
      : "memory");
}

// query planes, slice-major (a query's 32-column slice is 128 contiguous
// bytes): Qs[p][i / 32][r][i % 32] = hi (p = 0) or lo (p = 1) of q_ri; zero padding
__global__ void qsplit_kernel(const float* __restrict__ Q, int nq, int mp, int m, int Kq, int nqp,
                              float* __restrict__ Qs) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nqp * Kq) return;
  const int r = (int)(t / Kq), i = (int)(t % Kq);
  const float v = (r < nq && i < m) ? Q[(size_t)r * mp + i] : 0.0f;
  const float hi = tf32_rna(v);
  const size_t o = ((size_t)(i / kSlice) * nqp + r) * kSlice + i % kSlice;
  Qs[o] = hi;
  Qs[(size_t)nqp * Kq + o] = tf32_rna(v - hi);
}

// weight planes from W1t [F][m][h], slice-major so that each TMA box (one
// 32-column slice of one plane, hp rows) is 16-32 KB of contiguous memory:
// Ws[(2f + p)][i / 32][j][i % 32], p = 0 hi, 1 lo
__global__ void wsplit_kernel(const float* __restrict__ W1t, int F, int m, int h, int hp, int Kq,
                              float* __restrict__ Ws) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)F * hp * Kq) return;
  const int f = (int)(t / ((int64_t)hp * Kq));
  const int j = (int)((t / Kq) % hp), i = (int)(t % Kq);
  const float w = (j < h && i < m) ? W1t[((size_t)f * m + i) * h + j] : 0.0f;
  const float hi = tf32_rna(w);
  const int nK = Kq / kSlice, kc = i / kSlice, ii = i % kSlice;
  Ws[(((size_t)(2 * f) * nK + kc) * hp + j) * kSlice + ii] = hi;
  Ws[(((size_t)(2 * f + 1) * nK + kc) * hp + j) * kSlice + ii] = tf32_rna(w - hi);
}

struct FShared {
  u64 full[kFStages], empty[kFStages], done;
  uint32_t tmem_base;
  float b1[256], w2[256];
};

// rows_of / cnt (nullable): the tile's rows are queries rows_of[f][tile*128 +
// r] for r < cnt[f] - tile*128 (the queries whose prediction of filter f a
// search can read); otherwise queries tile*128 + r of the batch.
__global__ void __launch_bounds__(kFThreads, 1) filter_tc_kernel(
    const __grid_constant__ CUtensorMap wmap, const float* __restrict__ Qs, int nq, int nqp,
    int F, int h, int hp, int Kq, const float* __restrict__ b1, const float* __restrict__ w2,
    const float* __restrict__ b2, const int32_t* __restrict__ rows_of,
    const int32_t* __restrict__ cnt, int list_stride, float* __restrict__ out,
    int32_t* __restrict__ err, unsigned long long* evals) {
  extern __shared__ __align__(1024) unsigned char fsm_raw[];
  __shared__ FShared S;
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(fsm_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int f = blockIdx.x, tile = blockIdx.y;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int rows = min(kFRows, (cnt ? cnt[f] : nq) - tile * kFRows);
  if (rows <= 0) return;  // the whole block: nothing to predict
  if (evals && tid == 0) atomicAdd(evals, (unsigned long long)rows);
  const int nK = Kq / kSlice;
  // thread tid owns row tid of the tile: it gathers that query's operand
  // slices and, as TMEM lane tid, writes its prediction
  const int q = tid < rows ? (cnt ? rows_of[(size_t)f * list_stride + tile * kFRows + tid]
                                  : tile * kFRows + tid)
                           : -1;
  if (tid == 0) {
    for (int i = 0; i < kFStages; ++i) {
      dev::mbar_init(&S.full[i], 1);
      dev::mbar_init(&S.empty[i], 1);
    }
    dev::mbar_init(&S.done, 1);
  }
  for (int j = tid; j < hp; j += kFThreads) {
    S.b1[j] = j < h ? b1[(size_t)f * h + j] : 0.0f;
    S.w2[j] = j < h ? w2[(size_t)f * h + j] : 0.0f;
  }
  if (warp == 0) dev::tmem_alloc(&S.tmem_base, 256);
  dev::fence_async_smem();
  dev::tc_fence_before();
  __syncthreads();
  dev::tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  // query planes of slice kc into its stage: row tid, eight 16-byte pieces per
  // plane placed as the 128-byte swizzle places them (piece c of row r at
  // piece c ^ (r & 7) of the row); a padding row reads nothing and is zero
  auto load_a = [&](int kc) {
    unsigned char* st = sm + (kc % kFStages) * kStage;
    const int src_bytes = q >= 0 ? 16 : 0;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const float* src = Qs + (size_t)p * nqp * Kq + ((size_t)kc * nqp + (q >= 0 ? q : 0)) * kSlice;
      unsigned char* dst = st + p * kAPlane + tid * 128;
#pragma unroll
      for (int c = 0; c < 8; ++c)
        dev::cp_async16_zfill(dst + ((c ^ (tid & 7)) << 4), src + 4 * c, src_bytes);
    }
    dev::cp_async_commit();
  };
  // weight planes of slice kc (thread 0): two 128-byte swizzled TMA boxes
  const uint32_t bbytes = (uint32_t)(2 * hp * kSlice * 4);
  long long b_issued[kFStages] = {}, b_done[kFStages] = {};
  auto load_b = [&](int kc) {
    const int sx = kc % kFStages;
    unsigned char* st = sm + sx * kStage;
    dev::mbar_expect_tx(&S.full[sx], bbytes);
    dev::tma_load_2d(st + 2 * kAPlane, &wmap, 0, ((2 * f) * nK + kc) * hp, &S.full[sx]);
    dev::tma_load_2d(st + 2 * kAPlane + kBPlane, &wmap, 0, ((2 * f + 1) * nK + kc) * hp,
                     &S.full[sx]);
    ++b_issued[sx];
  };
  const uint32_t idesc = idesc_tf32(kFRows, hp);
  int bad = 0;
  for (int kc = 0; kc < nK && kc < kFStages; ++kc) {
    load_a(kc);
    if (tid == 0) load_b(kc);
  }
  for (int kc = 0; kc < nK; ++kc) {
    const int s = kc % kFStages;
    const uint32_t ph = (uint32_t)((kc / kFStages) & 1);
    // this thread's pieces of slice kc have landed (the next slice may pend)
    if (kc + 1 < nK) dev::cp_async_wait_group<1>();
    else dev::cp_async_wait_all();
    dev::fence_async_smem();
    if (__syncthreads_or(bad)) break;  // every row of slice kc is in shared memory
    if (tid == 0) {
      const bool okb = dev::mbar_wait(&S.full[s], ph, kFWait);
      if (okb) {
        ++b_done[s];
        dev::tc_fence_after();
        const uint32_t base = dev::smem_addr(sm + s * kStage);
        const uint64_t ahi = dev::smem_desc(base, 16, 1024, 2);
        const uint64_t alo = dev::smem_desc(base + kAPlane, 16, 1024, 2);
        const uint64_t bhi = dev::smem_desc(base + 2 * kAPlane, 16, 1024, 2);
        const uint64_t blo = dev::smem_desc(base + 2 * kAPlane + kBPlane, 16, 1024, 2);
        // four K steps of 8 tf32 (32 bytes) inside each 128-byte swizzled row
        for (int ks = 0; ks < kSlice / 8; ++ks) {
          const uint64_t o = (uint64_t)(ks * 2);
          mma_tf32(tmem, ahi + o, bhi + o, idesc, (kc | ks) ? 1u : 0u);
          mma_tf32(tmem, ahi + o, blo + o, idesc, 1u);
          mma_tf32(tmem, alo + o, bhi + o, idesc, 1u);
        }
      } else {
        bad = 1;
      }
      // arrives once the MMAs issued so far are done (at once if none)
      dev::mma_commit(&S.empty[s]);
    }
    if (kc + kFStages < nK) {
      // the stage is refilled once the MMAs reading it are done
      if (!dev::mbar_wait(&S.empty[s], ph, kFWait)) bad = 1;
      if (__syncthreads_or(bad)) break;
      load_a(kc + kFStages);
      if (tid == 0) load_b(kc + kFStages);
    }
  }
  if (tid == 0) dev::mma_commit(&S.done);
  // every thread waits for the accumulator (bounded)
  if (!dev::mbar_wait(&S.done, 0u, kFWait)) bad = 1;
  // copies still in flight after a failure land before the block exits
  dev::cp_async_wait_all();
  if (tid == 0)
    for (int sx = 0; sx < kFStages; ++sx)
      if (b_issued[sx] > b_done[sx])
        dev::mbar_wait(&S.full[sx], (uint32_t)((b_issued[sx] - 1) & 1), kFWait);
  const bool okw = !__syncthreads_or(bad);
  dev::tc_fence_after();
  if (okw) {
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    float y = 0.0f;
    for (int c0 = 0; c0 < hp; c0 += 16) {
      float z[16];
      dev::tmem_ld16(tl + (uint32_t)c0, z);
#pragma unroll
      for (int jj = 0; jj < 16; ++jj)
        y = fmaf(fmaxf(z[jj] + S.b1[c0 + jj], 0.0f), S.w2[c0 + jj], y);
    }
    if (q >= 0) out[(size_t)q * F + f] = b2[f] + y;
  } else if (tid == 0) {
    atomicOr(err, 2);
  }
  dev::tc_fence_before();
  __syncthreads();
  if (warp == 0) dev::tmem_dealloc(tmem, 256);
}

}  // namespace

bool filter_tc_fits(int m, int h, int smem_optin) {
  const int hp = (h + 15) / 16 * 16;
  (void)m;
  return h >= 1 && hp <= 256 && (size_t)(1024 + kFStages * kStage) + sizeof(FShared) <= (size_t)smem_optin;
}

void launch_wsplit(const float* W1t, int F, int m, int h, float* Ws, cudaStream_t s) {
  const int hp = (h + 15) / 16 * 16, Kq = (m + kSlice - 1) / kSlice * kSlice;
  const int64_t tot = (int64_t)F * hp * Kq;
  if (tot == 0) return;
  wsplit_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(W1t, F, m, h, hp, Kq, Ws);
  LF_CHECK_LAUNCH();
}

void launch_filter_tc(const CUtensorMap& wmap, const float* Q, int nq, int mp, int m, int F,
                      int h, float* Qs, const float* b1, const float* w2, const float* b2,
                      float* out, int32_t* err, cudaStream_t s, const int32_t* rows_of,
                      const int32_t* cnt, unsigned long long* evals) {
  if (nq <= 0 || F <= 0) return;
  const int hp = (h + 15) / 16 * 16, Kq = (m + kSlice - 1) / kSlice * kSlice;
  const int nqp = (nq + kFRows - 1) / kFRows * kFRows;
  const int64_t tot = (int64_t)nqp * Kq;
  qsplit_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Q, nq, mp, m, Kq, nqp, Qs);
  LF_CHECK_LAUNCH();
  const size_t smem = 1024 + kFStages * (size_t)kStage;
  LF_CUDA(cudaFuncSetAttribute(filter_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem));
  dim3 grid(F, nqp / kFRows);
  filter_tc_kernel<<<grid, kFThreads, smem, s>>>(wmap, Qs, nq, nqp, F, h, hp, Kq, b1, w2, b2,
                                                 rows_of, cnt, nq, out, err, evals);
  LF_CHECK_LAUNCH();
}

}  // namespace leafi
