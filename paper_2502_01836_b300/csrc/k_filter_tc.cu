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
// 32-column slices (one 128-byte swizzled TMA box per operand plane) through
// kFStages stages; one thread issues TMA and MMA, the accumulator (128
// queries x h hidden units) sits in TMEM and four warps read it back for the
// ReLU and output layer.
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
// one stage of 96 KB per CTA, so two CTAs share an SM (their loads and MMAs
// overlap each other) and the 2 x F CTAs of a 256-query batch run in one wave
constexpr int kFStages = 1;
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

// query planes: Qs[r][i] = hi(q_ri), Qs[nqp + r][i] = lo(q_ri); zero padding
__global__ void qsplit_kernel(const float* __restrict__ Q, int nq, int mp, int m, int Kq, int nqp,
                              float* __restrict__ Qs) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nqp * Kq) return;
  const int r = (int)(t / Kq), i = (int)(t % Kq);
  const float v = (r < nq && i < m) ? Q[(size_t)r * mp + i] : 0.0f;
  const float hi = tf32_rna(v);
  Qs[t] = hi;
  Qs[(size_t)nqp * Kq + t] = tf32_rna(v - hi);
}

// weight planes from W1t [F][m][h]: Ws[(2f + p) hp + j][i], p = 0 hi, 1 lo
__global__ void wsplit_kernel(const float* __restrict__ W1t, int F, int m, int h, int hp, int Kq,
                              float* __restrict__ Ws) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)F * hp * Kq) return;
  const int f = (int)(t / ((int64_t)hp * Kq));
  const int j = (int)((t / Kq) % hp), i = (int)(t % Kq);
  const float w = (j < h && i < m) ? W1t[((size_t)f * m + i) * h + j] : 0.0f;
  const float hi = tf32_rna(w);
  Ws[((size_t)(2 * f) * hp + j) * Kq + i] = hi;
  Ws[((size_t)(2 * f + 1) * hp + j) * Kq + i] = tf32_rna(w - hi);
}

struct FShared {
  u64 full[kFStages], empty[kFStages], done;
  uint32_t tmem_base;
  int fail;
  float b1[256], w2[256];
};

__global__ void __launch_bounds__(kFThreads, 2) filter_tc_kernel(
    const __grid_constant__ CUtensorMap qmap, const __grid_constant__ CUtensorMap wmap, int nq,
    int nqp, int F, int h, int hp, int Kq, const float* __restrict__ b1,
    const float* __restrict__ w2, const float* __restrict__ b2, float* __restrict__ out,
    int32_t* __restrict__ err, const int32_t* __restrict__ need, unsigned long long* evals) {
  extern __shared__ __align__(1024) unsigned char fsm_raw[];
  __shared__ FShared S;
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(fsm_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int f = blockIdx.x, tile = blockIdx.y;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // predictions nobody will read are not made (the whole block leaves)
  if (need && !need[(size_t)tile * F + f]) return;
  if (evals && tid == 0) atomicAdd(evals, (unsigned long long)min(kFRows, nq - tile * kFRows));
  const int nK = Kq / kSlice;
  if (tid == 0) {
    for (int i = 0; i < kFStages; ++i) {
      dev::mbar_init(&S.full[i], 1);
      dev::mbar_init(&S.empty[i], 1);
    }
    dev::mbar_init(&S.done, 1);
    S.fail = 0;
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

  if (tid == 0) {
    const uint32_t bytes = (uint32_t)(2 * kAPlane + 2 * hp * kSlice * 4);
    auto issue = [&](int kc) {
      const int sx = kc % kFStages;
      unsigned char* st = sm + sx * kStage;
      dev::mbar_expect_tx(&S.full[sx], bytes);
      dev::tma_load_2d(st, &qmap, kc * kSlice, tile * kFRows, &S.full[sx]);
      dev::tma_load_2d(st + kAPlane, &qmap, kc * kSlice, nqp + tile * kFRows, &S.full[sx]);
      dev::tma_load_2d(st + 2 * kAPlane, &wmap, kc * kSlice, (2 * f) * hp, &S.full[sx]);
      dev::tma_load_2d(st + 2 * kAPlane + kBPlane, &wmap, kc * kSlice, (2 * f + 1) * hp,
                       &S.full[sx]);
    };
    const uint32_t idesc = idesc_tf32(kFRows, hp);
    bool ok = true;
    for (int kc = 0; kc < nK && kc < kFStages; ++kc) issue(kc);
    for (int kc = 0; kc < nK && ok; ++kc) {
      const int s = kc % kFStages;
      const uint32_t ph = (uint32_t)((kc / kFStages) & 1);
      ok = dev::mbar_wait(&S.full[s], ph, kFWait);
      if (!ok) break;
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
      dev::mma_commit(&S.empty[s]);
      if (kc + kFStages < nK) {
        ok = dev::mbar_wait(&S.empty[s], ph, kFWait);
        if (ok) issue(kc + kFStages);
      }
    }
    if (!ok) {
      S.fail = 1;
      atomicOr(err, 2);
    }
    dev::mma_commit(&S.done);
  }
  // every thread waits for the accumulator (bounded)
  const bool ok = dev::mbar_wait(&S.done, 0u, kFWait);
  const bool okw = __all_sync(0xffffffffu, ok) && !*(volatile int*)&S.fail;
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
    const int r = tile * kFRows + warp * 32 + lane;
    if (r < nq) out[(size_t)r * F + f] = b2[f] + y;
  } else if (lane == 0) {
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

void launch_filter_tc(const CUtensorMap& qmap, const CUtensorMap& wmap, const float* Q, int nq,
                      int mp, int m, int F, int h, float* Qs, const float* b1, const float* w2,
                      const float* b2, float* out, int32_t* err, cudaStream_t s,
                      const int32_t* need, unsigned long long* evals) {
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
  filter_tc_kernel<<<grid, kFThreads, smem, s>>>(qmap, wmap, nq, nqp, F, h, hp, Kq, b1, w2, b2,
                                                 out, err, need, evals);
  LF_CHECK_LAUNCH();
}

}  // namespace leafi
