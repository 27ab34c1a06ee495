// Device helpers shared by the scan kernels: result keys, warp-level top-k
// insertion, and thin wrappers over the sm_100-family PTX used by the
// tensor-core scan (shared-memory descriptors, mbarriers, tcgen05).
#pragma once
#include <cuda.h>

#include <cstdint>

#include "internal.h"

namespace leafi {
namespace dev {

typedef unsigned long long u64;

__device__ __forceinline__ u64 make_key(float d2, uint32_t id) {
  return ((u64)__float_as_uint(d2) << 32) | (u64)id;
}

__device__ __forceinline__ float key_d2(u64 k) { return __uint_as_float((uint32_t)(k >> 32)); }

// Insert `key` into the ascending list (cnt entries, capacity k <= LEAFI_MAX_K);
// all lanes of the warp call it with the same arguments.
__device__ __forceinline__ int warp_insert(u64* list, int cnt, int k, u64 key, int lane) {
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

// canonical squared distance of two padded float32 rows (m4 float4 words):
// acc = fmaf(q_i - x_i, q_i - x_i, acc) for i in order; padding is zero
__device__ __forceinline__ float canonical_d2(const float4* __restrict__ q,
                                              const float4* __restrict__ x, int m4) {
  float acc = 0.0f;
  for (int c = 0; c < m4; ++c) {
    const float4 a = q[c], b = x[c];
    float t = __fsub_rn(a.x, b.x);
    acc = __fmaf_rn(t, t, acc);
    t = __fsub_rn(a.y, b.y);
    acc = __fmaf_rn(t, t, acc);
    t = __fsub_rn(a.z, b.z);
    acc = __fmaf_rn(t, t, acc);
    t = __fsub_rn(a.w, b.w);
    acc = __fmaf_rn(t, t, acc);
  }
  return acc;
}

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor of a K-major operand.  No swizzle:
// core matrices of 8 rows x 16 bytes, `lbo` = byte step between K-adjacent
// core matrices, `sbo` = byte step between 8-row groups.  128-byte swizzle:
// rows of 128 bytes (64 fp16) in 8-row atoms of 1024 bytes, `sbo` = 1024.
// `layout` 0 = no swizzle, 2 = 128-byte swizzle (tile base 1024-byte aligned).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo,
                                              uint32_t layout = 0) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for the tcgen05 family
  d |= (uint64_t)(layout & 7u) << 61;
  return d;
}

// instruction descriptor: kind::f16 with f16 A/B, f32 accumulator, both K-major
__device__ __forceinline__ uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(u64* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(u64* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count)
               : "memory");
}

// bounded wait for the phase with parity `parity`; returns false on timeout
__device__ __forceinline__ bool mbar_wait(u64* mbar, uint32_t parity, long long limit) {
  uint32_t done = 0;
  for (long long it = 0; it < limit; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_addr(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns (one TMEM lane per thread)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// 32 consecutive accumulator columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// arrive on the mbarrier and add `bytes` to its expected transaction count
__device__ __forceinline__ void mbar_expect_tx(u64* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)),
               "r"(bytes)
               : "memory");
}

// 2-D tiled TMA load of one box into shared memory, completing on `mbar`
__device__ __forceinline__ void tma_load_2d(void* dst_smem, const CUtensorMap* tmap, int x, int y,
                                            u64* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst_smem)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_addr(mbar))
      : "memory");
}

__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst_smem)), "l"(src)
               : "memory");
}
// 16-byte asynchronous copy that reads `src_bytes` (16 or 0) and zero-fills the rest
__device__ __forceinline__ void cp_async16_zfill(void* dst_smem, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst_smem)), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// wait until at most N of this thread's committed groups are still pending
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace dev
}  // namespace leafi
