// Alg. 1's random draws inside the library: the training queries of
// GenerateGlobalQueries / GenerateLocalQueries (Alg. 1), the
// filters' initial weights and the per-epoch SGD shuffles, plus float64
// z-normalisation of caller data.
//
// Every draw comes from a counter-based generator, Philox4x32-10 (Salmon,
// Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011),
// addressed by counter (i, j, tag, stream) under key (seed low, seed high), so
// results do not depend on launch shapes or thread counts.  Readings of what
// the paper leaves open: picks without replacement by Floyd's algorithm (with
// replacement when a leaf holds fewer series than requested); sigma ~ U[lo, hi]
// per query; Gaussian noise by the Box-Muller transform; re-z-normalisation in
// float64 (population sigma; rows with sigma < 1e-8 become zeros).
#include <algorithm>
#include <unordered_set>

#include "internal.h"

namespace leafi {

__host__ __device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t a = (uint64_t)0xD2511F53u * c[0];
    const uint64_t b = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t x0 = (uint32_t)(b >> 32) ^ c[1] ^ k0;
    const uint32_t x2 = (uint32_t)(a >> 32) ^ c[3] ^ k1;
    c[1] = (uint32_t)b;
    c[3] = (uint32_t)a;
    c[0] = x0;
    c[2] = x2;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

__host__ __device__ inline void gen_draw(uint64_t seed, uint32_t i, uint32_t j, uint32_t tag,
                                         uint32_t stream, uint32_t w[4]) {
  w[0] = i;
  w[1] = j;
  w[2] = tag;
  w[3] = stream;
  philox4x32_10(w, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// [0, 1) with 53 random bits: 27 bits of a, 26 of b
__host__ __device__ inline double gen_unit(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

// floor(u64 * n / 2^64): an integer in [0, n)
inline uint64_t gen_below(uint32_t a, uint32_t b, uint64_t n) {
  const unsigned __int128 v = (unsigned __int128)((((uint64_t)a) << 32) | b) * n;
  return (uint64_t)(v >> 64);
}

void gen_floyd(uint64_t seed, uint32_t tag, uint32_t stream, uint64_t n, int64_t k,
               int64_t* out) {
  std::unordered_set<int64_t> taken;
  taken.reserve((size_t)k * 2 + 1);
  for (int64_t s = 0; s < k; ++s) {
    const uint64_t j = n - (uint64_t)k + (uint64_t)s;
    uint32_t w[4];
    gen_draw(seed, (uint32_t)s, 0, tag, stream, w);
    int64_t t = (int64_t)gen_below(w[0], w[1], j + 1);
    if (!taken.insert(t).second) {
      t = (int64_t)j;
      taken.insert(t);
    }
    out[s] = t;
  }
}

void gen_with_replacement(uint64_t seed, uint32_t tag, uint32_t stream, uint64_t n, int64_t k,
                          int64_t* out) {
  for (int64_t i = 0; i < k; ++i) {
    uint32_t w[4];
    gen_draw(seed, (uint32_t)i, 0, tag, stream, w);
    out[i] = (int64_t)gen_below(w[0], w[1], n);
  }
}

void gen_epoch_perms(int epochs, int n, uint64_t seed, int32_t* perms) {
  std::vector<std::pair<uint64_t, int32_t>> v((size_t)std::max(n, 0));
  for (int e = 0; e < epochs; ++e) {
    for (int i = 0; i < n; ++i) {
      uint32_t w[4];
      gen_draw(seed, (uint32_t)i, (uint32_t)e, kTagPerm, 0, w);
      v[i] = {((uint64_t)w[0] << 32) | w[1], i};
    }
    std::sort(v.begin(), v.end());
    for (int i = 0; i < n; ++i) perms[(size_t)e * n + i] = v[i].second;
  }
}

namespace {

constexpr int kGenMaxPerLane = 16;  // m <= 512 points per query, 32 lanes

// One warp per query: source row + sigma * Box-Muller noise, then float64
// two-pass z-normalisation.  Query q < ng is global query q (stream 0);
// otherwise local query i of filter f with q - ng = f * nl + i (stream 1 + f).
__global__ void gen_queries_kernel(const float* __restrict__ X, int mp, int m,
                                   const int64_t* __restrict__ pos, int ng, int nl, int nrows,
                                   uint64_t seed, double lo, double hi, float* __restrict__ out) {
  const int q = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= nrows) return;
  uint32_t idx, stream;
  if (q < ng) {
    idx = (uint32_t)q;
    stream = 0;
  } else {
    const int r = q - ng;
    idx = (uint32_t)(r % nl);
    stream = (uint32_t)(1 + r / nl);
  }
  uint32_t w[4];
  gen_draw(seed, idx, 0, kTagSigma, stream, w);
  const double sigma = __dadd_rn(lo, __dmul_rn(__dsub_rn(hi, lo), gen_unit(w[0], w[1])));
  const float* x = X + pos[q] * (int64_t)mp;
  double v[kGenMaxPerLane];
  double sum = 0.0;
  // lane handles point pairs p = lane, lane + 32, ...: points 2p and 2p + 1
#pragma unroll
  for (int t = 0; t < kGenMaxPerLane / 2; ++t) {
    const int p = lane + 32 * t;
    v[2 * t] = 0.0;
    v[2 * t + 1] = 0.0;
    if (2 * p < m) {
      gen_draw(seed, idx, (uint32_t)p, kTagNoise, stream, w);
      const double u1 = gen_unit(w[0], w[1]), u2 = gen_unit(w[2], w[3]);
      const double rad = sqrt(__dmul_rn(-2.0, log(__dsub_rn(1.0, u1))));
      const double th = __dmul_rn(6.283185307179586, u2);
      double sn, cs;
      sincos(th, &sn, &cs);
      v[2 * t] = __dadd_rn((double)x[2 * p], __dmul_rn(sigma, __dmul_rn(rad, cs)));
      sum = __dadd_rn(sum, v[2 * t]);
      if (2 * p + 1 < m) {
        v[2 * t + 1] = __dadd_rn((double)x[2 * p + 1], __dmul_rn(sigma, __dmul_rn(rad, sn)));
        sum = __dadd_rn(sum, v[2 * t + 1]);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  const double mu = sum / (double)m;
  double ss = 0.0;
#pragma unroll
  for (int t = 0; t < kGenMaxPerLane / 2; ++t) {
    const int p = lane + 32 * t;
    if (2 * p < m) ss = fma(v[2 * t] - mu, v[2 * t] - mu, ss);
    if (2 * p + 1 < m) ss = fma(v[2 * t + 1] - mu, v[2 * t + 1] - mu, ss);
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  const double sd = sqrt(ss / (double)m);
  float* o = out + (int64_t)q * mp;
#pragma unroll
  for (int t = 0; t < kGenMaxPerLane / 2; ++t) {
    const int p = lane + 32 * t;
    if (2 * p < m) o[2 * p] = sd < 1e-8 ? 0.0f : (float)((v[2 * t] - mu) / sd);
    if (2 * p + 1 < m) o[2 * p + 1] = sd < 1e-8 ? 0.0f : (float)((v[2 * t + 1] - mu) / sd);
  }
  for (int i = m + lane; i < mp; i += 32) o[i] = 0.0f;
}

// Initial weights, U(-a, a) with a = 1/sqrt(fan in); W1 element (j, i) of
// filter f is written transposed, W1t [F][m][h]
__global__ void gen_weights_kernel(int F, int h, int m, uint64_t seed, float* __restrict__ W1t,
                                   float* __restrict__ b1, float* __restrict__ w2,
                                   float* __restrict__ b2) {
  const int64_t per = (int64_t)h * m;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double a1 = 1.0 / sqrt((double)m), a2 = 1.0 / sqrt((double)h);
  uint32_t w[4];
  if (t < per * F) {
    const int f = (int)(t / per);
    const int64_t e = t % per;  // row-major (j, i) of W1 [h][m]
    gen_draw(seed, (uint32_t)e, (uint32_t)f, kTagW1, 0, w);
    const int j = (int)(e / m), i = (int)(e % m);
    W1t[(int64_t)f * per + (int64_t)i * h + j] =
        (float)__dmul_rn(__dsub_rn(__dmul_rn(2.0, gen_unit(w[0], w[1])), 1.0), a1);
  }
  if (t < (int64_t)F * h) {
    const int f = (int)(t / h), j = (int)(t % h);
    gen_draw(seed, (uint32_t)j, (uint32_t)f, kTagB1, 0, w);
    b1[t] = (float)__dmul_rn(__dsub_rn(__dmul_rn(2.0, gen_unit(w[0], w[1])), 1.0), a1);
    gen_draw(seed, (uint32_t)j, (uint32_t)f, kTagW2, 0, w);
    w2[t] = (float)__dmul_rn(__dsub_rn(__dmul_rn(2.0, gen_unit(w[0], w[1])), 1.0), a2);
  }
  if (t < F) {
    gen_draw(seed, 0, (uint32_t)t, kTagB2, 0, w);
    b2[t] = (float)__dmul_rn(__dsub_rn(__dmul_rn(2.0, gen_unit(w[0], w[1])), 1.0), a2);
  }
}

// CNN filters' initial parameters (flat layout w1, b1, w2, b2, wo, bo):
// U(-a, a) with a = 1/sqrt(fan in), fan in 3 (w1, b1), 3C (w2, b2), C (wo, bo)
__global__ void gen_cnn_weights_kernel(int F, int C, int64_t P, uint64_t seed,
                                       float* __restrict__ theta) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P * F) return;
  const int f = (int)(t / P);
  const int64_t e = t % P;
  const int64_t e_w2 = 4 * (int64_t)C, e_wo = e_w2 + 3 * (int64_t)C * C + C;
  const double a = e < e_w2 ? 1.0 / sqrt(3.0)
                            : (e < e_wo ? 1.0 / sqrt(3.0 * (double)C) : 1.0 / sqrt((double)C));
  uint32_t w[4];
  gen_draw(seed, (uint32_t)e, (uint32_t)f, kTagCnn, 0, w);
  theta[t] = (float)__dmul_rn(__dsub_rn(__dmul_rn(2.0, gen_unit(w[0], w[1])), 1.0), a);
}

// float64 z-normalisation of rows of m floats (row strides in / out), one warp
// per row, two passes; sigma < 1e-8 gives zeros
__global__ void znorm_kernel(const float* __restrict__ in, int64_t in_stride, int64_t n, int m,
                             float* __restrict__ out, int64_t out_stride) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= n) return;
  const float* x = in + r * in_stride;
  double s = 0.0;
  for (int i = lane; i < m; i += 32) s += (double)x[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const double mu = s / (double)m;
  double ss = 0.0;
  for (int i = lane; i < m; i += 32) {
    const double d = (double)x[i] - mu;
    ss = fma(d, d, ss);
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  const double sd = sqrt(ss / (double)m);
  float* y = out + r * out_stride;
  for (int i = lane; i < m; i += 32) y[i] = sd < 1e-8 ? 0.0f : (float)(((double)x[i] - mu) / sd);
}

unsigned grid_for(int64_t threads, int block) { return (unsigned)((threads + block - 1) / block); }

}  // namespace

void launch_gen_queries(const float* X, int mp, int m, const int64_t* pos, int ng, int nl, int F,
                        uint64_t seed, double lo, double hi, float* out, cudaStream_t s) {
  const int nrows = ng + F * nl;
  if (nrows <= 0) return;
  gen_queries_kernel<<<grid_for((int64_t)nrows * 32, 256), 256, 0, s>>>(X, mp, m, pos, ng, nl,
                                                                       nrows, seed, lo, hi, out);
  LF_CHECK_LAUNCH();
}

void launch_gen_weights(int F, int h, int m, uint64_t seed, float* W1t, float* b1, float* w2,
                        float* b2, cudaStream_t s) {
  const int64_t n = (int64_t)F * h * m;
  gen_weights_kernel<<<grid_for(n, 256), 256, 0, s>>>(F, h, m, seed, W1t, b1, w2, b2);
  LF_CHECK_LAUNCH();
}

void launch_gen_cnn_weights(int F, int C, uint64_t seed, float* theta, cudaStream_t s) {
  const int64_t P = cnn_params(C), n = P * F;
  if (n <= 0) return;
  gen_cnn_weights_kernel<<<grid_for(n, 256), 256, 0, s>>>(F, C, P, seed, theta);
  LF_CHECK_LAUNCH();
}

void launch_znorm(const float* in, int64_t in_stride, int64_t n, int m, float* out,
                  int64_t out_stride, cudaStream_t s) {
  if (n <= 0) return;
  znorm_kernel<<<grid_for(n * 32, 256), 256, 0, s>>>(in, in_stride, n, m, out, out_stride);
  LF_CHECK_LAUNCH();
}

}  // namespace leafi
