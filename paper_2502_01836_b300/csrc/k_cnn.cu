// CNN filters (Sec. 5.2, model-type study): two convolutional layers of
// kernel size 3 with C = m latent channels.  Readings of what the paper leaves
// open (the same in the oracle): one input channel, stride 1 and zero padding
// 1 (every layer keeps length m), bias and ReLU after both convolutions, a
// head that averages each channel over the m positions followed by a linear
// layer C -> 1 without activation, predicting the Euclidean d^L like the MLP.
//
// Parameters of one filter, flat float32 (P = 3C^2 + 6C + 1):
//   w1 [C][3], b1 [C], w2 [C][C][3] (out, in, tap), b2 [C], wo [C], bo.
//
// Forward for a query batch against all filters in one launch (one block per
// (filter, query tile); the first layer's activations of one query at a time
// live in shared memory, each thread accumulates a 4-channel x 8-position tile
// of the second layer), and SGD of all filters in one launch (one block per
// filter, the protocol of the MLP trainer: minibatch MSE, lr / 10 after
// `patience` epochs without a lower validation loss, best-validation
// parameters restored).  Float32 throughout; the second layer is the dense
// part (3C MACs per output) and runs on the CUDA cores.
#include <cfloat>

#include "internal.h"

namespace leafi {
namespace {

constexpr int kCT = 4;    // output channels per thread tile
constexpr int kPT = 8;    // positions per thread tile
constexpr int kCnnQ = 8;  // queries per forward block (processed in turn)

struct Lay {
  int64_t w1, b1, w2, b2, wo, bo, P;
};

__host__ __device__ inline Lay lay(int C) {
  Lay l;
  l.w1 = 0;
  l.b1 = 3 * (int64_t)C;
  l.w2 = l.b1 + C;
  l.b2 = l.w2 + 3 * (int64_t)C * C;
  l.wo = l.b2 + C;
  l.bo = l.wo + C;
  l.P = l.bo + 1;
  return l;
}

// row stride of the padded activation planes: position i sits at column i + 1,
// columns 0 and >= m + 1 hold zeros, and every 8-position tile reads 10 columns
__host__ __device__ inline int act_stride(int m) { return (m + kPT - 1) / kPT * kPT + 2; }

__device__ __forceinline__ float block_sum(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float s = 0.0f;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

// first layer of one query: x (padded, ms columns) -> a1 [C][ms] (ReLU'd)
// (no __restrict__ on th: the trainer updates the parameters in the same
// kernel, so their loads must not go through the non-coherent cache)
__device__ __forceinline__ void conv1(const float* th, const Lay& L, int C, int m,
                                      int ms, const float* xs, float* a1) {
  for (int e = threadIdx.x; e < C * m; e += blockDim.x) {
    const int c = e / m, i = e - (e / m) * m;
    float z = th[L.b1 + c];
    z = fmaf(th[L.w1 + 3 * c + 0], xs[i], z);
    z = fmaf(th[L.w1 + 3 * c + 1], xs[i + 1], z);
    z = fmaf(th[L.w1 + 3 * c + 2], xs[i + 2], z);
    a1[c * ms + i + 1] = fmaxf(z, 0.0f);
  }
}

// second layer, tile (channels c0..c0+3, positions i0..i0+7): pre-activations
// (kRO: the parameters are read-only for the kernel's lifetime, so the
// non-coherent cache may serve them; the trainer updates them in place)
template <bool kRO>
__device__ __forceinline__ void conv2_tile(const float* th, const Lay& L, int C,
                                           int ms, const float* a1, int c0, int i0,
                                           float acc[kCT][kPT]) {
#pragma unroll
  for (int r = 0; r < kCT; ++r) {
    const float b = c0 + r < C ? th[L.b2 + c0 + r] : 0.0f;
#pragma unroll
    for (int j = 0; j < kPT; ++j) acc[r][j] = b;
  }
  for (int cp = 0; cp < C; ++cp) {
    float a[kPT + 2];
    const float* row = a1 + cp * ms + i0;  // column i0 = position i0 - 1
#pragma unroll
    for (int j = 0; j < kPT + 2; ++j) a[j] = row[j];
#pragma unroll
    for (int r = 0; r < kCT; ++r) {
      if (c0 + r >= C) break;
      const float* w = th + L.w2 + ((int64_t)(c0 + r) * C + cp) * 3;
      const float w0 = kRO ? __ldg(w) : w[0], w1 = kRO ? __ldg(w + 1) : w[1],
                  w2 = kRO ? __ldg(w + 2) : w[2];
#pragma unroll
      for (int j = 0; j < kPT; ++j) {
        float z = acc[r][j];
        z = fmaf(w0, a[j], z);
        z = fmaf(w1, a[j + 1], z);
        z = fmaf(w2, a[j + 2], z);
        acc[r][j] = z;
      }
    }
  }
}

// out[q][f] for every query of the block's tile
__global__ void cnn_fwd_kernel(const float* __restrict__ Q, int nq, int mp, int m, int F, int C,
                               const float* __restrict__ theta, float* __restrict__ out) {
  extern __shared__ float sm[];
  const int ms = act_stride(m);
  const int npg = (m + kPT - 1) / kPT, ncg = (C + kCT - 1) / kCT;
  float* xs = sm;                 // [ms]
  float* a1 = xs + ms;            // [C][ms]
  float* part = a1 + C * ms;      // [C][npg] ReLU sums of the tiles
  float* red = part + C * npg;    // [32]
  const int f = blockIdx.x;
  const Lay L = lay(C);
  const float* th = theta + (int64_t)f * L.P;
  for (int e = threadIdx.x; e < ms + C * ms; e += blockDim.x) sm[e] = 0.0f;
  __syncthreads();
  for (int qq = 0; qq < kCnnQ; ++qq) {
    const int q = blockIdx.y * kCnnQ + qq;
    if (q >= nq) break;
    for (int i = threadIdx.x; i < m; i += blockDim.x) xs[i + 1] = Q[(int64_t)q * mp + i];
    __syncthreads();
    conv1(th, L, C, m, ms, xs, a1);
    __syncthreads();
    for (int tile = threadIdx.x; tile < ncg * npg; tile += blockDim.x) {
      const int cg = tile / npg, pg = tile - (tile / npg) * npg;
      const int c0 = cg * kCT, i0 = pg * kPT;
      float acc[kCT][kPT];
      conv2_tile<true>(th, L, C, ms, a1, c0, i0, acc);
#pragma unroll
      for (int r = 0; r < kCT; ++r) {
        if (c0 + r >= C) break;
        float s = 0.0f;
#pragma unroll
        for (int j = 0; j < kPT; ++j)
          if (i0 + j < m) s += fmaxf(acc[r][j], 0.0f);
        part[(c0 + r) * npg + pg] = s;
      }
    }
    __syncthreads();
    float contrib = 0.0f;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
      float s = 0.0f;
      for (int g = 0; g < npg; ++g) s += part[c * npg + g];
      contrib = fmaf(th[L.wo + c], s / (float)m, contrib);
    }
    const float y = block_sum(contrib, red);
    if (threadIdx.x == 0) out[(int64_t)q * F + f] = th[L.bo] + y;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ SGD
// One block per filter.  Shared memory per sample: x (padded), a1 [C][ms]
// (first-layer activations), d2 [C][ms] (second-layer pre-activations, later
// their gradient), gz1 [C][ms] (the first layer's gradient), pooled means p [C].
// Gradients of a minibatch accumulate in global memory (each element owned
// by one thread across the samples, so no atomics); the second layer's
// weight gradient is tiled 2 output x 2 input channels x 3 taps per thread.
struct CnnTrainShared {
  float y, dy, tgt, b;
  int stop;
  double vsum;
  float red[32];
};

__device__ __forceinline__ const float* cnn_sample(const CnnTrainArgs& a, int f, int s, bool val,
                                                   float* target) {
  const int nl = a.n_ltrain + a.n_lval;
  if (!val) {
    if (s < a.n_gtrain) {
      *target = a.Tg[(size_t)s * a.F + f];
      return a.Qg + (size_t)s * a.mp;
    }
    const int l = s - a.n_gtrain;
    *target = a.Tl[(size_t)f * nl + l];
    return a.Ql + ((size_t)f * nl + l) * a.mp;
  }
  if (s < a.n_gval) {
    const int g = a.n_gtrain + s;
    *target = a.Tg[(size_t)g * a.F + f];
    return a.Qg + (size_t)g * a.mp;
  }
  const int l = a.n_ltrain + (s - a.n_gval);
  *target = a.Tl[(size_t)f * nl + l];
  return a.Ql + ((size_t)f * nl + l) * a.mp;
}

// forward of the sample in xs: a1 (ReLU'd), d2 (pre-activations), p, returns y
__device__ float cnn_train_forward(const float* th, const Lay& L, int C, int m, int ms,
                                   const float* xs, float* a1, float* d2, float* p, float* part,
                                   CnnTrainShared& S) {
  const int npg = (m + kPT - 1) / kPT, ncg = (C + kCT - 1) / kCT;
  conv1(th, L, C, m, ms, xs, a1);
  __syncthreads();
  for (int tile = threadIdx.x; tile < ncg * npg; tile += blockDim.x) {
    const int cg = tile / npg, pg = tile - (tile / npg) * npg;
    const int c0 = cg * kCT, i0 = pg * kPT;
    float acc[kCT][kPT];
    conv2_tile<false>(th, L, C, ms, a1, c0, i0, acc);
#pragma unroll
    for (int r = 0; r < kCT; ++r) {
      if (c0 + r >= C) break;
      float s = 0.0f;
#pragma unroll
      for (int j = 0; j < kPT; ++j)
        if (i0 + j < m) {
          d2[(c0 + r) * ms + i0 + j + 1] = acc[r][j];
          s += fmaxf(acc[r][j], 0.0f);
        }
      part[(c0 + r) * npg + pg] = s;
    }
  }
  __syncthreads();
  float contrib = 0.0f;
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    float s = 0.0f;
    for (int g = 0; g < npg; ++g) s += part[c * npg + g];
    p[c] = s / (float)m;
    contrib = fmaf(th[L.wo + c], p[c], contrib);
  }
  const float y = th[L.bo] + block_sum(contrib, S.red);
  return y;
}

__global__ void __launch_bounds__(512) cnn_train_kernel(CnnTrainArgs a) {
  extern __shared__ float sm[];
  __shared__ CnnTrainShared S;
  const int C = a.C, m = a.m;
  const int ms = act_stride(m);
  const int npg = (m + kPT - 1) / kPT;
  float* xs = sm;
  float* a1 = xs + ms;
  float* d2 = a1 + C * ms;
  float* gz1 = d2 + C * ms;
  float* p = gz1 + C * ms;
  float* part = p + C;
  const int f = blockIdx.x;
  const Lay L = lay(C);
  float* th = a.theta + (int64_t)f * L.P;
  float* bt = a.btheta + (int64_t)f * L.P;
  float* G = a.grad + (int64_t)f * L.P;
  for (int64_t e = threadIdx.x; e < L.P; e += blockDim.x) bt[e] = th[e];
  for (int e = threadIdx.x; e < ms + 3 * C * ms; e += blockDim.x) sm[e] = 0.0f;
  if (threadIdx.x == 0) S.stop = 0;
  __syncthreads();
  const int ntr = a.n_gtrain + a.n_ltrain;
  const int nval = a.n_gval + a.n_lval;
  const int C2 = (C + 1) / 2;  // 2-channel groups of the second layer's weight gradient
  float lr = a.lr0;
  double best = DBL_MAX;
  int bad = 0, decays = 0, ep = 0;
  for (ep = 0; ep < a.max_epochs; ++ep) {
    const int32_t* perm = a.perms + (size_t)ep * ntr;
    for (int st = 0; st < ntr; st += a.batch) {
      const int bs = min(a.batch, ntr - st);
      for (int64_t e = threadIdx.x; e < L.P; e += blockDim.x) G[e] = 0.0f;
      for (int b = 0; b < bs; ++b) {
        float tgt = 0.0f;
        const float* x = cnn_sample(a, f, perm[st + b], false, &tgt);
        for (int i = threadIdx.x; i < m; i += blockDim.x) xs[i + 1] = x[i];
        __syncthreads();
        const float y = cnn_train_forward(th, L, C, m, ms, xs, a1, d2, p, part, S);
        const float dy = 2.0f * (y - tgt) / (float)bs;
        // output layer; second-layer gradient dz2 = dy wo / m where z2 > 0
        for (int c = threadIdx.x; c < C; c += blockDim.x) {
          G[L.wo + c] += dy * p[c];
          const float g = dy * th[L.wo + c] / (float)m;
          float gb = 0.0f;
          for (int i = 0; i < m; ++i) {
            const float dz = d2[c * ms + i + 1] > 0.0f ? g : 0.0f;
            d2[c * ms + i + 1] = dz;
            gb += dz;
          }
          G[L.b2 + c] += gb;
        }
        if (threadIdx.x == 0) G[L.bo] += dy;
        __syncthreads();
        // w2 gradient: tiles of 2 output x 2 input channels, 3 taps
        for (int tile = threadIdx.x; tile < C2 * C2; tile += blockDim.x) {
          const int co = (tile / C2) * 2, ci = (tile - (tile / C2) * C2) * 2;
          float g[2][2][3];
#pragma unroll
          for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int v = 0; v < 2; ++v)
#pragma unroll
              for (int t = 0; t < 3; ++t) g[u][v][t] = 0.0f;
          const bool u1 = co + 1 < C, v1 = ci + 1 < C;
          const float* dz0 = d2 + co * ms;
          const float* dz1 = d2 + (u1 ? co + 1 : co) * ms;
          const float* x0 = a1 + ci * ms;
          const float* x1 = a1 + (v1 ? ci + 1 : ci) * ms;
          for (int i = 0; i < m; ++i) {
            const float e0 = dz0[i + 1], e1 = dz1[i + 1];
#pragma unroll
            for (int t = 0; t < 3; ++t) {
              const float s0 = x0[i + t], s1 = x1[i + t];  // a1 at position i + t - 1
              g[0][0][t] = fmaf(e0, s0, g[0][0][t]);
              g[0][1][t] = fmaf(e0, s1, g[0][1][t]);
              g[1][0][t] = fmaf(e1, s0, g[1][0][t]);
              g[1][1][t] = fmaf(e1, s1, g[1][1][t]);
            }
          }
#pragma unroll
          for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int v = 0; v < 2; ++v) {
              if ((u && !u1) || (v && !v1)) continue;
              float* gw = G + L.w2 + ((int64_t)(co + u) * C + ci + v) * 3;
#pragma unroll
              for (int t = 0; t < 3; ++t) gw[t] += g[u][v][t];
            }
        }
        __syncthreads();
        // first-layer gradient: dz1 = sum_c sum_t w2 dz2 where a1 > 0
        for (int tile = threadIdx.x; tile < C * npg; tile += blockDim.x) {
          const int cp = tile / npg, i0 = (tile - (tile / npg) * npg) * kPT;
          float acc[kPT];
#pragma unroll
          for (int j = 0; j < kPT; ++j) acc[j] = 0.0f;
          for (int c = 0; c < C; ++c) {
            const float* w = th + L.w2 + ((int64_t)c * C + cp) * 3;
            const float w0 = w[0], w1 = w[1], w2 = w[2];
            // position j takes dz2 at j + 1 (tap 0), j (tap 1), j - 1 (tap 2)
            float e[kPT + 2];
            const float* row = d2 + c * ms + i0;  // column i0 = position i0 - 1
#pragma unroll
            for (int jj = 0; jj < kPT + 2; ++jj) e[jj] = row[jj];
#pragma unroll
            for (int j = 0; j < kPT; ++j) {
              float z = acc[j];
              z = fmaf(w0, e[j + 2], z);
              z = fmaf(w1, e[j + 1], z);
              z = fmaf(w2, e[j], z);
              acc[j] = z;
            }
          }
#pragma unroll
          for (int j = 0; j < kPT; ++j) {
            const int i = i0 + j;
            if (i < m) gz1[cp * ms + i + 1] = a1[cp * ms + i + 1] > 0.0f ? acc[j] : 0.0f;
          }
        }
        __syncthreads();
        for (int c = threadIdx.x; c < C; c += blockDim.x) {
          float gb = 0.0f, g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
          for (int i = 0; i < m; ++i) {
            const float d = gz1[c * ms + i + 1];
            gb += d;
            g0 = fmaf(d, xs[i], g0);
            g1 = fmaf(d, xs[i + 1], g1);
            g2 = fmaf(d, xs[i + 2], g2);
          }
          G[L.b1 + c] += gb;
          G[L.w1 + 3 * c + 0] += g0;
          G[L.w1 + 3 * c + 1] += g1;
          G[L.w1 + 3 * c + 2] += g2;
        }
        __syncthreads();
      }
      for (int64_t e = threadIdx.x; e < L.P; e += blockDim.x) th[e] -= lr * G[e];
      __syncthreads();
    }
    // validation loss
    if (threadIdx.x == 0) S.vsum = 0.0;
    for (int v = 0; v < nval; ++v) {
      float tgt = 0.0f;
      const float* x = cnn_sample(a, f, v, true, &tgt);
      for (int i = threadIdx.x; i < m; i += blockDim.x) xs[i + 1] = x[i];
      __syncthreads();
      const float y = cnn_train_forward(th, L, C, m, ms, xs, a1, d2, p, part, S);
      if (threadIdx.x == 0) {
        const double e = (double)y - (double)tgt;
        S.vsum += e * e;
      }
      __syncthreads();
    }
    const double vl = S.vsum / (double)nval;
    if (vl < best) {
      best = vl;
      bad = 0;
      for (int64_t e = threadIdx.x; e < L.P; e += blockDim.x) bt[e] = th[e];
    } else if (++bad >= a.patience) {
      bad = 0;
      ++decays;
      lr = lr / 10.0f;
      if (decays > a.max_decays) {
        ++ep;
        break;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < L.P; e += blockDim.x) th[e] = bt[e];
  if (threadIdx.x == 0) {
    if (a.epochs_run) a.epochs_run[f] = ep;
    if (a.best_val) a.best_val[f] = best;
  }
}

size_t fwd_smem(int m, int C) {
  const int ms = act_stride(m), npg = (m + kPT - 1) / kPT;
  return sizeof(float) * ((size_t)ms + (size_t)C * ms + (size_t)C * npg + 32);
}

size_t train_smem(int m, int C) {
  const int ms = act_stride(m), npg = (m + kPT - 1) / kPT;
  return sizeof(float) * ((size_t)ms + 3 * (size_t)C * ms + C + (size_t)C * npg);
}

}  // namespace

int64_t cnn_params(int C) { return lay(C).P; }

bool cnn_fits(int m, int C, int smem_optin) {
  return C >= 1 && m >= 1 && (int64_t)train_smem(m, C) <= (int64_t)smem_optin &&
         (int64_t)fwd_smem(m, C) <= (int64_t)smem_optin;
}

void launch_cnn_forward(const float* Q, int nq, int mp, int m, int F, int C, const float* theta,
                        float* out, cudaStream_t s) {
  if (nq <= 0 || F <= 0) return;
  const size_t smem = fwd_smem(m, C);
  LF_CUDA(cudaFuncSetAttribute(cnn_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem));
  const int tiles = ((C + kCT - 1) / kCT) * ((m + kPT - 1) / kPT);
  const int threads = std::min(512, std::max(64, (tiles + 31) / 32 * 32));
  dim3 grid(F, (nq + kCnnQ - 1) / kCnnQ);
  cnn_fwd_kernel<<<grid, threads, smem, s>>>(Q, nq, mp, m, F, C, theta, out);
  LF_CHECK_LAUNCH();
}

void launch_cnn_train(const CnnTrainArgs& a, cudaStream_t s) {
  if (a.F <= 0) return;
  const size_t smem = train_smem(a.m, a.C);
  LF_CUDA(cudaFuncSetAttribute(cnn_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem));
  cnn_train_kernel<<<a.F, 512, smem, s>>>(a);
  LF_CHECK_LAUNCH();
}

}  // namespace leafi
