// Learned filters (Sec. 4; Sec. 5.1): MLP m -> h -> 1 with a ReLU hidden
// layer, one per filtered leaf.  Forward for a whole query batch against all
// filters in one launch, and SGD training of all filters in one launch.
#include <cfloat>

#include "internal.h"

namespace leafi {
namespace {

constexpr int kQT = 32;         // queries per forward block
constexpr int kFwdThreads = 256;
constexpr int kMaxBatch = 64;   // SGD minibatch held in registers

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// out[q][f] = b2_f + sum_j w2_fj * relu(b1_fj + sum_i W1_fji q_i)
// grid (F, ceil(nq / kQT)); each thread owns hidden units j = tid, tid + 256, ...
__global__ void __launch_bounds__(kFwdThreads) filter_fwd_kernel(
    const float* __restrict__ Q, int nq, int mp, int m, int F, int h,
    const float* __restrict__ W1t, const float* __restrict__ b1, const float* __restrict__ w2,
    const float* __restrict__ b2, float* __restrict__ out) {
  extern __shared__ float4 smem4[];
  float* Qs = reinterpret_cast<float*>(smem4);  // [m][kQT]
  __shared__ float red[kFwdThreads / 32][kQT];
  const int f = blockIdx.x;
  const int q0 = blockIdx.y * kQT;
  for (int idx = threadIdx.x; idx < kQT * m; idx += blockDim.x) {
    const int qq = idx / m, i = idx % m;
    Qs[i * kQT + qq] = (q0 + qq < nq) ? Q[(size_t)(q0 + qq) * mp + i] : 0.0f;
  }
  __syncthreads();
  const float* W = W1t + (size_t)f * m * h;
  float y[kQT];
#pragma unroll
  for (int qq = 0; qq < kQT; ++qq) y[qq] = 0.0f;
  for (int j = threadIdx.x; j < h; j += blockDim.x) {
    float z[kQT];
    const float bj = b1[(size_t)f * h + j];
#pragma unroll
    for (int qq = 0; qq < kQT; ++qq) z[qq] = bj;
    for (int i = 0; i < m; ++i) {
      const float w = W[(size_t)i * h + j];
      const float4* qv = reinterpret_cast<const float4*>(Qs + i * kQT);
#pragma unroll
      for (int c = 0; c < kQT / 4; ++c) {
        const float4 v = qv[c];
        z[4 * c + 0] = fmaf(w, v.x, z[4 * c + 0]);
        z[4 * c + 1] = fmaf(w, v.y, z[4 * c + 1]);
        z[4 * c + 2] = fmaf(w, v.z, z[4 * c + 2]);
        z[4 * c + 3] = fmaf(w, v.w, z[4 * c + 3]);
      }
    }
    const float wj = w2[(size_t)f * h + j];
#pragma unroll
    for (int qq = 0; qq < kQT; ++qq) y[qq] = fmaf(fmaxf(z[qq], 0.0f), wj, y[qq]);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int qq = 0; qq < kQT; ++qq) {
    const float s = warp_sum(y[qq]);
    if (lane == 0) red[warp][qq] = s;
  }
  __syncthreads();
  if (threadIdx.x < kQT && q0 + threadIdx.x < nq) {
    float s = 0.0f;
    for (int w = 0; w < kFwdThreads / 32; ++w) s += red[w][threadIdx.x];
    out[(size_t)(q0 + threadIdx.x) * F + f] = b2[f] + s;
  }
}

// ------------------------------------------------------------------ SGD
// One block per filter; thread j owns hidden unit j (h <= blockDim).  The
// minibatch is staged transposed in shared memory (Xt[i][b]).  MSE loss
// averaged over the minibatch; the learning rate is divided by 10 after
// `patience` epochs without a lower validation loss, training stops after
// `max_decays` divisions or max_epochs, and the best-validation weights are
// restored at the end.
struct TrainShared {
  float y[kMaxBatch];
  float dy[kMaxBatch];
  float tgt[kMaxBatch];
  int rows[kMaxBatch];
  float red[32][kMaxBatch / 2];
  float b2;
  int stop;
  double vsum;
};

__device__ __forceinline__ const float* sample_row(const TrainArgs& a, int f, int s, bool val,
                                                   float* target) {
  // train index s: [0, n_gtrain) global, [n_gtrain, +n_ltrain) local
  // val index s:   [0, n_gval) global, [n_gval, +n_lval) local
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

// y[b] for the staged batch (b < bs); z receives the hidden pre-activations
__device__ void forward_batch(const TrainArgs& a, int f, const float* Xt, int bs, float bj,
                              float wj, bool own, float* z, TrainShared& S) {
  const int j = threadIdx.x;
  const float* W = a.W1t + (size_t)f * a.m * a.h;
#pragma unroll
  for (int b = 0; b < kMaxBatch; ++b) z[b] = bj;
  if (own) {
    for (int i = 0; i < a.m; ++i) {
      const float w = W[(size_t)i * a.h + j];
      const float4* xv = reinterpret_cast<const float4*>(Xt + i * kMaxBatch);
#pragma unroll
      for (int c = 0; c < kMaxBatch / 4; ++c) {
        const float4 v = xv[c];
        z[4 * c + 0] = fmaf(w, v.x, z[4 * c + 0]);
        z[4 * c + 1] = fmaf(w, v.y, z[4 * c + 1]);
        z[4 * c + 2] = fmaf(w, v.z, z[4 * c + 2]);
        z[4 * c + 3] = fmaf(w, v.w, z[4 * c + 3]);
      }
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  // reduce relu(z) * w2 over hidden units, two halves of the batch
  for (int half = 0; half < 2; ++half) {
#pragma unroll
    for (int bb = 0; bb < kMaxBatch / 2; ++bb) {
      const int b = half * (kMaxBatch / 2) + bb;
      float c = own ? fmaxf(z[b], 0.0f) * wj : 0.0f;
      c = warp_sum(c);
      if (lane == 0) S.red[warp][bb] = c;
    }
    __syncthreads();
    if (threadIdx.x < kMaxBatch / 2) {
      float s = 0.0f;
      for (int w = 0; w < nw; ++w) s += S.red[w][threadIdx.x];
      S.y[half * (kMaxBatch / 2) + threadIdx.x] = S.b2 + s;
    }
    __syncthreads();
  }
  (void)bs;
}

__global__ void __launch_bounds__(256) train_kernel(TrainArgs a) {
  extern __shared__ float4 smem4[];
  float* Xt = reinterpret_cast<float*>(smem4);  // [m][kMaxBatch]
  __shared__ TrainShared S;
  const int f = blockIdx.x;
  const int j = threadIdx.x;
  const bool own = j < a.h;
  float bj = own ? a.b1[(size_t)f * a.h + j] : 0.0f;
  float wj = own ? a.w2[(size_t)f * a.h + j] : 0.0f;
  float* W = a.W1t + (size_t)f * a.m * a.h;
  float* BW = a.bW1t + (size_t)f * a.m * a.h;
  if (threadIdx.x == 0) {
    S.b2 = a.b2[f];
    S.stop = 0;
  }
  // best copy starts as the initial weights
  if (own) {
    for (int i = 0; i < a.m; ++i) BW[(size_t)i * a.h + j] = W[(size_t)i * a.h + j];
    a.bb1[(size_t)f * a.h + j] = bj;
    a.bw2[(size_t)f * a.h + j] = wj;
  }
  if (threadIdx.x == 0) a.bb2[f] = a.b2[f];
  __syncthreads();
  const int ntr = a.n_gtrain + a.n_ltrain;
  const int nval = a.n_gval + a.n_lval;
  float lr = a.lr0;
  double best = DBL_MAX;
  int bad = 0, decays = 0, ep = 0;
  float z[kMaxBatch];
  for (ep = 0; ep < a.max_epochs; ++ep) {
    const int32_t* perm = a.perms + (size_t)ep * ntr;
    for (int st = 0; st < ntr; st += a.batch) {
      const int bs = min(a.batch, ntr - st);
      if (threadIdx.x < kMaxBatch) {
        float t = 0.0f;
        S.rows[threadIdx.x] = threadIdx.x < bs ? perm[st + threadIdx.x] : -1;
        if (threadIdx.x < bs) sample_row(a, f, S.rows[threadIdx.x], false, &t);
        S.tgt[threadIdx.x] = t;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < kMaxBatch * a.m; idx += blockDim.x) {
        const int b = idx / a.m, i = idx % a.m;
        float t;
        Xt[i * kMaxBatch + b] = (b < bs) ? sample_row(a, f, S.rows[b], false, &t)[i] : 0.0f;
      }
      __syncthreads();
      forward_batch(a, f, Xt, bs, bj, wj, own, z, S);
      if (threadIdx.x < kMaxBatch)
        S.dy[threadIdx.x] =
            threadIdx.x < bs ? 2.0f * (S.y[threadIdx.x] - S.tgt[threadIdx.x]) / (float)bs : 0.0f;
      __syncthreads();
      // gradients of this hidden unit, then the update
      float gw2 = 0.0f, gb1 = 0.0f;
      float dz[kMaxBatch];
#pragma unroll
      for (int b = 0; b < kMaxBatch; ++b) {
        const float d = S.dy[b];
        const bool on = z[b] > 0.0f;
        gw2 = fmaf(d, on ? z[b] : 0.0f, gw2);
        dz[b] = on ? d * wj : 0.0f;
        gb1 += dz[b];
      }
      if (own) {
        for (int i = 0; i < a.m; ++i) {
          const float4* xv = reinterpret_cast<const float4*>(Xt + i * kMaxBatch);
          float g = 0.0f;
#pragma unroll
          for (int c = 0; c < kMaxBatch / 4; ++c) {
            const float4 v = xv[c];
            g = fmaf(dz[4 * c + 0], v.x, g);
            g = fmaf(dz[4 * c + 1], v.y, g);
            g = fmaf(dz[4 * c + 2], v.z, g);
            g = fmaf(dz[4 * c + 3], v.w, g);
          }
          W[(size_t)i * a.h + j] -= lr * g;
        }
        bj -= lr * gb1;
        wj -= lr * gw2;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        float g = 0.0f;
        for (int b = 0; b < bs; ++b) g += S.dy[b];
        S.b2 -= lr * g;
      }
      __syncthreads();
    }
    // validation loss
    if (threadIdx.x == 0) S.vsum = 0.0;
    for (int st = 0; st < nval; st += kMaxBatch) {
      const int bs = min(kMaxBatch, nval - st);
      if (threadIdx.x < kMaxBatch) {
        float t = 0.0f;
        S.rows[threadIdx.x] = (int)threadIdx.x < bs ? st + (int)threadIdx.x : -1;
        if (threadIdx.x < bs) sample_row(a, f, st + threadIdx.x, true, &t);
        S.tgt[threadIdx.x] = t;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < kMaxBatch * a.m; idx += blockDim.x) {
        const int b = idx / a.m, i = idx % a.m;
        float t;
        Xt[i * kMaxBatch + b] = (b < bs) ? sample_row(a, f, st + b, true, &t)[i] : 0.0f;
      }
      __syncthreads();
      forward_batch(a, f, Xt, bs, bj, wj, own, z, S);
      if (threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < bs; ++b) {
          const double e = (double)S.y[b] - (double)S.tgt[b];
          s += e * e;
        }
        S.vsum += s;
      }
      __syncthreads();
    }
    const double vl = S.vsum / (double)nval;
    bool improved = vl < best;
    if (improved) {
      best = vl;
      bad = 0;
      if (own) {
        for (int i = 0; i < a.m; ++i) BW[(size_t)i * a.h + j] = W[(size_t)i * a.h + j];
        a.bb1[(size_t)f * a.h + j] = bj;
        a.bw2[(size_t)f * a.h + j] = wj;
      }
      if (threadIdx.x == 0) a.bb2[f] = S.b2;
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
  // restore the best-validation weights
  if (own) {
    for (int i = 0; i < a.m; ++i) W[(size_t)i * a.h + j] = BW[(size_t)i * a.h + j];
    a.b1[(size_t)f * a.h + j] = a.bb1[(size_t)f * a.h + j];
    a.w2[(size_t)f * a.h + j] = a.bw2[(size_t)f * a.h + j];
  }
  if (threadIdx.x == 0) {
    a.b2[f] = a.bb2[f];
    if (a.epochs_run) a.epochs_run[f] = ep;
    if (a.best_val) a.best_val[f] = best;
  }
}

}  // namespace

void launch_filter_forward(const float* Q, int nq, int mp, int m, int F, int h, const float* W1t,
                           const float* b1, const float* w2, const float* b2, float* out,
                           cudaStream_t s) {
  if (nq <= 0 || F <= 0) return;
  const size_t smem = (size_t)m * kQT * sizeof(float);
  if (smem > 48 * 1024)
    LF_CUDA(cudaFuncSetAttribute(filter_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  dim3 grid(F, (nq + kQT - 1) / kQT);
  filter_fwd_kernel<<<grid, kFwdThreads, smem, s>>>(Q, nq, mp, m, F, h, W1t, b1, w2, b2, out);
  LF_CHECK_LAUNCH();
}

void launch_train(const TrainArgs& a, cudaStream_t s) {
  if (a.F <= 0) return;
  if (a.batch < 1 || a.batch > kMaxBatch) fail(LEAFI_EINVAL, "batch must be in [1, %d]", kMaxBatch);
  if (a.h > 256) fail(LEAFI_EINVAL, "hidden width > 256 is not supported by the trainer");
  const int threads = ((a.h + 31) / 32) * 32;
  const size_t smem = (size_t)a.m * kMaxBatch * sizeof(float);
  LF_CUDA(cudaFuncSetAttribute(train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem));
  train_kernel<<<a.F, threads < 64 ? 64 : threads, smem, s>>>(a);
  LF_CHECK_LAUNCH();
}

}  // namespace leafi
