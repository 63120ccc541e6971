// mlp.cu -- training and evaluation kernels of the learned con2prim bracket (see mlp.cuh).
//
// Training minimises the mean of (z - zt)^2 / 2 over samples, z the network output and
// zt = (log mu - P[12]) / P[13] the normalised target, with Adam.  One mini-batch is two launches:
//   k_mlp_grad_partial  one CTA per 128 samples: forward, backward, and that CTA's sum of the
//                       per-sample gradients (reduced over its samples in shared memory)
//   k_mlp_reduce_adam   one thread per parameter: sum of the CTA partials in a fixed order
//                       (deterministic), then the Adam update in place
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "internal.h"
#include "mlp.cuh"

namespace grs {
namespace {

constexpr int kS = 128;   // samples (threads) per CTA

struct GradSmem {
  float H1[kS][kMlpH];
  float H2[kS][kMlpH];
  float G1[kS][kMlpH];
  float G2[kS][kMlpH];
  float X[kS][kMlpIn];
  float dz[kS];
  float loss[kS / 32];
};

__global__ void __launch_bounds__(kS) k_mlp_forward(const float* __restrict__ P, const float* __restrict__ x,
                                                   long long n, float* __restrict__ t) {
  const long long e = blockIdx.x * (long long)kS + threadIdx.x;
  if (e >= n) return;
  float xe[kMlpIn];
#pragma unroll
  for (int j = 0; j < kMlpIn; ++j) xe[j] = x[kMlpIn * e + j];
  t[e] = P[kMlpTMean] + P[kMlpTStd] * mlp_z(P, xe);
}

__global__ void __launch_bounds__(kS) k_mlp_grad_partial(const float* __restrict__ P, const float* __restrict__ x,
                                                        const float* __restrict__ t, long long n0, long long nb,
                                                        float inv_n, float* __restrict__ partial,
                                                        float* __restrict__ loss_partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GradSmem& S = *reinterpret_cast<GradSmem*>(smem_raw);
  const int s = threadIdx.x;
  const long long e = blockIdx.x * (long long)kS + s;
  const bool valid = e < nb;
  float h1[kMlpH];
  float xn[kMlpIn];
#pragma unroll
  for (int j = 0; j < kMlpIn; ++j) xn[j] = 0.f;
  float dz = 0.f, loss = 0.f;
  if (valid) {
    float xe[kMlpIn];
#pragma unroll
    for (int j = 0; j < kMlpIn; ++j) xe[j] = x[kMlpIn * (n0 + e) + j];
#pragma unroll
    for (int j = 0; j < kMlpIn; ++j) xn[j] = (xe[j] - P[kMlpMean + j]) * P[kMlpIStd + j];
    mlp_layer1(P, xe, h1);
    float z = P[kB3];
    for (int i = 0; i < kMlpH; ++i) {
      const float h2 = mlp_tanh(mlp_row2(P, i, h1));
      S.H2[s][i] = h2;
      z = fmaf(P[kW3 + i], h2, z);
    }
    const float zt = (t[n0 + e] - P[kMlpTMean]) / P[kMlpTStd];
    dz = (z - zt) * inv_n;
    loss = 0.5f * (z - zt) * (z - zt) * inv_n;
  } else {
#pragma unroll
    for (int i = 0; i < kMlpH; ++i) h1[i] = 0.f;
    for (int i = 0; i < kMlpH; ++i) S.H2[s][i] = 0.f;
  }
  // backward: g2 = dz W3 (1 - h2^2), g1 = W2^T g2 (1 - h1^2)
  float g1[kMlpH];
#pragma unroll
  for (int j = 0; j < kMlpH; ++j) g1[j] = 0.f;
  for (int i = 0; i < kMlpH; ++i) {
    const float h2 = S.H2[s][i];
    const float g2 = dz * P[kW3 + i] * (1.f - h2 * h2);
    S.G2[s][i] = g2;
    const float4* row = reinterpret_cast<const float4*>(P + kW2 + i * kMlpH);
#pragma unroll
    for (int j4 = 0; j4 < kMlpH / 4; ++j4) {
      const float4 w = __ldg(row + j4);
      g1[4 * j4 + 0] = fmaf(w.x, g2, g1[4 * j4 + 0]);
      g1[4 * j4 + 1] = fmaf(w.y, g2, g1[4 * j4 + 1]);
      g1[4 * j4 + 2] = fmaf(w.z, g2, g1[4 * j4 + 2]);
      g1[4 * j4 + 3] = fmaf(w.w, g2, g1[4 * j4 + 3]);
    }
  }
#pragma unroll
  for (int j = 0; j < kMlpH; ++j) {
    S.H1[s][j] = h1[j];
    S.G1[s][j] = g1[j] * (1.f - h1[j] * h1[j]);
  }
#pragma unroll
  for (int j = 0; j < kMlpIn; ++j) S.X[s][j] = xn[j];
  S.dz[s] = dz;
  for (int o = 16; o > 0; o >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, o);
  if ((s & 31) == 0) S.loss[s >> 5] = loss;
  __syncthreads();
  // this CTA's gradient: sums over its samples, one output per thread and stride
  float* out = partial + (long long)blockIdx.x * kMlpNW;
  for (int k = s; k < kMlpNW; k += kS) {
    float acc = 0.f;
    if (k < kB1 - kMlpOff) {                         // W1 (64 x kMlpIn)
      const int i = k / kMlpIn, j = k % kMlpIn;
      for (int q = 0; q < kS; ++q) acc = fmaf(S.G1[q][i], S.X[q][j], acc);
    } else if (k < kW2 - kMlpOff) {                  // b1
      const int i = k - (kB1 - kMlpOff);
      for (int q = 0; q < kS; ++q) acc += S.G1[q][i];
    } else if (k < kB2 - kMlpOff) {                  // W2 (64 x 64)
      const int kk = k - (kW2 - kMlpOff), i = kk / kMlpH, j = kk % kMlpH;
      for (int q = 0; q < kS; ++q) acc = fmaf(S.G2[q][i], S.H1[q][j], acc);
    } else if (k < kW3 - kMlpOff) {                  // b2
      const int i = k - (kB2 - kMlpOff);
      for (int q = 0; q < kS; ++q) acc += S.G2[q][i];
    } else if (k < kB3 - kMlpOff) {                  // W3
      const int i = k - (kW3 - kMlpOff);
      for (int q = 0; q < kS; ++q) acc = fmaf(S.dz[q], S.H2[q][i], acc);
    } else {                                         // b3
      for (int q = 0; q < kS; ++q) acc += S.dz[q];
    }
    out[k] = acc;
  }
  if (s == 0) {
    float l = 0.f;
    for (int w = 0; w < kS / 32; ++w) l += S.loss[w];
    loss_partial[blockIdx.x] = l;
  }
}

struct AdamArgs {
  float lr, beta1, beta2, eps;
  float bc1, bc2;     // 1 - beta^step
  int nblk;
  int apply;          // 0: only write the summed gradient
};

__global__ void __launch_bounds__(256) k_mlp_reduce_adam(const float* __restrict__ partial,
                                                        const float* __restrict__ loss_partial, float* P,
                                                        float* m, float* v, float* grad_out, float* loss_acc,
                                                        float loss_weight, AdamArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0 && loss_acc) {
    float l = 0.f;
    for (int b = 0; b < a.nblk; ++b) l += loss_partial[b];
    *loss_acc += loss_weight * l;
  }
  if (k >= kMlpNW) return;
  float g = 0.f;
  for (int b = 0; b < a.nblk; ++b) g += partial[(long long)b * kMlpNW + k];
  if (grad_out) grad_out[k] = g;
  if (!a.apply) return;
  const float mk = a.beta1 * m[k] + (1.f - a.beta1) * g;
  const float vk = a.beta2 * v[k] + (1.f - a.beta2) * g * g;
  m[k] = mk;
  v[k] = vk;
  P[kMlpOff + k] -= a.lr * (mk / a.bc1) / (sqrtf(vk / a.bc2) + a.eps);
}

thread_local std::string g_mlp_error;

int mfail(int code, const std::string& msg) {
  g_mlp_error = msg;
  return code;
}

int mcuda(cudaError_t e, const char* where) {
  return mfail(GR_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

cudaError_t grad_launch(const float* P, const float* x, const float* t, long long n0, long long nb, float* partial,
                        float* loss_partial, cudaStream_t st) {
  const int nblk = (int)((nb + kS - 1) / kS);
  cudaError_t e = cudaFuncSetAttribute(k_mlp_grad_partial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(GradSmem));   // per device, cheap to repeat
  if (e != cudaSuccess) return e;
  k_mlp_grad_partial<<<nblk, kS, sizeof(GradSmem), st>>>(P, x, t, n0, nb, 1.f / (float)nb, partial, loss_partial);
  return cudaGetLastError();
}

}  // namespace
}  // namespace grs

using namespace grs;

extern "C" {

int gr_mlp_nparam(void) { return kMlpN; }

const char* gr_mlp_last_error(void) { return g_mlp_error.c_str(); }

int gr_mlp_forward(const float* P, const float* x, int64_t n, float* t, void* stream) {
  if (!P || !x || !t || n < 0) return mfail(GR_EINVAL, "gr_mlp_forward: bad argument");
  if (((uintptr_t)P) & 15u) return mfail(GR_EINVAL, "gr_mlp_forward: parameters must be 16-byte aligned");
  if (n == 0) return GR_OK;
  k_mlp_forward<<<(unsigned)((n + kS - 1) / kS), kS, 0, (cudaStream_t)stream>>>(P, x, n, t);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GR_OK : mcuda(e, "gr_mlp_forward");
}

int gr_mlp_grad(const float* P, const float* x, const float* t, int64_t n, float* grad, float* loss, void* stream) {
  if (!P || !x || !t || !grad || !loss || n < 1) return mfail(GR_EINVAL, "gr_mlp_grad: bad argument");
  if (((uintptr_t)P) & 15u) return mfail(GR_EINVAL, "gr_mlp_grad: parameters must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  const int nblk = (int)((n + kS - 1) / kS);
  float *partial = nullptr, *lp = nullptr;
  cudaError_t e = cudaMalloc(&partial, sizeof(float) * (size_t)nblk * kMlpNW);
  if (e == cudaSuccess) e = cudaMalloc(&lp, sizeof(float) * nblk);
  if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float), st);
  if (e == cudaSuccess) e = grad_launch(P, x, t, 0, n, partial, lp, st);
  if (e == cudaSuccess) {
    AdamArgs a{};
    a.nblk = nblk;
    a.apply = 0;
    k_mlp_reduce_adam<<<(kMlpNW + 255) / 256, 256, 0, st>>>(partial, lp, nullptr, nullptr, nullptr, grad, loss, 1.f, a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(partial);
  cudaFree(lp);
  return e == cudaSuccess ? GR_OK : mcuda(e, "gr_mlp_grad");
}

int gr_mlp_train(float* P, const float* x, const float* t, int64_t n, int32_t epochs, int32_t batch, float lr,
                 float* losses, void* stream) {
  if (!P || !x || !t || n < 1 || epochs < 1 || batch < 1 || !(lr > 0.f))
    return mfail(GR_EINVAL, "gr_mlp_train: bad argument");
  if (((uintptr_t)P) & 15u) return mfail(GR_EINVAL, "gr_mlp_train: parameters must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  const long long bsz = std::min<long long>(batch, n);
  const int nblk_max = (int)((bsz + kS - 1) / kS);
  float *partial = nullptr, *lp = nullptr, *mv = nullptr, *dloss = nullptr;
  cudaError_t e = cudaMalloc(&partial, sizeof(float) * (size_t)nblk_max * kMlpNW);
  if (e == cudaSuccess) e = cudaMalloc(&lp, sizeof(float) * nblk_max);
  if (e == cudaSuccess) e = cudaMalloc(&mv, sizeof(float) * 2 * kMlpNW);
  if (e == cudaSuccess) e = cudaMalloc(&dloss, sizeof(float) * epochs);
  if (e == cudaSuccess) e = cudaMemsetAsync(mv, 0, sizeof(float) * 2 * kMlpNW, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dloss, 0, sizeof(float) * epochs, st);
  long long step = 0;
  const float b1 = 0.9f, b2 = 0.999f;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    for (long long n0 = 0; n0 < n && e == cudaSuccess; n0 += bsz) {
      const long long nb = std::min<long long>(bsz, n - n0);
      e = grad_launch(P, x, t, n0, nb, partial, lp, st);
      if (e != cudaSuccess) break;
      ++step;
      AdamArgs a;
      a.lr = lr; a.beta1 = b1; a.beta2 = b2; a.eps = 1e-8f;
      a.bc1 = 1.f - (float)std::pow((double)b1, (double)step);
      a.bc2 = 1.f - (float)std::pow((double)b2, (double)step);
      a.nblk = (int)((nb + kS - 1) / kS);
      a.apply = 1;
      k_mlp_reduce_adam<<<(kMlpNW + 255) / 256, 256, 0, st>>>(partial, lp, P, mv, mv + kMlpNW, nullptr, dloss + ep,
                                                              (float)nb / (float)n, a);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess && losses) e = cudaMemcpyAsync(losses, dloss, sizeof(float) * epochs, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(partial);
  cudaFree(lp);
  cudaFree(mv);
  cudaFree(dloss);
  return e == cudaSuccess ? GR_OK : mcuda(e, "gr_mlp_train");
}

}  // extern "C"
