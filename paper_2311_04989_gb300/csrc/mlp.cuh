// mlp.cuh -- the learned con2prim bracket (not in the paper: a bracket proposal for the root find of Sec. 3.5).
//
// A 6-64-64-1 tanh network maps features of the KKC invariants of a cell (and, with a table, log D~
// and Y_e) to the logarithm of the master-function root mu = 1/(hW).  Con2prim starts its bracket search there and accepts a bracket
// only where the FP64 master function changes sign.
//
// Parameter vector (float, GR_MLP_NPARAM entries, documented in include/grstage.h):
//   [0..5] feature means, [6..11] feature inverse standard deviations, [12] target mean,
//   [13] target standard deviation, [14] first bracket step delta in log mu, [15] unused,
//   [16..]  W1 (64 x 6), b1 (64), W2 (64 x 64), b2 (64), W3 (64), b3 (1), row-major (out, in).
#pragma once

#include <cuda_runtime.h>

#include "grstage.h"

namespace grs {

constexpr int kMlpH = 64, kMlpIn = 6, kMlpOff = 16;
constexpr int kMlpNW = kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH + kMlpH + kMlpH + 1;   // 4673
constexpr int kMlpN = kMlpOff + kMlpNW;                                              // 4689
constexpr int kMlpMean = 0, kMlpIStd = 6, kMlpTMean = 12, kMlpTStd = 13, kMlpStep = 14;
static_assert(kMlpN == GR_MLP_NPARAM && kMlpIn == GR_MLP_NIN, "parameter layout of include/grstage.h");
constexpr int kW1 = kMlpOff, kB1 = kW1 + kMlpH * kMlpIn, kW2 = kB1 + kMlpH, kB2 = kW2 + kMlpH * kMlpH,
              kW3 = kB2 + kMlpH, kB3 = kW3 + kMlpH;

// Features 0..3 of the KKC invariants: log(1+q), log(1+r^2), log(1+calb^2), (r.calb)^2/(r^2 calb^2)
// (features 4, 5 -- log D~ and Y_e, or 0 for the ideal gas -- are set by the caller)
__device__ __forceinline__ void c2p_features(double q, double r2, double b2, double rb, float f[kMlpIn]) {
  f[0] = (float)log1p(q);
  f[1] = (float)log1p(r2);
  f[2] = (float)log1p(b2);
  const double den = r2 * b2;
  f[3] = den > 0.0 ? (float)(rb * rb / den) : 0.f;
}

// tanh from the exponential, tanh x = 1 - 2/(exp(2x) + 1), with the fast hardware exponential and
// division: absolute error ~1e-6, enough for a bracket proposal that is verified by a sign change
// (the training kernels use the same function, so the trained network is the evaluated one)
__device__ __forceinline__ float mlp_tanh(float x) { return 1.f - __fdividef(2.f, __expf(2.f * x) + 1.f); }

// First hidden layer of a normalised input (registers; fully unrolled)
__device__ __forceinline__ void mlp_layer1(const float* __restrict__ P, const float x[kMlpIn], float h1[kMlpH]) {
  float xn[kMlpIn];
#pragma unroll
  for (int j = 0; j < kMlpIn; ++j) xn[j] = (x[j] - __ldg(P + kMlpMean + j)) * __ldg(P + kMlpIStd + j);
#pragma unroll
  for (int i = 0; i < kMlpH; ++i) {
    float a = __ldg(P + kB1 + i);
#pragma unroll
    for (int j = 0; j < kMlpIn; ++j) a = fmaf(__ldg(P + kW1 + i * kMlpIn + j), xn[j], a);
    h1[i] = mlp_tanh(a);
  }
}

// Pre-activation of second-layer unit i from h1 (row i of W2 read as float4; two partial sums so
// that the FMA chain is half as long)
__device__ __forceinline__ float mlp_row2(const float* __restrict__ P, int i, const float h1[kMlpH]) {
  const float4* row = reinterpret_cast<const float4*>(P + kW2 + i * kMlpH);
  float a = __ldg(P + kB2 + i), b = 0.f;
#pragma unroll
  for (int j4 = 0; j4 < kMlpH / 4; ++j4) {
    const float4 w = __ldg(row + j4);
    a = fmaf(w.x, h1[4 * j4 + 0], a);
    b = fmaf(w.y, h1[4 * j4 + 1], b);
    a = fmaf(w.z, h1[4 * j4 + 2], a);
    b = fmaf(w.w, h1[4 * j4 + 3], b);
  }
  return a + b;
}

// Normalised network output z (the prediction of log mu is P[12] + P[13] z).  Kept out of line so
// that the con2prim kernel carries one compact copy.
static __device__ __noinline__ float mlp_z(const float* __restrict__ P, const float x[kMlpIn]) {
  float h1[kMlpH];
  mlp_layer1(P, x, h1);
  // four second-layer units at a time: independent FMA chains for the latency to hide behind
  float z0 = __ldg(P + kB3), z1 = 0.f, z2 = 0.f, z3 = 0.f;
  for (int i = 0; i < kMlpH; i += 4) {
    const float a0 = mlp_row2(P, i, h1), a1 = mlp_row2(P, i + 1, h1);
    const float a2 = mlp_row2(P, i + 2, h1), a3 = mlp_row2(P, i + 3, h1);
    z0 = fmaf(__ldg(P + kW3 + i), mlp_tanh(a0), z0);
    z1 = fmaf(__ldg(P + kW3 + i + 1), mlp_tanh(a1), z1);
    z2 = fmaf(__ldg(P + kW3 + i + 2), mlp_tanh(a2), z2);
    z3 = fmaf(__ldg(P + kW3 + i + 3), mlp_tanh(a3), z3);
  }
  return (z0 + z1) + (z2 + z3);
}

}  // namespace grs
