// peaks.cu -- arithmetic-pipe throughput loops (measurement only; not part of the stage).
//
// The roofline of an ALU-bound kernel divides its counted operations by the GPU's peak rate of the
// pipe that runs them.  These kernels measure those peaks on the GPU at hand: every thread runs kChains
// independent chains of fused multiply-adds (so that issue, not latency, limits them) for `iters`
// rounds, on one of three pipes:
//   kind 0  FP32 FFMA              2 flops per instruction and lane
//   kind 1  packed FP32x2 FFMA2    4 flops per instruction and lane (two FMAs)
//   kind 2  FP64 DFMA              2 flops per instruction and lane
// The chains contract towards a fixed point (x <- a x + c with |a| < 1), so the values stay finite and
// normal; the result is stored only when it equals a value it never reaches, so the loop cannot be
// removed as dead code and no memory traffic enters the timing.
#include <cuda_runtime.h>

#include "internal.h"

namespace grs {

constexpr int kChains = 16;

template <int KIND>
__global__ void __launch_bounds__(256) k_peak(long long iters, float seed, float* sink) {
  const float t = seed + 1e-7f * (float)threadIdx.x;
  if constexpr (KIND == 0) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = t + (float)c;
    const float a = 0.999f, b = 1e-3f;
#pragma unroll 4
    for (long long i = 0; i < iters; ++i)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fmaf(a, x[c], b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.0f) sink[blockIdx.x] = s;
  } else if constexpr (KIND == 1) {
    float2 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2(t + (float)c, t - (float)c);
    const float2 a = make_float2(0.999f, 0.998f), b = make_float2(1e-3f, 2e-3f);
#pragma unroll 4
    for (long long i = 0; i < iters; ++i)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(a, x[c], b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    if (s == -1.0f) sink[blockIdx.x] = s;
  } else {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (double)t + (double)c;
    const double a = 0.999, b = 1e-3;
#pragma unroll 4
    for (long long i = 0; i < iters; ++i)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(a, x[c], b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.0) sink[blockIdx.x] = (float)s;
  }
}

}  // namespace grs

extern "C" int gr_peak_alu(int32_t kind, int32_t blocks, int32_t threads, int64_t iters, float* sink,
                           double* flops, void* stream) {
  using namespace grs;
  if (kind < 0 || kind > 2 || blocks < 1 || threads < 32 || threads > 256 || (threads & 31) || iters < 1 || !sink ||
      !flops)
    return GR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const float seed = 0.5f;
  if (kind == 0) k_peak<0><<<blocks, threads, 0, st>>>(iters, seed, sink);
  else if (kind == 1) k_peak<1><<<blocks, threads, 0, st>>>(iters, seed, sink);
  else k_peak<2><<<blocks, threads, 0, st>>>(iters, seed, sink);
  if (cudaGetLastError() != cudaSuccess) return GR_ECUDA;
  *flops = (double)blocks * threads * (double)iters * kChains * (kind == 1 ? 4.0 : 2.0);
  return GR_OK;
}
