// stage_common.cuh -- work-item decoding and launch-grid helpers shared by the stage kernels
// translation units (stage_kernels.cu, faces_f32.cu, faces_f64.cu).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace grs {

// beta dt of a stage: from the host, or from the device when the RK driver reduced dt there
__device__ __forceinline__ double stage_bdt(const KParams& kp) {
  return kp.dt_dev ? kp.rk_beta * __ldg(kp.dt_dev) : kp.bdt;
}

// ------------------------------------------------------------------------------------------------
// region decoding
// ------------------------------------------------------------------------------------------------
template <int KIND, int DIR>
__device__ __forceinline__ bool decode(const Work& w, const DBlock& b, int p[3]) {
  int lo[3], cnt[3], k[3];   // k: which of n, n + 1, n + 2, N the count is (its entry of b.mdiv)
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (KIND == R_CELLS_ALL) { lo[a] = -b.g; k[a] = 3; }
    else if (KIND == R_FACES) { lo[a] = (a == DIR) ? 0 : -1; k[a] = (a == DIR) ? 1 : 2; }
    else if (KIND == R_EDGES) { lo[a] = 0; k[a] = (a == DIR) ? 0 : 1; }
    else if (KIND == R_CTFACES) { lo[a] = 0; k[a] = (a == DIR) ? 1 : 0; }
    else { lo[a] = 0; k[a] = 0; }
    cnt[a] = k[a] == 3 ? b.N[a] : b.n[a] + k[a];
  }
  const int e = w.start + threadIdx.x;
  if (e >= cnt[0] * cnt[1] * cnt[2]) return false;
  const unsigned q0 = udiv_m((unsigned)e, b.mdiv[0][k[0]]);
  const unsigned q1 = udiv_m(q0, b.mdiv[1][k[1]]);
  p[0] = lo[0] + (e - (int)q0 * cnt[0]);
  p[1] = lo[1] + ((int)q0 - (int)q1 * cnt[1]);
  p[2] = lo[2] + (int)q1;
  return true;
}

template <int D>
__device__ __forceinline__ long long face_stride(const DBlock& b, int of_dir) {
  // element stride of one step along direction of_dir in the D-face layout
  return of_dir == 0 ? 1 : (of_dir == 1 ? (long long)(b.N[0] + (D == 0)) : (long long)(b.N[0] + (D == 0)) * (b.N[1] + (D == 1)));
}

__device__ __forceinline__ long long cell_stride(const DBlock& b, int dir) {
  return dir == 0 ? 1 : (dir == 1 ? (long long)b.N[0] : (long long)b.N[0] * b.N[1]);
}


// Grid of a stage-kernel launch: one CTA per work item, or (persistent) the number of CTAs that are
// resident at once on the device, capped by the number of work items.
template <class K>
inline int stage_grid(K kernel, const KLaunch& l, size_t smem) {
  if (!l.persistent) return l.nwork;
  int dev = 0, nsm = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, l.threads, smem);
  const long long g = (long long)nsm * (occ > 0 ? occ : 1);
  return (int)(g < l.nwork ? g : l.nwork);
}

}  // namespace grs
