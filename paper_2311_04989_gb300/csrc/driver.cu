// driver.cu -- device side of the multi-block RK step: ghost exchange between same-level blocks and
// the time step on the device (the RK3 integration stated at the start of Sec. 4; the global CFL time
// step of Sec. 3.1, or a wave-speed rule).
//
//   k_ghost_cells / k_ghost_faces  every ghost cell and ghost face of every block is copied from the
//                block that the neighbour table names for its direction (or, at an outflow boundary,
//                from the nearest owned element of the same block).  Sources are always owned
//                elements, so copies never race with each other.
//   k_cfl_rate   max over interior cells and directions of max(|lambda-|, |lambda+|)/dx_d (the fast
//                speeds of Sec. 2.2 at the cell state), warp-reduced, one atomic max per warp
//   k_cfl_dt     dt = CFL / rate, left on the device for the stages to read
#include "internal.h"
#include "physics.cuh"
#include "stage_common.cuh"

namespace grs {

struct GhostArgs {
  double* W[7];
  int nw;
  double* B[3];
  const int* nbr;   // 27 entries per block
};

__device__ __forceinline__ int nbr_slot(const int o[3]) { return (o[2] + 1) * 9 + (o[1] + 1) * 3 + (o[0] + 1); }

__global__ void __launch_bounds__(kTile) k_ghost_cells(const DBlock* __restrict__ blocks, const Work* __restrict__ work,
                                                       const __grid_constant__ GhostArgs a) {
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  int p[3];
  if (!decode<R_CELLS_ALL, 0>(w, b, p)) return;
  int o[3];
  bool ghost = false;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    o[d] = p[d] < 0 ? -1 : (p[d] >= b.n[d] ? 1 : 0);
    ghost = ghost || o[d] != 0;
  }
  if (!ghost) return;
  const int src = a.nbr[27 * w.block + nbr_slot(o)];
  int q[3];
  long long cs;
  if (src >= 0) {
    const DBlock& sb = blocks[src];
#pragma unroll
    for (int d = 0; d < 3; ++d) q[d] = p[d] - o[d] * b.n[d];
    cs = sb.cell + cix(sb, q[0], q[1], q[2]);
  } else {   // outflow: nearest interior cell of this block
#pragma unroll
    for (int d = 0; d < 3; ++d) q[d] = min(max(p[d], 0), b.n[d] - 1);
    cs = b.cell + cix(b, q[0], q[1], q[2]);
  }
  const long long c = b.cell + cix(b, p[0], p[1], p[2]);
  for (int v = 0; v < a.nw; ++v) a.W[v][c] = a.W[v][cs];
}

template <int D>
__device__ __forceinline__ void ghost_face(const Work& w, const DBlock& b, const DBlock* blocks, const GhostArgs& a) {
  int p[3];
  if (!decode<R_FACES_ALL, D>(w, b, p)) return;
  // owned faces: 0..n along D, 0..n-1 across
  int o[3];
  bool ghost = false;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int own = b.n[d] + (d == D);
    o[d] = p[d] < 0 ? -1 : (p[d] >= own ? 1 : 0);
    ghost = ghost || o[d] != 0;
  }
  if (!ghost) return;
  const int src = a.nbr[27 * w.block + nbr_slot(o)];
  int q[3];
  long long fs;
  if (src >= 0) {
    const DBlock& sb = blocks[src];
#pragma unroll
    for (int d = 0; d < 3; ++d) q[d] = p[d] - o[d] * b.n[d];
    fs = sb.face[D] + fix(sb, D, q[0], q[1], q[2]);
  } else {
#pragma unroll
    for (int d = 0; d < 3; ++d) q[d] = min(max(p[d], 0), b.n[d] - (d == D ? 0 : 1));
    fs = b.face[D] + fix(b, D, q[0], q[1], q[2]);
  }
  a.B[D][b.face[D] + fix(b, D, p[0], p[1], p[2])] = a.B[D][fs];
}

__global__ void __launch_bounds__(kTile) k_ghost_faces(const DBlock* __restrict__ blocks, const Work* __restrict__ work,
                                                       const __grid_constant__ GhostArgs a) {
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  if (w.dir == 0) ghost_face<0>(w, b, blocks, a);
  else if (w.dir == 1) ghost_face<1>(w, b, blocks, a);
  else ghost_face<2>(w, b, blocks, a);
}

__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

template <int EOS>
__global__ void __launch_bounds__(kTile) k_cfl_rate(const DBlock* __restrict__ blocks, const Work* __restrict__ work,
                                                    const __grid_constant__ InView<double> in,
                                                    const __grid_constant__ KParams kp, double* rate) {
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  int p[3];
  double r = 0.0;
  if (decode<R_INTERIOR, 0>(w, b, p)) {
    const int i = p[0], j = p[1], k = p[2];
    double val[16];
    cell_metric<double>(b, in, in.order, i, j, k, 0, 10, val, nullptr);
    CellMet<double> M;
    cellmet_from<double>(val, true, M);
    const long long c = b.cell + cix(b, i, j, k);
    double wv[6], Bd[3];
    for (int v = 0; v < 5; ++v) wv[v] = in.W[v][c];
    wv[5] = EOS ? in.W[5][c] : 0.0;
    const long long f0 = b.face[0] + fix(b, 0, i, j, k), f1 = b.face[1] + fix(b, 1, i, j, k);
    const long long f2 = b.face[2] + fix(b, 2, i, j, k);
    Bd[0] = 0.5 * (in.B[0][f0] + in.B[0][f0 + 1]);
    Bd[1] = 0.5 * (in.B[1][f1] + in.B[1][f1 + b.N[0]]);
    Bd[2] = 0.5 * (in.B[2][f2] + in.B[2][f2 + (long long)b.N[0] * b.N[1]]);
    CellFluid<double> fl;
    cell_fluid<double, EOS>(M, kp, wv, Bd, fl);
    double rhoh, cs2;
    eos_rhoh_cs2<double, EOS>(kp, fl.rho, fl.p, wv[5], &rhoh, &cs2);
    // fast speeds along each direction (the expression of the face states, at the cell centre)
    const double ca2 = fl.b2 / (rhoh + fl.b2);
    const double c2 = cs2 + ca2 - cs2 * ca2;
    const double v2 = fl.v[0] * fl.vl[0] + fl.v[1] * fl.vl[1] + fl.v[2] * fl.vl[2];
    const double iden = 1.0 / (1.0 - v2 * c2);
    const double cc = sqrt(c2);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double gdd = M.gi[d == 0 ? 0 : (d == 1 ? 3 : 5)];
      double disc = (1.0 - v2) * (gdd * (1.0 - v2 * c2) - fl.v[d] * fl.v[d] * (1.0 - c2));
      disc = disc > 0.0 ? disc : 0.0;
      const double cr = cc * sqrt(disc);
      const double vc = fl.v[d] * (1.0 - c2);
      const double lp = M.alpha * (vc + cr) * iden - M.beta[d];
      const double lm = M.alpha * (vc - cr) * iden - M.beta[d];
      r = fmax(r, fmax(fabs(lp), fabs(lm)) * b.idx[d]);
    }
    if (!(r == r)) r = __longlong_as_double(0x7FF0000000000000LL);   // NaN state: no finite dt
  }
  for (int off = 16; off > 0; off >>= 1) r = fmax(r, __shfl_down_sync(0xffffffffu, r, off));
  if ((threadIdx.x & 31) == 0) atomic_max_pos(rate, r);
}

__global__ void k_set_scalar(double* dst, double v) { *dst = v; }

cudaError_t launch_set_scalar(double* dst, double value, cudaStream_t st) {
  k_set_scalar<<<1, 1, 0, st>>>(dst, value);
  return cudaGetLastError();
}

__global__ void k_cfl_dt(const double* rate, double cfl, double* dt) {
  const double r = *rate;
  *dt = r > 0.0 ? cfl / r : 0.0;
}

cudaError_t launch_ghost_fill(const DBlock* blocks, const Work* wc, int nwc, const Work* wf, int nwf, const int* nbr,
                              double* const W[7], int nw, double* const B[3], cudaStream_t st) {
  GhostArgs a{};
  for (int v = 0; v < 7; ++v) a.W[v] = v < nw ? W[v] : nullptr;
  a.nw = nw;
  for (int d = 0; d < 3; ++d) a.B[d] = B[d];
  a.nbr = nbr;
  if (nwc) k_ghost_cells<<<nwc, kTile, 0, st>>>(blocks, wc, a);
  if (nwf) k_ghost_faces<<<nwf, kTile, 0, st>>>(blocks, wf, a);
  return cudaGetLastError();
}

cudaError_t launch_cfl_dt(const DBlock* blocks, const Work* wi, int nwi, const MetricView& m,
                          const double* const W[7], const double* const B[3], const KParams& kp, double cfl,
                          double* rate, double* dt, cudaStream_t st) {
  InView<double> in;
  for (int c = 0; c < 16; ++c) in.M[c] = m.v[c];
  for (int v = 0; v < 6; ++v) in.W[v] = W[v];
  for (int d = 0; d < 3; ++d) in.B[d] = B[d];
  in.order = m.order;
  in.k_zero = m.k_zero;
  cudaError_t e = cudaMemsetAsync(rate, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  if (nwi) {
    if (kp.eos == GR_EOS_TABLE) k_cfl_rate<GR_EOS_TABLE><<<nwi, kTile, 0, st>>>(blocks, wi, in, kp, rate);
    else k_cfl_rate<GR_EOS_IDEAL><<<nwi, kTile, 0, st>>>(blocks, wi, in, kp, rate);
  }
  k_cfl_dt<<<1, 1, 0, st>>>(rate, cfl, dt);
  return cudaGetLastError();
}

}  // namespace grs
