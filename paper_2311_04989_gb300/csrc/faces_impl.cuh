// faces_impl.cuh -- k_faces: reconstruction (Sec. 3.4) + face metric (Sec. 3.2) + HLLE flux
// (Eq. fluxB_def) on every face with normal index 0..n and transverse index -1..n; with a tabulated EOS
// (Sec. 2.2.1) also Y_e and the D Y_e flux = D flux x upwind Y_e.  Instantiated per precision (one
// translation unit each: faces_f32.cu, faces_f64.cu), EOS and reconstruction method, so each kernel
// carries the code of one method only.
#pragma once

#include "faces_core.cuh"
#include "internal.h"
#include "physics.cuh"
#include "stage_common.cuh"

namespace grs {

// ------------------------------------------------------------------------------------------------
// k_faces<R>
// ------------------------------------------------------------------------------------------------
template <class R, int EOS, int METHOD, int D>
__device__ __forceinline__ void face_body(const Work& w, const DBlock& b, const InView<R>& in,
                                          const Workspace& ws, const KParams& kp) {
  int p[3];
  if (!decode<R_FACES, D>(w, b, p)) return;
  constexpr int t1 = (D + 1) % 3, t2 = (D + 2) % 3;
  constexpr int NV = EOS ? 8 : 7;   // rho, u~^i, p, calB^{t1}, calB^{t2}[, Y_e]
  // stencil cells p[D]-3 .. p[D]+2 along D; 32-bit offsets within the block, one base pointer per pool
  const int stride = D == 0 ? 1 : (D == 1 ? b.N[0] : b.N[0] * b.N[1]);
  int q[3] = {p[0], p[1], p[2]};
  q[D] -= 3;
  const int c0 = ((q[2] + b.g) * b.N[1] + (q[1] + b.g)) * b.N[0] + (q[0] + b.g);
  R st[NV][6];
  const bool wide = (b.g >= 3 || METHOD != GR_RECON_PLM);
  const R* bc1 = reinterpret_cast<const R*>(ws.bcc[t1]) + b.wcell;
  const R* bc2 = reinterpret_cast<const R*>(ws.bcc[t2]) + b.wcell;
  const R* wp[6];
#pragma unroll
  for (int v = 0; v < 6; ++v) wp[v] = (v < 5 || EOS) ? in.W[v] + b.cell : nullptr;
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    if (!wide && (t == 0 || t == 5)) {
#pragma unroll
      for (int v = 0; v < NV; ++v) st[v][t] = R(0);
      continue;
    }
    const int c = c0 + t * stride;
#pragma unroll
    for (int v = 0; v < 5; ++v) st[v][t] = wp[v][c];
    st[5][t] = bc1[c];
    st[6][t] = bc2[c];
    if constexpr (EOS == GR_EOS_TABLE) st[7][t] = wp[5][c];
  }
  R L[NV], Rr[NV];
  face_recon<R, EOS, METHOD>(st, kp, L, Rr);
  R met[10];
  face_metric<R>(b, in, in.order, D, p, met);
  const long long fi = fix(b, D, p[0], p[1], p[2]);
  const R Bn = in.B[D][b.face[D] + fi];
  R F[7], ye_up;
  face_flux<R, EOS, D>(L, Rr, met, Bn, kp, F, &ye_up);
  R* out = reinterpret_cast<R*>(ws.flux[D]);
  const long long o = b.wface[D] + fi;
#pragma unroll
  for (int v = 0; v < 7; ++v) out[v * ws.fstride[D] + o] = F[v];
  // D Y_e: the D equation times Y_e (Sec. 2.2.1), Y_e taken from the upwind state of the mass flux
  if constexpr (EOS == GR_EOS_TABLE) out[7 * ws.fstride[D] + o] = F[0] * ye_up;
  if constexpr (sizeof(R) == sizeof(float)) {   // the block's flux flag (NaN and inf fail the test too)
    R a = fabs(F[1]) + fabs(F[2]) + fabs(F[3]) + fabs(F[4]);
    if constexpr (EOS == GR_EOS_TABLE) a += fabs(F[0] * ye_up);
    if (!(a < kFluxSafe)) ws.fbad[w.block] = 1;
  }
}

// FP32: at most 72 registers, so that 14 CTAs of 64 threads (the autotuned shape) fit on an SM: 28
// warps instead of 24 at the ~80 the kernel would take, for 16-44 spilled bytes (measured on the two-star
// workload: 3.60 ms at 80 registers, 3.47 ms at 72, 3.55 ms at 68); with a table, whose face physics
// holds more, 80.  FP64: 168, about what the compiler takes for it unconstrained (166)
template <class R, int EOS, int METHOD>
__global__ void __maxnreg__(sizeof(R) == sizeof(float) ? (EOS == GR_EOS_TABLE ? 80 : 72) : 168) k_faces(const DBlock* __restrict__ blocks, const Work* __restrict__ work,
                                                    int nwork, const __grid_constant__ InView<R> in,
                                                    const __grid_constant__ Workspace ws,
                                                    const __grid_constant__ KParams kp) {
  for (int it = blockIdx.x; it < nwork; it += gridDim.x) {
    const Work w = work[it];
    const DBlock b = blocks[w.block];
    if (w.dir == 0) face_body<R, EOS, METHOD, 0>(w, b, in, ws, kp);
    else if (w.dir == 1) face_body<R, EOS, METHOD, 1>(w, b, in, ws, kp);
    else face_body<R, EOS, METHOD, 2>(w, b, in, ws, kp);
  }
}


template <class R, int EOS, int METHOD>
static cudaError_t launch_faces_m(const KLaunch& f, const DBlock* blocks, const InView<R>& in, const Workspace& ws,
                                  const KParams& kp, cudaStream_t st) {
  k_faces<R, EOS, METHOD><<<stage_grid(k_faces<R, EOS, METHOD>, f, 0), f.threads, 0, st>>>(blocks, f.work, f.nwork,
                                                                                          in, ws, kp);
  return cudaGetLastError();
}

template <class R, int EOS>
static cudaError_t launch_faces_e(const KLaunch& f, const DBlock* blocks, const InView<R>& in, const Workspace& ws,
                                  const KParams& kp, cudaStream_t st) {
  switch (kp.recon) {
    case GR_RECON_PLM: return launch_faces_m<R, EOS, GR_RECON_PLM>(f, blocks, in, ws, kp, st);
    case GR_RECON_WENO5: return launch_faces_m<R, EOS, GR_RECON_WENO5>(f, blocks, in, ws, kp, st);
    case GR_RECON_PPM: return launch_faces_m<R, EOS, GR_RECON_PPM>(f, blocks, in, ws, kp, st);
    default: return launch_faces_m<R, EOS, GR_RECON_WENOZ>(f, blocks, in, ws, kp, st);
  }
}

}  // namespace grs

#define GRS_DEFINE_LAUNCH_FACES(R)                                                                        \
  namespace grs {                                                                                        \
  cudaError_t launch_faces(const KLaunch& f, const DBlock* blocks, const InView<R>& in, const Workspace& ws, \
                           const KParams& kp, cudaStream_t st) {                                        \
    return kp.eos == GR_EOS_TABLE ? launch_faces_e<R, GR_EOS_TABLE>(f, blocks, in, ws, kp, st)           \
                                  : launch_faces_e<R, GR_EOS_IDEAL>(f, blocks, in, ws, kp, st);          \
  }                                                                                                      \
  }
