// faces_core.cuh -- the flux through one face from its reconstruction stencil and face metric, shared by
// every kernel that computes face fluxes (k_faces, the tiled face sweep, the fused sweep) so that they
// agree bitwise whatever memory their stencils come from.
//   reconstruction (Sec. 3.4) of rho, u~^i, p, the two transverse cell fields [, Y_e] -> left / right
//   states (both fall back to first order where a state has rho <= 0 or p <= 0), face metric -> sqrt(gamma),
//   gamma^{dd}; face states (Eq. consB_def, Eq. fluxB_def, fast speeds of Sec. 2.2) and HLLE.
#pragma once

#include "internal.h"
#include "physics.cuh"

namespace grs {

// Reconstruction: st[v][t] holds variable v (rho, u~^x, u~^y, u~^z, p, calB^{t1}, calB^{t2}[, Y_e]) of cells
// f-3 .. f+2 along the face normal.  L, Rr: the left / right states of the face (both first order where a
// state has rho <= 0 or p <= 0).
template <class R, int EOS, int METHOD>
__device__ __forceinline__ void face_recon(R (*st)[6], const KParams& kp, R* L, R* Rr) {
  constexpr int NV = EOS ? 8 : 7;
  const R eps = (sizeof(R) == 4) ? R(1e-30f) : R(kp.weno_eps);
  // density and pressure with power-of-two scaling in FP32 (they reach the atmosphere values);
  // velocities, the transverse field and Y_e without
  recon<R, METHOD, true>(st[0], eps, &L[0], &Rr[0]);
  recon<R, METHOD, true>(st[4], eps, &L[4], &Rr[4]);
#pragma unroll
  for (int v = 1; v < NV; ++v)
    if (v != 4) recon<R, METHOD, false>(st[v], eps, &L[v], &Rr[v]);
  // a non-physical reconstructed state (rho <= 0 or p <= 0) drops the face to first order
  if (!(L[0] > R(0)) || !(Rr[0] > R(0)) || !(L[4] > R(0)) || !(Rr[4] > R(0))) {
#pragma unroll
    for (int v = 0; v < NV; ++v) { L[v] = st[v][2]; Rr[v] = st[v][3]; }
  }
}

// Flux of direction D from the reconstructed states L, Rr, the face metric met (alpha, beta^i, gamma_ij at
// the face centre) and the densitised normal field Bn.  F[0..6]: fluxes of D, S_j, tau and the two
// induction components; *ye_up (table): Y_e of the upwind state of the mass flux.
template <class R, int EOS, int D>
__device__ __forceinline__ void face_flux(const R* L, const R* Rr, const R met[10], R Bn, const KParams& kp, R F[7],
                                          R* ye_up) {
  constexpr int t1 = (D + 1) % 3, t2 = (D + 2) % 3;
  constexpr int NV = EOS ? 8 : 7;
  R wl[6], wr[6];
#pragma unroll
  for (int v = 0; v < 5; ++v) { wl[v] = L[v]; wr[v] = Rr[v]; }
  wl[5] = EOS ? L[NV - 1] : R(0);
  wr[5] = EOS ? Rr[NV - 1] : R(0);
  const R det = det3(met + 4);
  const R sg = sqrt_r(det);
  const R gdd = inv_dd(met + 4, D, det);
  R BL[3], BR[3];
  BL[D] = Bn; BR[D] = Bn;
  BL[t1] = L[5] * sg; BL[t2] = L[6] * sg;
  BR[t1] = Rr[5] * sg; BR[t2] = Rr[6] * sg;
  R UL[7], FL[7], UR[7], FR[7], lmL, lpL, lmR, lpR;
  face_state<R, EOS>(D, met, sg, gdd, kp, wl, BL, UL, FL, &lmL, &lpL);
  face_state<R, EOS>(D, met, sg, gdd, kp, wr, BR, UR, FR, &lmR, &lpR);
  hlle<R>(UL, UR, FL, FR, lmL, lpL, lmR, lpR, F);
  if constexpr (EOS == GR_EOS_TABLE) *ye_up = F[0] > R(0) ? wl[5] : wr[5];
  else *ye_up = R(0);
}

}  // namespace grs
