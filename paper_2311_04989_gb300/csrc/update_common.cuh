// update_common.cuh -- the per-cell end of a stage shared by the separate kernels (stage_kernels.cu)
// and the fused sweep (fused.cu), so that both form U', the atmosphere test and the reset with the
// same operations in the same order (their results agree bitwise):
//   accumulate_vals   U' = g1 U + g0 U0 + beta dt (src - div F) from the six face fluxes of a cell,
//                     the fluxes widened exactly and the sum accumulated in FP64 (Eq. claw)
//   cell_sources_at   the geometric sources of a cell in R (Eq. hydsrc_def) from the stage-input metric
//                     (values and derivatives of its vertex interpolant), primitives and face field
//   mixed_atm_reset   the mixed path's atmosphere reset of a cell whose D' fell below the threshold
//                     (Sec. 3.5): D, tau of the atmosphere with the cell field of the updated faces
#pragma once

#include "internal.h"
#include "physics.cuh"
#include "stage_common.cuh"

namespace grs {

__device__ __forceinline__ void cell_field(const DBlock& b, const double* const* B, int i, int j, int k,
                                           double Bd[3]) {
  const long long f0 = b.face[0] + fix(b, 0, i, j, k);
  const long long f1 = b.face[1] + fix(b, 1, i, j, k);
  const long long f2 = b.face[2] + fix(b, 2, i, j, k);
  Bd[0] = 0.5 * (B[0][f0] + B[0][f0 + 1]);
  Bd[1] = 0.5 * (B[1][f1] + B[1][f1 + b.N[0]]);
  Bd[2] = 0.5 * (B[2][f2] + B[2][f2 + (long long)b.N[0] * b.N[1]]);
}

template <int EOS>
__device__ __forceinline__ void write_cell(const StateView& s, long long c, const double q[6], const double w[7],
                                           int st) {
  constexpr int NQ = EOS ? 6 : 5, NW = EOS ? 7 : 5, N32 = EOS ? 6 : 5;
#pragma unroll
  for (int v = 0; v < NQ; ++v) s.Uo[v][c] = q[v];
#pragma unroll
  for (int v = 0; v < NW; ++v) s.Wo[v][c] = w[v];
  if (s.Wo32[0]) {   // FP32 copies of the new primitives (the next stage's reconstruction input)
#pragma unroll
    for (int v = 0; v < N32; ++v) s.Wo32[v][c] = d2f_rn(w[v]);
  }
  if (s.status) s.status[c] = (uint8_t)st;   // optional for gr_con2prim
}

// Conserved variable v of interior cell c after the stage from its source and the fluxes through its six
// faces (low / high x, y, z), in the flux precision R.
template <class R>
__device__ __forceinline__ double accumulate_vals(const DBlock& b, const StateView& s, const KParams& kp, long long c,
                                                  int v, R src, R x0, R x1, R y0, R y1, R z0, R z1) {
  const double bdt = stage_bdt(kp);
  const double U = s.U[v][c];
  double u = fma(bdt, to64(src), (kp.rk_form & RK_G1) ? kp.rk_g1 * U : U);
  u -= (bdt * b.idx[0]) * diff64(x1, x0);
  u -= (bdt * b.idx[1]) * diff64(y1, y0);
  u -= (bdt * b.idx[2]) * diff64(z1, z0);
  if (kp.rk_form & RK_G0) u += kp.rk_g0 * s.U0[v][c];
  return u;
}

// Geometric sources src[0..5] of interior cell (i, j, k) (none for D and D Y_e) in R from the stage-input
// metric (vertex interpolant: values and first derivatives), primitives and mean densitised face field;
// M: the cell metric, for the caller.
template <class R, int EOS>
__device__ __forceinline__ void cell_sources_at(const DBlock& b, const InView<R>& in, const KParams& kp, int i, int j,
                                                int k, long long c, R src[6], CellMet<R>& M) {
  const bool kzero = in.k_zero != 0;
  R val[16], dm[3][10];
  cell_metric<R>(b, in, in.order, i, j, k, 0, 10, val, dm);
  if (!kzero) cell_metric<R>(b, in, in.order, i, j, k, 10, 16, val, nullptr);
  cellmet_from<R>(val, kzero, M);
  R wv[6], Bd[3];
#pragma unroll
  for (int v = 0; v < 5; ++v) wv[v] = in.W[v][c];
  wv[5] = EOS ? in.W[5][c] : R(0);
  const long long f0 = b.face[0] + fix(b, 0, i, j, k), f1 = b.face[1] + fix(b, 1, i, j, k);
  const long long f2 = b.face[2] + fix(b, 2, i, j, k);
  Bd[0] = R(0.5) * (in.B[0][f0] + in.B[0][f0 + 1]);
  Bd[1] = R(0.5) * (in.B[1][f1] + in.B[1][f1 + b.N[0]]);
  Bd[2] = R(0.5) * (in.B[2][f2] + in.B[2][f2 + (long long)b.N[0] * b.N[1]]);
  CellFluid<R> fl;
  cell_fluid<R, EOS>(M, kp, wv, Bd, fl);
  cell_sources<R>(M, fl, dm, kzero, src);
  src[5] = R(0);   // D Y_e has no source (Sec. 2.2.1)
}

// Mixed path: the cell's D' is below the atmosphere threshold (tested against the FP32 sqrt(gamma) sg of
// the cell metric gam).  Reset to the atmosphere (Sec. 3.5) with the FP32 cell field of the updated faces
// (only calB^2 enters); status failed instead when `finite` is false (a non-finite update of another
// variable).
template <class R, int EOS>
__device__ __forceinline__ void mixed_atm_reset(const DBlock& b, const StateView& s, const KParams& kp, int i, int j,
                                                int k, long long c, const R gam[6], R sg, bool finite) {
  double q[6], wn[7];
  const double sg32 = to64(sg);
  R Bf[3], Bl[3];
  {
    const long long f0 = b.face[0] + fix(b, 0, i, j, k), f1 = b.face[1] + fix(b, 1, i, j, k);
    const long long f2 = b.face[2] + fix(b, 2, i, j, k);
    const long long oy = b.N[0], oz = (long long)b.N[0] * b.N[1];
    if (s.Bo32[0]) {   // the FP32 copies the CT update wrote: the same values as converting Bo here
      Bf[0] = R(0.5) * (R(s.Bo32[0][f0]) + R(s.Bo32[0][f0 + 1]));
      Bf[1] = R(0.5) * (R(s.Bo32[1][f1]) + R(s.Bo32[1][f1 + oy]));
      Bf[2] = R(0.5) * (R(s.Bo32[2][f2]) + R(s.Bo32[2][f2 + oz]));
    } else {
      Bf[0] = R(0.5) * (R(d2f_rn(s.Bo[0][f0])) + R(d2f_rn(s.Bo[0][f0 + 1])));
      Bf[1] = R(0.5) * (R(d2f_rn(s.Bo[1][f1])) + R(d2f_rn(s.Bo[1][f1 + oy])));
      Bf[2] = R(0.5) * (R(d2f_rn(s.Bo[2][f2])) + R(d2f_rn(s.Bo[2][f2 + oz])));
    }
  }
  lower3(gam, Bf, Bl);
  const R BBd = Bf[0] * Bl[0] + Bf[1] * Bl[1] + Bf[2] * Bl[2];
  q[0] = sg32 * kp.rho_atm;
  q[1] = q[2] = q[3] = 0.0;
  q[4] = sg32 * kp.eint_atm + to64(R(0.5) * rdiv(BBd, sg));
  q[5] = 0.0;
  wn[0] = kp.rho_atm;
  wn[1] = wn[2] = wn[3] = 0.0;
  wn[4] = kp.p_atm;
  wn[5] = wn[6] = 0.0;
  if constexpr (EOS == GR_EOS_TABLE) {
    q[5] = q[0] * kp.Ye_atm;
    wn[5] = kp.Ye_atm;
    wn[6] = kp.T_atm;
  }
  write_cell<EOS>(s, c, q, wn, finite ? GR_ST_ATM_THRESHOLD : GR_ST_FAILED);
}

}  // namespace grs
