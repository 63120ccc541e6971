// stage_kernels.cu -- the GRMHD stage as five kernels per call (sm_103a).
//
//   k_cellprep   cell-centred field calB^i = mean of faces / sqrt(gamma) on all cells, and the
//                cell electric field E_m = alpha (v~^b B^a - v~^a B^b) on the ring -1..n  (Sec. 3.3)
//   k_faces<R>   reconstruction (Sec. 3.4) + face metric (Sec. 3.2) + HLLE flux (Eq. fluxB_def)
//                on every face with normal index 0..n and transverse index -1..n
//   k_edges<R>   upwinded corner electric field from the four adjacent face fluxes (Sec. 3.3)
//   k_ct         constrained-transport face update B' = g0 B0 + g1 B - beta dt curl E
//   k_update     flux divergence + geometric sources (Eq. claw, Eq. hydsrc_def), FP64
//                accumulation, then con2prim with atmosphere on the updated state (Sec. 3.5)
//
// Every kernel takes one work item (block, direction, first element) per CTA; blocks of different
// sizes share one launch.  Face fluxes and corner fields pass through the mesh's workspace.
#include <cstdio>

#include "internal.h"
#include "physics.cuh"

namespace grs {

// ------------------------------------------------------------------------------------------------
// region decoding
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void region(int kind, int dir, const DBlock& b, int lo[3], int cnt[3]) {
  for (int a = 0; a < 3; ++a) {
    switch (kind) {
      case R_CELLS_ALL: lo[a] = -b.g; cnt[a] = b.N[a]; break;
      case R_FACES: lo[a] = (a == dir) ? 0 : -1; cnt[a] = (a == dir) ? b.n[a] + 1 : b.n[a] + 2; break;
      case R_EDGES: lo[a] = 0; cnt[a] = (a == dir) ? b.n[a] : b.n[a] + 1; break;
      case R_CTFACES: lo[a] = 0; cnt[a] = (a == dir) ? b.n[a] + 1 : b.n[a]; break;
      default: lo[a] = 0; cnt[a] = b.n[a]; break;
    }
  }
}

// element index of this thread -> (i,j,k); false when past the region's end
__device__ __forceinline__ bool decode(int kind, const Work& w, const DBlock& b, int p[3]) {
  int lo[3], cnt[3];
  region(kind, w.dir, b, lo, cnt);
  const int e = w.start + threadIdx.x;
  const int total = cnt[0] * cnt[1] * cnt[2];
  if (e >= total) return false;
  p[0] = lo[0] + e % cnt[0];
  p[1] = lo[1] + (e / cnt[0]) % cnt[1];
  p[2] = lo[2] + e / (cnt[0] * cnt[1]);
  return true;
}

// ------------------------------------------------------------------------------------------------
// k_cellprep
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kTile) k_cellprep(const DBlock* __restrict__ blocks,
                                                    const Work* __restrict__ work, MetricView m,
                                                    StateView s, Workspace ws, KParams kp) {
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  int p[3];
  if (!decode(R_CELLS_ALL, w, b, p)) return;
  const int i = p[0], j = p[1], k = p[2];
  if (m.order == 4) {
    for (int a = 0; a < 3; ++a)
      if (p[a] < -b.g + 1 || p[a] > b.n[a] + b.g - 2) return;
  }
  double val[10];
  cell_metric(b, m, m.order, i, j, k, 10, val, nullptr);
  const double g6[6] = {val[4], val[5], val[6], val[7], val[8], val[9]};
  const double sg = sqrt(det3(g6));
  double Bd[3];
  const long long f0 = fix(b, 0, i, j, k), f1 = fix(b, 1, i, j, k), f2 = fix(b, 2, i, j, k);
  Bd[0] = 0.5 * (s.B[0][b.face[0] + f0] + s.B[0][b.face[0] + f0 + 1]);
  Bd[1] = 0.5 * (s.B[1][b.face[1] + f1] + s.B[1][b.face[1] + f1 + b.N[0]]);
  Bd[2] = 0.5 * (s.B[2][b.face[2] + f2] + s.B[2][b.face[2] + f2 + (long long)b.N[0] * b.N[1]]);
  const long long wc = b.wcell + cix(b, i, j, k);
  const double isg = 1.0 / sg;
#pragma unroll
  for (int a = 0; a < 3; ++a) ws.bcc[a][wc] = Bd[a] * isg;
  const bool ring = i >= -1 && i <= b.n[0] && j >= -1 && j <= b.n[1] && k >= -1 && k <= b.n[2];
  if (!ring) return;
  const long long c = b.cell + cix(b, i, j, k);
  const double ut[3] = {s.W[1][c], s.W[2][c], s.W[3][c]};
  double utl[3];
  lower3(g6, ut, utl);
  const double iW = 1.0 / sqrt(1.0 + ut[0] * utl[0] + ut[1] * utl[1] + ut[2] * utl[2]);
  const double ia = 1.0 / val[0];
  double vt[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) vt[a] = ut[a] * iW - val[1 + a] * ia;
#pragma unroll
  for (int mm = 0; mm < 3; ++mm) {
    const int a = (mm + 1) % 3, bb = (mm + 2) % 3;
    ws.ecc[mm][wc] = val[0] * (vt[bb] * Bd[a] - vt[a] * Bd[bb]);
  }
}

// ------------------------------------------------------------------------------------------------
// k_faces<R>
// ------------------------------------------------------------------------------------------------
template <class R>
__global__ void __launch_bounds__(kTile) k_faces(const DBlock* __restrict__ blocks,
                                                 const Work* __restrict__ work, MetricView m,
                                                 StateView s, Workspace ws, KParams kp) {
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  int p[3];
  if (!decode(R_FACES, w, b, p)) return;
  const int d = w.dir, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  // stencil cells p[d]-3 .. p[d]+2 along d
  const long long stride = (d == 0) ? 1 : (d == 1 ? (long long)b.N[0] : (long long)b.N[0] * b.N[1]);
  int q[3] = {p[0], p[1], p[2]};
  q[d] -= 3;
  const long long c0 = cix(b, q[0], q[1], q[2]);
  R st[7][6];
  const int tlo = (b.g >= 3 || kp.recon == GR_RECON_WENOZ) ? 0 : 1;
  const int thi = (b.g >= 3 || kp.recon == GR_RECON_WENOZ) ? 6 : 5;
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    if (t < tlo || t >= thi) {
#pragma unroll
      for (int v = 0; v < 7; ++v) st[v][t] = R(0);
      continue;
    }
    const long long c = c0 + t * stride;
#pragma unroll
    for (int v = 0; v < 5; ++v) st[v][t] = R(s.W[v][b.cell + c]);
    st[5][t] = R(ws.bcc[t1][b.wcell + c]);
    st[6][t] = R(ws.bcc[t2][b.wcell + c]);
  }
  const R eps = (sizeof(R) == 4) ? R(1e-30f) : R(kp.weno_eps);
  R L[7], Rr[7];
#pragma unroll
  for (int v = 0; v < 7; ++v) recon<R>(kp.recon, st[v], eps, &L[v], &Rr[v]);
  // a non-physical reconstructed state (rho <= 0 or p <= 0) drops the face to first order
  if (!(L[0] > R(0)) || !(Rr[0] > R(0)) || !(L[4] > R(0)) || !(Rr[4] > R(0))) {
#pragma unroll
    for (int v = 0; v < 7; ++v) { L[v] = st[v][2]; Rr[v] = st[v][3]; }
  }
  R met[10];
  face_metric<R>(b, m, m.order, d, p, met);
  const R det = det3(met + 4);
  const R sg = rsqrt_(det);
  const R gdd = inv_dd(met + 4, d, det);
  const long long fi = fix(b, d, p[0], p[1], p[2]);
  const R Bn = R(s.B[d][b.face[d] + fi]);
  R BL[3], BR[3];
  BL[d] = Bn; BR[d] = Bn;
  BL[t1] = L[5] * sg; BL[t2] = L[6] * sg;
  BR[t1] = Rr[5] * sg; BR[t2] = Rr[6] * sg;
  const R gam = R(kp.gamma_ad);
  R UL[7], FL[7], UR[7], FR[7], lmL, lpL, lmR, lpR;
  face_state<R>(d, met, sg, gdd, gam, L, BL, UL, FL, &lmL, &lpL);
  face_state<R>(d, met, sg, gdd, gam, Rr, BR, UR, FR, &lmR, &lpR);
  R F[7];
  hlle<R>(UL, UR, FL, FR, lmL, lpL, lmR, lpR, F);
  R* out = reinterpret_cast<R*>(ws.flux[d]);
  const long long o = b.wface[d] + fi;
#pragma unroll
  for (int v = 0; v < 7; ++v) out[v * ws.fstride[d] + o] = F[v];
}

// ------------------------------------------------------------------------------------------------
// k_edges<R>: corner electric field E_m at (a-face ia, b-face ib, m-cell im), (a, b, m) cyclic
// ------------------------------------------------------------------------------------------------
template <class R>
__global__ void __launch_bounds__(kTile) k_edges(const DBlock* __restrict__ blocks,
                                                 const Work* __restrict__ work, Workspace ws,
                                                 KParams kp) {
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  int e[3];
  if (!decode(R_EDGES, w, b, e)) return;
  const int m = w.dir, a = (m + 1) % 3, bb = (m + 2) % 3;
  const R* Fa = reinterpret_cast<const R*>(ws.flux[a]);
  const R* Fb = reinterpret_cast<const R*>(ws.flux[bb]);
  const long long sa = ws.fstride[a], sb = ws.fstride[bb];
  const int ia = e[a], ib = e[bb];
  auto pos = [&](int ja, int jb, int r[3]) { r[a] = ja; r[bb] = jb; r[m] = e[m]; };
  int r[3];
  // a-face values at b-cells ib and ib-1; b-face values at a-cells ia and ia-1
  pos(ia, ib, r);      const long long fa1 = b.wface[a] + fix(b, a, r[0], r[1], r[2]);
  pos(ia, ib - 1, r);  const long long fa0 = b.wface[a] + fix(b, a, r[0], r[1], r[2]);
  pos(ia, ib, r);      const long long fb1 = b.wface[bb] + fix(b, bb, r[0], r[1], r[2]);
  pos(ia - 1, ib, r);  const long long fb0 = b.wface[bb] + fix(b, bb, r[0], r[1], r[2]);
  const R Ea1 = -Fa[5 * sa + fa1], Ea0 = -Fa[5 * sa + fa0];   // E_m = -F^a_{B^b}
  const R Eb1 = Fb[6 * sb + fb1], Eb0 = Fb[6 * sb + fb0];     // E_m = +F^b_{B^a}
  R E = R(0.25) * (Ea1 + Ea0 + Eb1 + Eb0);
  if (kp.emf == GR_EMF_UPWIND) {
    pos(ia, ib, r);         const R C11 = R(ws.ecc[m][b.wcell + cix(b, r[0], r[1], r[2])]);
    pos(ia - 1, ib, r);     const R C01 = R(ws.ecc[m][b.wcell + cix(b, r[0], r[1], r[2])]);
    pos(ia, ib - 1, r);     const R C10 = R(ws.ecc[m][b.wcell + cix(b, r[0], r[1], r[2])]);
    pos(ia - 1, ib - 1, r); const R C00 = R(ws.ecc[m][b.wcell + cix(b, r[0], r[1], r[2])]);
    const R va1 = Fa[fa1], va0 = Fa[fa0], vb1 = Fb[fb1], vb0 = Fb[fb0];   // mass fluxes
    auto upw = [](R vel, R lowside, R highside) {
      return vel > R(0) ? lowside : (vel < R(0) ? highside : R(0.5) * (lowside + highside));
    };
    const R db_hi = upw(va1, C01 - Eb0, C11 - Eb1);
    const R db_lo = upw(va0, Eb0 - C00, Eb1 - C10);
    const R da_hi = upw(vb1, C10 - Ea0, C11 - Ea1);
    const R da_lo = upw(vb0, Ea0 - C00, Ea1 - C01);
    E += R(0.25) * (db_lo - db_hi) + R(0.25) * (da_lo - da_hi);
  }
  R* out = reinterpret_cast<R*>(ws.edge[m]);
  out[b.wvert + vix(b, e[0], e[1], e[2])] = E;
}

// ------------------------------------------------------------------------------------------------
// k_ct: B'^d on faces of interior cells (FP64)
// ------------------------------------------------------------------------------------------------
template <class R>
__global__ void __launch_bounds__(kTile) k_ct(const DBlock* __restrict__ blocks,
                                              const Work* __restrict__ work, StateView s, Workspace ws,
                                              KParams kp) {
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  int p[3];
  if (!decode(R_CTFACES, w, b, p)) return;
  const int d = w.dir, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  const R* E2 = reinterpret_cast<const R*>(ws.edge[t2]);
  const R* E1 = reinterpret_cast<const R*>(ws.edge[t1]);
  int q[3] = {p[0], p[1], p[2]};
  const long long v0 = b.wvert + vix(b, q[0], q[1], q[2]);
  q[t1] += 1;
  const long long v1 = b.wvert + vix(b, q[0], q[1], q[2]);
  q[t1] -= 1;
  q[t2] += 1;
  const long long v2 = b.wvert + vix(b, q[0], q[1], q[2]);
  const double dE2 = ((double)E2[v1] - (double)E2[v0]) * b.idx[t1];
  const double dE1 = ((double)E1[v2] - (double)E1[v0]) * b.idx[t2];
  const long long f = b.face[d] + fix(b, d, p[0], p[1], p[2]);
  double Bn = kp.rk_g1 * s.B[d][f] - kp.rk_beta * kp.dt * (dE2 - dE1);
  if (kp.rk_g0 != 0.0) Bn += kp.rk_g0 * s.B0[d][f];
  s.Bo[d][f] = Bn;
}

// ------------------------------------------------------------------------------------------------
// k_update: U' and con2prim on interior cells (FP64)
// ------------------------------------------------------------------------------------------------
template <class R>
__global__ void __launch_bounds__(kTile) k_update(const DBlock* __restrict__ blocks,
                                                  const Work* __restrict__ work, MetricView m,
                                                  StateView s, Workspace ws, KParams kp) {
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  int p[3];
  if (!decode(R_INTERIOR, w, b, p)) return;
  const int i = p[0], j = p[1], k = p[2];
  const bool kzero = m.k_zero != 0;
  double val[16], dm[3][10];
  cell_metric(b, m, m.order, i, j, k, kzero ? 10 : 16, val, dm);
  CellMet M;
  cellmet_from(val, kzero, M);
  const long long c = b.cell + cix(b, i, j, k);
  // stage-input state at the cell: primitives and the mean densitised field of the input faces
  double wv[5], Bd[3];
#pragma unroll
  for (int v = 0; v < 5; ++v) wv[v] = s.W[v][c];
  const long long f0 = b.face[0] + fix(b, 0, i, j, k);
  const long long f1 = b.face[1] + fix(b, 1, i, j, k);
  const long long f2 = b.face[2] + fix(b, 2, i, j, k);
  const long long sy = b.N[0], sz = (long long)b.N[0] * b.N[1];
  Bd[0] = 0.5 * (s.B[0][f0] + s.B[0][f0 + 1]);
  Bd[1] = 0.5 * (s.B[1][f1] + s.B[1][f1 + sy]);
  Bd[2] = 0.5 * (s.B[2][f2] + s.B[2][f2 + sz]);
  CellFluid fl;
  cell_fluid(M, kp.gamma_ad, wv, Bd, fl);
  double src[5];
  cell_sources(M, fl, dm, kzero, src);
  // flux divergence
  const R* F0 = reinterpret_cast<const R*>(ws.flux[0]);
  const R* F1 = reinterpret_cast<const R*>(ws.flux[1]);
  const R* F2 = reinterpret_cast<const R*>(ws.flux[2]);
  const long long g0 = b.wface[0] + fix(b, 0, i, j, k);
  const long long g1 = b.wface[1] + fix(b, 1, i, j, k);
  const long long g2 = b.wface[2] + fix(b, 2, i, j, k);
  const long long oy = b.N[0], oz = (long long)b.N[0] * b.N[1];
  const double bdt = kp.rk_beta * kp.dt;
  double q[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const double dF = ((double)F0[v * ws.fstride[0] + g0 + 1] - (double)F0[v * ws.fstride[0] + g0]) * b.idx[0] +
                      ((double)F1[v * ws.fstride[1] + g1 + oy] - (double)F1[v * ws.fstride[1] + g1]) * b.idx[1] +
                      ((double)F2[v * ws.fstride[2] + g2 + oz] - (double)F2[v * ws.fstride[2] + g2]) * b.idx[2];
    double u = kp.rk_g1 * s.U[v][c] + bdt * (-dF + src[v]);
    if (kp.rk_g0 != 0.0) u += kp.rk_g0 * s.U0[v][c];
    q[v] = u;
  }
  // con2prim on the updated state; the cell field is the mean of the updated faces
  double Bn[3];
  Bn[0] = 0.5 * (s.Bo[0][f0] + s.Bo[0][f0 + 1]);
  Bn[1] = 0.5 * (s.Bo[1][f1] + s.Bo[1][f1 + sy]);
  Bn[2] = 0.5 * (s.Bo[2][f2] + s.Bo[2][f2 + sz]);
  double wn[5];
  int iters;
  const int st = con2prim_cell(M, kp, q, Bn, wn, &iters);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    s.Uo[v][c] = q[v];
    s.Wo[v][c] = wn[v];
  }
  s.status[c] = (uint8_t)st;
}

// ------------------------------------------------------------------------------------------------
// stand-alone prim2con / con2prim / diagnostics
// ------------------------------------------------------------------------------------------------
struct P2CArgs {
  const double* W[5];
  const double* B[3];
  double* U[5];
  uint8_t* status;
};

__device__ __forceinline__ void cell_field(const DBlock& b, const double* const* B, int i, int j, int k,
                                           double Bd[3]) {
  const long long f0 = b.face[0] + fix(b, 0, i, j, k);
  const long long f1 = b.face[1] + fix(b, 1, i, j, k);
  const long long f2 = b.face[2] + fix(b, 2, i, j, k);
  Bd[0] = 0.5 * (B[0][f0] + B[0][f0 + 1]);
  Bd[1] = 0.5 * (B[1][f1] + B[1][f1 + b.N[0]]);
  Bd[2] = 0.5 * (B[2][f2] + B[2][f2 + (long long)b.N[0] * b.N[1]]);
}

__global__ void __launch_bounds__(kTile) k_prim2con(const DBlock* __restrict__ blocks,
                                                    const Work* __restrict__ work, MetricView m,
                                                    P2CArgs a, KParams kp) {
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  int p[3];
  if (!decode(R_INTERIOR, w, b, p)) return;
  double val[16];
  cell_metric(b, m, m.order, p[0], p[1], p[2], 10, val, nullptr);
  CellMet M;
  cellmet_from(val, true, M);
  const long long c = b.cell + cix(b, p[0], p[1], p[2]);
  double wv[5], Bd[3], q[5];
  for (int v = 0; v < 5; ++v) wv[v] = a.W[v][c];
  cell_field(b, a.B, p[0], p[1], p[2], Bd);
  CellFluid f;
  cell_fluid(M, kp.gamma_ad, wv, Bd, f);
  cell_cons(M, f, q);
  for (int v = 0; v < 5; ++v) a.U[v][c] = q[v];
}

__global__ void __launch_bounds__(kTile) k_con2prim(const DBlock* __restrict__ blocks,
                                                    const Work* __restrict__ work, MetricView m,
                                                    P2CArgs a, KParams kp) {
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  int p[3];
  if (!decode(R_INTERIOR, w, b, p)) return;
  double val[16];
  cell_metric(b, m, m.order, p[0], p[1], p[2], 10, val, nullptr);
  CellMet M;
  cellmet_from(val, true, M);
  const long long c = b.cell + cix(b, p[0], p[1], p[2]);
  double q[5], Bd[3], wn[5];
  for (int v = 0; v < 5; ++v) q[v] = a.U[v][c];
  cell_field(b, a.B, p[0], p[1], p[2], Bd);
  int iters;
  const int st = con2prim_cell(M, kp, q, Bd, wn, &iters);
  for (int v = 0; v < 5; ++v) {
    a.U[v][c] = q[v];
    const_cast<double*>(a.W[v])[c] = wn[v];
  }
  if (a.status) a.status[c] = (uint8_t)st;
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// out: [0] sum D dV, [1] max |divB|, [2] sum |divB| dV, [3] max |B|, [4] sum dV, [5] min dx
__global__ void __launch_bounds__(kTile) k_diag(const DBlock* __restrict__ blocks,
                                                const Work* __restrict__ work, P2CArgs a, double* out) {
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  int p[3];
  double md = 0, dv = 0, mdiv = 0, sdiv = 0, mB = 0;
  if (decode(R_INTERIOR, w, b, p)) {
    const long long c = b.cell + cix(b, p[0], p[1], p[2]);
    dv = b.dx[0] * b.dx[1] * b.dx[2];
    md = a.U[0][c] * dv;
    const long long f0 = b.face[0] + fix(b, 0, p[0], p[1], p[2]);
    const long long f1 = b.face[1] + fix(b, 1, p[0], p[1], p[2]);
    const long long f2 = b.face[2] + fix(b, 2, p[0], p[1], p[2]);
    const double bx0 = a.B[0][f0], bx1 = a.B[0][f0 + 1];
    const double by0 = a.B[1][f1], by1 = a.B[1][f1 + b.N[0]];
    const double bz0 = a.B[2][f2], bz1 = a.B[2][f2 + (long long)b.N[0] * b.N[1]];
    const double div = (bx1 - bx0) * b.idx[0] + (by1 - by0) * b.idx[1] + (bz1 - bz0) * b.idx[2];
    mdiv = fabs(div);
    sdiv = fabs(div) * dv;
    mB = fmax(fmax(fmax(fabs(bx0), fabs(bx1)), fmax(fabs(by0), fabs(by1))), fmax(fabs(bz0), fabs(bz1)));
  }
  // warp reductions then one atomic per warp
  for (int o = 16; o > 0; o >>= 1) {
    md += __shfl_down_sync(0xffffffffu, md, o);
    dv += __shfl_down_sync(0xffffffffu, dv, o);
    sdiv += __shfl_down_sync(0xffffffffu, sdiv, o);
    mdiv = fmax(mdiv, __shfl_down_sync(0xffffffffu, mdiv, o));
    mB = fmax(mB, __shfl_down_sync(0xffffffffu, mB, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out + 0, md);
    atomic_max_nonneg(out + 1, mdiv);
    atomicAdd(out + 2, sdiv);
    atomic_max_nonneg(out + 3, mB);
    atomicAdd(out + 4, dv);
  }
}

// ------------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------------
template <class R>
static cudaError_t stage_impl(const DBlock* blocks, const Work* const work[R_NREGION],
                              const int nwork[R_NREGION], const MetricView& m, const StateView& s,
                              const Workspace& ws, const KParams& kp, cudaStream_t st, cudaEvent_t* ev) {
  if (ev) cudaEventRecord(ev[0], st);
  if (nwork[R_CELLS_ALL]) k_cellprep<<<nwork[R_CELLS_ALL], kTile, 0, st>>>(blocks, work[R_CELLS_ALL], m, s, ws, kp);
  if (ev) cudaEventRecord(ev[1], st);
  if (nwork[R_FACES]) k_faces<R><<<nwork[R_FACES], kTile, 0, st>>>(blocks, work[R_FACES], m, s, ws, kp);
  if (ev) cudaEventRecord(ev[2], st);
  if (nwork[R_EDGES]) k_edges<R><<<nwork[R_EDGES], kTile, 0, st>>>(blocks, work[R_EDGES], ws, kp);
  if (ev) cudaEventRecord(ev[3], st);
  if (nwork[R_CTFACES]) k_ct<R><<<nwork[R_CTFACES], kTile, 0, st>>>(blocks, work[R_CTFACES], s, ws, kp);
  if (ev) cudaEventRecord(ev[4], st);
  if (nwork[R_INTERIOR]) k_update<R><<<nwork[R_INTERIOR], kTile, 0, st>>>(blocks, work[R_INTERIOR], m, s, ws, kp);
  if (ev) cudaEventRecord(ev[5], st);
  return cudaGetLastError();
}

cudaError_t launch_stage(int precision, const DBlock* blocks, const Work* const work[R_NREGION],
                         const int nwork[R_NREGION], const MetricView& m, const StateView& s,
                         const Workspace& ws, const KParams& kp, cudaStream_t st, cudaEvent_t* ev) {
  if (precision == GR_PREC_MIXED) return stage_impl<float>(blocks, work, nwork, m, s, ws, kp, st, ev);
  return stage_impl<double>(blocks, work, nwork, m, s, ws, kp, st, ev);
}

cudaError_t launch_prim2con(const DBlock* blocks, const Work* work, int nwork, const MetricView& m,
                            const double* const W[5], const double* const B[3], double* const U[5],
                            const KParams& kp, cudaStream_t st) {
  P2CArgs a;
  for (int v = 0; v < 5; ++v) { a.W[v] = W[v]; a.U[v] = U[v]; }
  for (int d = 0; d < 3; ++d) a.B[d] = B[d];
  a.status = nullptr;
  if (nwork) k_prim2con<<<nwork, kTile, 0, st>>>(blocks, work, m, a, kp);
  return cudaGetLastError();
}

cudaError_t launch_con2prim(const DBlock* blocks, const Work* work, int nwork, const MetricView& m,
                            double* const U[5], const double* const B[3], double* const W[5],
                            uint8_t* status, const KParams& kp, cudaStream_t st) {
  P2CArgs a;
  for (int v = 0; v < 5; ++v) { a.W[v] = W[v]; a.U[v] = U[v]; }
  for (int d = 0; d < 3; ++d) a.B[d] = B[d];
  a.status = status;
  if (nwork) k_con2prim<<<nwork, kTile, 0, st>>>(blocks, work, m, a, kp);
  return cudaGetLastError();
}

cudaError_t launch_diag(const DBlock* blocks, const Work* work, int nwork, const double* const U[5],
                        const double* const B[3], double* dev_out, cudaStream_t st) {
  P2CArgs a;
  for (int v = 0; v < 5; ++v) { a.W[v] = nullptr; a.U[v] = const_cast<double*>(U[v]); }
  for (int d = 0; d < 3; ++d) a.B[d] = B[d];
  a.status = nullptr;
  cudaError_t e = cudaMemsetAsync(dev_out, 0, 8 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  if (nwork) k_diag<<<nwork, kTile, 0, st>>>(blocks, work, a, dev_out);
  return cudaGetLastError();
}

}  // namespace grs
