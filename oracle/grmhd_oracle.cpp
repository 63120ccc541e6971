// grmhd_oracle.cpp -- plain FP64 CPU oracle for one Runge-Kutta stage of the ideal-GRMHD
// conservative update of GR-Athena++ (arXiv:2311.04989), Sec. 2 and Sec. 3.
//
// TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct reference that the CUDA library
// is checked against.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
// reference legs may load it; the product path never does.  It shares no code, header, table or
// constant generator with the CUDA side: every formula below is written out again from the paper.
//
// Layout conventions (this file's own; the Python wrapper in oracle/__init__.py mirrors them):
//   cell arrays   (Nz, Ny, Nx)         N = n + 2g, cell i in [-g, n+g-1], x fastest
//   x-face arrays (Nz, Ny, Nx+1)       face i sits at x0 + i*dx (low side of cell i)
//   y-face arrays (Nz, Ny+1, Nx),  z-face arrays (Nz+1, Ny, Nx)
//   vertex arrays (Nz+1, Ny+1, Nx+1)   vertex i in [-g, n+g] at x0 + i*dx
//   metric components: 0 alpha, 1..3 beta^i, 4..9 gamma_{xx,xy,xz,yy,yz,zz}, 10..15 K_ij (same order)
//   primitives w = (rho, u~^x, u~^y, u~^z, p)                      (Sec. 2.1, after Eq. hydsrc_def)
//   conserved  q = (D, S_x, S_y, S_z, tau), B^k densitised          (Eq. consB_def)
//   tabulated EOS (Sec. 2.2.1): w = (rho, u~^i, p, Y_e, T), q = (D, S_j, tau, D Y_e); the thermodynamic
//   state of a point is (rho, p, Y_e), T is derived from it (an output of con2prim).
//
// Functions whose result has no independent pin say "parity unpinned" in their comment; the pins
// live in tests/test_oracle_*.py.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>

#ifdef ORACLE_COUNT_FLOPS
#include "flopcount.h"
typedef Counted real;
inline double to_d(const Counted& x) { return x.v; }
#else
typedef double real;
inline double to_d(double x) { return x; }
#endif

extern "C" {

// ------------------------------------------------------------------------------------------------
// Public structs (plain C, mirrored with ctypes)
// ------------------------------------------------------------------------------------------------
typedef struct {
  int32_t n[3];   // interior cells per direction
  int32_t ng;     // ghost cells on every side (cells, faces and vertices alike)
  double dx[3];   // cell widths
} ob_geom;

typedef struct {
  double gamma_ad;   // ideal-gas Gamma, p = rho*eps*(Gamma-1)  (Sec. 2.2.1)
  double rho_atm;    // atmosphere density f_atm*rho_max        (Sec. 3.5)
  double p_atm;      // atmosphere pressure p(rho_atm)           (Sec. 3.5)
  double f_thr;      // atmosphere threshold factor              (Sec. 3.5)
  double W_max;      // Lorentz-factor ceiling                   (App. A)
  double M_max;      // B^2/D ceiling                            (App. A)
  double tol;        // relative bracket tolerance of the root find (Sec. 3.5: 1e-10)
  double weno_eps;   // WENOZ epsilon
  double rk_g0, rk_g1, rk_beta;  // stage U' = g0 U0 + g1 U + beta dt L(U)
  int32_t max_iter;  // root-find iteration cap
  int32_t recon;     // 0 PLM, 1 WENOZ, 2 WENO5, 3 PPM
  int32_t emf;       // 0 upwinded corner average (Gardiner-Stone), 1 plain mean of 4 faces
  int32_t ceiling;   // 0 clamp W (App. A), 1 atmosphere (Sec. 3.5)
  int32_t interp_order;  // 2 or 4
  int32_t pad_;
  // tabulated EOS (Sec. 2.2.1); eos = 0 ideal gas (the fields below unused), 1 table
  int32_t eos;
  int32_t pad2_;
  double T_atm;      // atmosphere temperature (App. A)
  double Ye_atm;     // atmosphere electron fraction (reading: a parameter)
  double h0;         // minimum enthalpy of the table (from oracle_table_hmin)
  const struct otable_* table;
  // Atmosphere band: rho or D below f_thr rho_atm (1 + atm_band) takes the atmosphere branch.  The
  // paper resets only below the threshold (Sec. 3.5, App. A); atm_band = 1e-12 (the default) only
  // takes values equal to the threshold up to FP64 rounding off the knife-edge of a strict test.
  double atm_band;
} oparams;

// EOS table (Sec. 2.2.1): log p, log e (e = rho(1 + eps)) and c_s^2 on a uniform grid in
// (log rho, log T, Y_e), natural logarithms (the base does not change a linear interpolant).
typedef struct otable_ {
  int32_t n[3];       // nodes along log rho, log T, Y_e
  int32_t pad_;
  double x0[3];       // first node of each axis
  double dx[3];       // node spacing of each axis
  const double* lp;   // node (ir, iT, iy) at index (iy * n[1] + iT) * n[0] + ir
  const double* le;
  const double* cs2;
} otable;

}  // extern "C"

namespace {

// ------------------------------------------------------------------------------------------------
// Geometry of one ghost-padded MeshBlock
// ------------------------------------------------------------------------------------------------
struct Blk {
  int n[3], g, N[3];
  double dx[3];
  explicit Blk(const ob_geom* G) {
    g = G->ng;
    for (int d = 0; d < 3; ++d) { n[d] = G->n[d]; N[d] = n[d] + 2 * g; dx[d] = G->dx[d]; }
  }
  long ncell() const { return (long)N[0] * N[1] * N[2]; }
  long nvert() const { return (long)(N[0] + 1) * (N[1] + 1) * (N[2] + 1); }
  long nface(int d) const {
    return (long)(N[0] + (d == 0)) * (N[1] + (d == 1)) * (N[2] + (d == 2));
  }
  long c(int i, int j, int k) const { return ((long)(k + g) * N[1] + (j + g)) * N[0] + (i + g); }
  long v(int i, int j, int k) const {
    return ((long)(k + g) * (N[1] + 1) + (j + g)) * (N[0] + 1) + (i + g);
  }
  long f(int d, int i, int j, int k) const {
    const int sx = N[0] + (d == 0), sy = N[1] + (d == 1);
    return ((long)(k + g) * sy + (j + g)) * sx + (i + g);
  }
};

// index helpers: ijk[dir] convention
inline long cidx(const Blk& b, const int p[3]) { return b.c(p[0], p[1], p[2]); }
inline long fidx(const Blk& b, int d, const int p[3]) { return b.f(d, p[0], p[1], p[2]); }

// ------------------------------------------------------------------------------------------------
// 3+1 metric at a point (Sec. 2.1)
// ------------------------------------------------------------------------------------------------
struct PM {
  real alpha, beta[3], g[3][3], K[3][3], gu[3][3], detg, sqrtg;
  real beta_d[3];  // beta_i = gamma_ij beta^j
};

const int SYM[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};

void pm_from16(const real m[16], PM& P) {
  P.alpha = m[0];
  for (int i = 0; i < 3; ++i) P.beta[i] = m[1 + i];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      P.g[i][j] = m[4 + SYM[i][j]];
      P.K[i][j] = m[10 + SYM[i][j]];
    }
  // gamma = det(gamma_ij), inverse by cofactors
  const real (&g)[3][3] = P.g;
  real c00 = g[1][1] * g[2][2] - g[1][2] * g[2][1];
  real c01 = g[1][2] * g[2][0] - g[1][0] * g[2][2];
  real c02 = g[1][0] * g[2][1] - g[1][1] * g[2][0];
  real det = g[0][0] * c00 + g[0][1] * c01 + g[0][2] * c02;
  P.detg = det;
  P.sqrtg = std::sqrt(det);
  P.gu[0][0] = c00 / det;
  P.gu[0][1] = (g[0][2] * g[2][1] - g[0][1] * g[2][2]) / det;
  P.gu[0][2] = (g[0][1] * g[1][2] - g[0][2] * g[1][1]) / det;
  P.gu[1][0] = c01 / det;
  P.gu[1][1] = (g[0][0] * g[2][2] - g[0][2] * g[2][0]) / det;
  P.gu[1][2] = (g[0][2] * g[1][0] - g[0][0] * g[1][2]) / det;
  P.gu[2][0] = c02 / det;
  P.gu[2][1] = (g[0][1] * g[2][0] - g[0][0] * g[2][1]) / det;
  P.gu[2][2] = (g[0][0] * g[1][1] - g[0][1] * g[1][0]) / det;
  for (int i = 0; i < 3; ++i) {
    P.beta_d[i] = 0;
    for (int j = 0; j < 3; ++j) P.beta_d[i] += g[i][j] * P.beta[j];
  }
}

// ------------------------------------------------------------------------------------------------
// Ideal-gas EOS, p = rho*eps*(Gamma - 1)  (Sec. 2.2.1).  Minimum enthalpy h0 = 1, eps >= 0.
// ------------------------------------------------------------------------------------------------
inline real eos_eps(const oparams& Q, real rho, real p) { return p / ((Q.gamma_ad - 1) * rho); }
inline real eos_p(const oparams& Q, real rho, real eps) { return (Q.gamma_ad - 1) * rho * eps; }
// Sound speed of the ideal gas, c_s^2 = Gamma p / (rho h)  (reading c3; the paper does not print it)
inline real eos_cs2(const oparams& Q, real rho, real p, real h) { return Q.gamma_ad * p / (rho * h); }

// ------------------------------------------------------------------------------------------------
// Tabulated EOS (Sec. 2.2.1): trilinear interpolation of log p, log e and c_s^2 in (log rho, log T,
// Y_e).  The interpolation is written for the specific quantities log(p/rho) = log p - log rho and
// log(e/rho) = log(1 + eps): log rho is linear along its axis, so their interpolants are exactly the
// interpolants of log p and log e minus log rho, while their values stay O(1) (no loss of eps to
// the rest-mass part of e).  Values outside the table are moved to the nearest permissible value
// (App. A); a density outside the table takes the specific quantities of the nearest table density
// (reading).  These lookups work in double (the operation-counting build does not count them).
// ------------------------------------------------------------------------------------------------
enum { TAB_LP = 0, TAB_LE = 1, TAB_CS2 = 2 };
// Cell index i in [0, n-2] and fraction w in [0, 1] of x on axis ax; clamps x into the axis range.
void tab_axis(const otable& T, int ax, double x, int* i, double* w, bool* clamped) {
  const double lo = T.x0[ax], hi = T.x0[ax] + (T.n[ax] - 1) * T.dx[ax];
  if (!(x >= lo)) { x = lo; *clamped = true; }   // also catches NaN
  if (x > hi) { x = hi; *clamped = true; }
  const double sx = (x - lo) / T.dx[ax];
  int k = (int)std::floor(sx);
  if (k > T.n[ax] - 2) k = T.n[ax] - 2;
  if (k < 0) k = 0;
  *i = k;
  *w = sx - k;
}
inline long tab_idx(const otable& T, int ir, int iT, int iy) {
  return ((long)iy * T.n[1] + iT) * T.n[0] + ir;
}
// node value of log(p/rho), log(e/rho) or c_s^2
double tab_node(const otable& T, int f, int ir, int iT, int iy) {
  const long k = tab_idx(T, ir, iT, iy);
  const double lrho = T.x0[0] + ir * T.dx[0];
  if (f == TAB_LP) return T.lp[k] - lrho;
  if (f == TAB_LE) return T.le[k] - lrho;
  return T.cs2[k];
}
// Trilinear interpolant of field f at the point with cell indices i[3] and fractions w[3]
double tab_tri(const otable& T, int f, const int i[3], const double w[3]) {
  double s = 0;
  for (int c = 0; c < 8; ++c) {
    const int a = c & 1, b = (c >> 1) & 1, e = (c >> 2) & 1;
    const double wt = (a ? w[0] : 1 - w[0]) * (b ? w[1] : 1 - w[1]) * (e ? w[2] : 1 - w[2]);
    s += wt * tab_node(T, f, i[0] + a, i[1] + b, i[2] + e);
  }
  return s;
}
// Interpolant of field f at T node k (bilinear in log rho, Y_e)
double tab_at_T_node(const otable& T, int f, const int i[3], const double w[3], int k) {
  double s = 0;
  for (int c = 0; c < 4; ++c) {
    const int a = c & 1, e = (c >> 1) & 1;
    s += (a ? w[0] : 1 - w[0]) * (e ? w[2] : 1 - w[2]) * tab_node(T, f, i[0] + a, k, i[2] + e);
  }
  return s;
}
// log T at which the interpolant of field f (increasing in T) equals y at the (log rho, Y_e) of i, w
// (the nested temperature root of App. A).  Between T nodes the interpolant is linear in log T, so
// the root lies on the node interval where the node values cross y and is found there in closed
// form; y outside the values at the table's T ends gives that end (clamped).
double tab_inverse_T(const otable& T, int f, const int i[3], const double w[3], double y, bool* clamped) {
  const int nT = T.n[1];
  const double g0 = tab_at_T_node(T, f, i, w, 0), gN = tab_at_T_node(T, f, i, w, nT - 1);
  if (!(y > g0)) { if (y < g0 || !(y == y)) *clamped = true; return T.x0[1]; }
  if (y >= gN) { if (y > gN) *clamped = true; return T.x0[1] + (nT - 1) * T.dx[1]; }
  double gk = g0;
  for (int k = 0; k < nT - 1; ++k) {
    const double gk1 = tab_at_T_node(T, f, i, w, k + 1);
    if (gk <= y && y <= gk1) return T.x0[1] + T.dx[1] * (k + (y - gk) / (gk1 - gk));
    gk = gk1;
  }
  return T.x0[1] + (nT - 1) * T.dx[1];   // not reached for a table increasing in T
}

// Thermodynamics of a point from (rho, p, Y_e): eps, h, c_s^2 and T.  Ideal gas: T = p/rho.
struct Thermo {
  real eps, h, cs2, T;
  bool clamped;
};
void eos_from_rho_p(const oparams& Q, real rho, real p, real ye, Thermo& t) {
  t.clamped = false;
  if (Q.eos == 0) {
    t.eps = eos_eps(Q, rho, p);
    t.h = 1 + t.eps + p / rho;
    t.cs2 = eos_cs2(Q, rho, p, t.h);
    t.T = p / rho;
    return;
  }
  const otable& T = *Q.table;
  int i[3];
  double w[3];
  tab_axis(T, 0, std::log(to_d(rho)), &i[0], &w[0], &t.clamped);
  tab_axis(T, 2, to_d(ye), &i[2], &w[2], &t.clamped);
  // temperature at which the table's p/rho equals this point's
  const double lT = tab_inverse_T(T, TAB_LP, i, w, std::log(to_d(p / rho)), &t.clamped);
  tab_axis(T, 1, lT, &i[1], &w[1], &t.clamped);
  const double l1e = tab_tri(T, TAB_LE, i, w);     // log(1 + eps)
  t.eps = std::expm1(l1e);
  t.h = real(std::exp(l1e)) + p / rho;
  t.cs2 = tab_tri(T, TAB_CS2, i, w);
  t.T = std::exp(lT);
}
// Pressure and eps at (rho, T, Y_e) from the table (atmosphere, temperature floor, tau floor)
void eos_table_rho_T(const oparams& Q, real rho, real Tt, real ye, real* p, real* eps) {
  const otable& T = *Q.table;
  int i[3];
  double w[3];
  bool cl = false;
  tab_axis(T, 0, std::log(to_d(rho)), &i[0], &w[0], &cl);
  tab_axis(T, 1, std::log(to_d(Tt)), &i[1], &w[1], &cl);
  tab_axis(T, 2, to_d(ye), &i[2], &w[2], &cl);
  *p = rho * std::exp(tab_tri(T, TAB_LP, i, w));
  *eps = std::expm1(tab_tri(T, TAB_LE, i, w));
}

// ------------------------------------------------------------------------------------------------
// Fluid and field at a point: the kinematics of Sec. 2.1 and the comoving field of Sec. 2.2
// ------------------------------------------------------------------------------------------------
struct FP {
  real rho, p, eps, h, W, ye, T, cs2;
  real ut_u[3], ut_d[3];   // u~^i, u~_i
  real v_u[3], v_d[3];     // v^i = u~^i / W
  real vt_u[3];            // v~^i = v^i - beta^i/alpha
  real B_u[3], B_d[3];     // Eulerian field calB^i (undensitised) and calB_i
  real Bd_u[3];            // densitised B^i = sqrt(gamma) calB^i
  real b0, b_u[3], b_d[3], b2;
};

// w = (rho, u~^i, p[, Y_e]); Bdens = densitised B^i
void fluid_point(const PM& M, const oparams& Q, const real w[], const real Bdens[3], FP& F) {
  F.rho = w[0];
  F.p = w[4];
  F.ye = Q.eos ? w[5] : real(0);
  for (int i = 0; i < 3; ++i) F.ut_u[i] = w[1 + i];
  real uu = 0;
  for (int i = 0; i < 3; ++i) {
    F.ut_d[i] = 0;
    for (int j = 0; j < 3; ++j) F.ut_d[i] += M.g[i][j] * F.ut_u[j];
  }
  for (int i = 0; i < 3; ++i) uu += F.ut_u[i] * F.ut_d[i];
  F.W = std::sqrt(1 + uu);  // W^2 = 1 + u~_i u~^i for the projected 4-velocity
  for (int i = 0; i < 3; ++i) {
    F.v_u[i] = F.ut_u[i] / F.W;
    F.v_d[i] = F.ut_d[i] / F.W;
    F.vt_u[i] = F.v_u[i] - M.beta[i] / M.alpha;
  }
  Thermo th;
  eos_from_rho_p(Q, F.rho, F.p, F.ye, th);
  F.eps = th.eps;
  F.h = th.h;
  F.cs2 = th.cs2;
  F.T = th.T;
  // B^k = sqrt(gamma) calB^k  (Eq. consB_def)
  for (int i = 0; i < 3; ++i) {
    F.Bd_u[i] = Bdens[i];
    F.B_u[i] = Bdens[i] / M.sqrtg;
  }
  for (int i = 0; i < 3; ++i) {
    F.B_d[i] = 0;
    for (int j = 0; j < 3; ++j) F.B_d[i] += M.g[i][j] * F.B_u[j];
  }
  // b^0 = W calB^i v_i / alpha ;  b^i = (calB^i + alpha b^0 W v~^i)/W  (Sec. 2.2)
  real Bv = 0, BB = 0;
  for (int i = 0; i < 3; ++i) { Bv += F.B_u[i] * F.v_d[i]; BB += F.B_u[i] * F.B_d[i]; }
  F.b0 = F.W * Bv / M.alpha;
  for (int i = 0; i < 3; ++i) F.b_u[i] = (F.B_u[i] + M.alpha * F.b0 * F.W * F.vt_u[i]) / F.W;
  // b^2 = ((alpha b^0)^2 + calB^i calB^j gamma_ij) / W^2
  F.b2 = ((M.alpha * F.b0) * (M.alpha * F.b0) + BB) / (F.W * F.W);
  // b_i = g_{i mu} b^mu = beta_i b^0 + gamma_ij b^j
  for (int i = 0; i < 3; ++i) {
    F.b_d[i] = M.beta_d[i] * F.b0;
    for (int j = 0; j < 3; ++j) F.b_d[i] += M.g[i][j] * F.b_u[j];
  }
}

// Conserved variables, Eq. consB_def: q = sqrt(gamma) (rho W, (rho h + b^2) W u~_j - alpha b^0 b_j,
//   (rho h + b^2) W^2 - rho W - (p + b^2/2) - (alpha b^0)^2)
void cons_from_fp(const PM& M, const FP& F, real q[5]) {
  const real sg = M.sqrtg, ab0 = M.alpha * F.b0, eb = F.rho * F.h + F.b2;
  q[0] = sg * F.rho * F.W;
  for (int j = 0; j < 3; ++j) q[1 + j] = sg * (eb * F.W * F.ut_d[j] - ab0 * F.b_d[j]);
  q[4] = sg * (eb * F.W * F.W - F.rho * F.W - (F.p + 0.5 * F.b2) - ab0 * ab0);
}
// All conserved variables of the EOS: with a table also D Y_e (Sec. 2.2.1)
void cons_all(const oparams& Q, const PM& M, const FP& F, real q[]) {
  cons_from_fp(M, F, q);
  if (Q.eos) q[5] = q[0] * F.ye;
}

// Fluxes in direction d, Eq. fluxB_def.  Fq = (D, S_j, tau) rows; Fb[0], Fb[1] = induction flux of
// B^{t1}, B^{t2} with t1 = (d+1)%3, t2 = (d+2)%3:  F^d_{B^k} = alpha (B^k v~^d - B^d v~^k).
void flux_from_fp(const PM& M, const FP& F, const real q[5], int d, real Fq[5], real Fb[2]) {
  const real a = M.alpha, sg = M.sqrtg, pt = F.p + 0.5 * F.b2;
  Fq[0] = q[0] * a * F.vt_u[d];
  for (int j = 0; j < 3; ++j)
    Fq[1 + j] = q[1 + j] * a * F.vt_u[d] + (j == d ? pt * a * sg : 0.0) -
                a * sg * F.b_d[j] * F.B_u[d] / F.W;
  Fq[4] = q[4] * a * F.vt_u[d] + a * sg * (pt * F.v_u[d] - a * F.b0 * F.B_u[d] / F.W);
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  Fb[0] = a * (F.Bd_u[t1] * F.vt_u[d] - F.Bd_u[d] * F.vt_u[t1]);
  Fb[1] = a * (F.Bd_u[t2] * F.vt_u[d] - F.Bd_u[d] * F.vt_u[t2]);
}

// Fast speeds along d (reading c2 of the approximate quadratic dispersion relation of Sec. 2.2):
// c^2 = cs^2 + cA^2 - cs^2 cA^2, cA^2 = b^2/(rho h + b^2), and the 3+1 closed form
// lam = alpha [v^d (1-c^2) +- c sqrt((1-v^2)(gamma^dd (1 - v^2 c^2) - v^d v^d (1-c^2)))]/(1-v^2c^2) - beta^d
void speeds_from_fp(const PM& M, const oparams& Q, const FP& F, int d, real* lm, real* lp) {
  (void)Q;
  const real cs2 = F.cs2;
  const real ca2 = F.b2 / (F.rho * F.h + F.b2);
  const real c2 = cs2 + ca2 - cs2 * ca2;
  real v2 = 0;
  for (int i = 0; i < 3; ++i) v2 += F.v_u[i] * F.v_d[i];
  const real vd = F.v_u[d];
  real disc = (1 - v2) * (M.gu[d][d] * (1 - v2 * c2) - vd * vd * (1 - c2));
  if (disc < 0) disc = 0;
  const real c = std::sqrt(c2);
  const real den = 1 - v2 * c2;
  *lp = M.alpha * (vd * (1 - c2) + c * std::sqrt(disc)) / den - M.beta[d];
  *lm = M.alpha * (vd * (1 - c2) - c * std::sqrt(disc)) / den - M.beta[d];
}

// HLLE numerical flux (reading c1; the paper does not name its Riemann solver).
// lam+ = max(0, lam+_L, lam+_R), lam- = min(0, lam-_L, lam-_R);
// F = (lam+ F_L - lam- F_R + lam+ lam- (U_R - U_L)) / (lam+ - lam-), or (F_L + F_R)/2 if lam+ = lam-.
void hlle(int nv, const real* UL, const real* UR, const real* FL, const real* FR, real lmL, real lpL,
          real lmR, real lpR, real* Fout) {
  real lp = std::max((real)0, std::max(lpL, lpR));
  real lm = std::min((real)0, std::min(lmL, lmR));
  if (lp - lm == 0) {
    for (int v = 0; v < nv; ++v) Fout[v] = 0.5 * (FL[v] + FR[v]);
    return;
  }
  for (int v = 0; v < nv; ++v)
    Fout[v] = (lp * FL[v] - lm * FR[v] + lp * lm * (UR[v] - UL[v])) / (lp - lm);
}

// Face flux from two primitive states at one face (shared by the stage and the point entry).
// wL/wR: prims; BL/BR: densitised B^i of the two states (same normal component).  With a table,
// Fq[5] is the D Y_e flux: the HLLE D flux times the electron fraction of the upwind state (the
// D equation multiplied by Y_e, Sec. 2.2.1; reading: upwinded as in the consistent multi-fluid
// advection it cites).
void face_flux(const PM& M, const oparams& Q, int d, const real wL[], const real BL[3],
               const real wR[], const real BR[3], real Fq[], real Fb[2]) {
  FP L, R;
  fluid_point(M, Q, wL, BL, L);
  fluid_point(M, Q, wR, BR, R);
  real UL[7], UR[7], FL[7], FR[7];
  cons_from_fp(M, L, UL);
  cons_from_fp(M, R, UR);
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  UL[5] = BL[t1]; UL[6] = BL[t2];
  UR[5] = BR[t1]; UR[6] = BR[t2];
  flux_from_fp(M, L, UL, d, FL, FL + 5);
  flux_from_fp(M, R, UR, d, FR, FR + 5);
  real lmL, lpL, lmR, lpR;
  speeds_from_fp(M, Q, L, d, &lmL, &lpL);
  speeds_from_fp(M, Q, R, d, &lmR, &lpR);
  real F[7];
  hlle(7, UL, UR, FL, FR, lmL, lpL, lmR, lpR, F);
  for (int v = 0; v < 5; ++v) Fq[v] = F[v];
  Fb[0] = F[5];
  Fb[1] = F[6];
  if (Q.eos) Fq[5] = F[0] * (F[0] > 0 ? L.ye : R.ye);
}

// ------------------------------------------------------------------------------------------------
// Reconstruction (Sec. 3.4).  Readings c4 (van Leer PLM) and c5 (WENOZ, Borges et al., exponent 1).
// ------------------------------------------------------------------------------------------------
// Harmonic van Leer slope of cell 0 from its neighbours
inline real vl_slope(real wm, real w0, real wp) {
  const real dL = w0 - wm, dR = wp - w0;
  return (dL * dR > 0) ? 2 * dL * dR / (dL + dR) : 0.0;
}
// WENOZ value at the right edge of the middle cell of v[0..4]
real wenoz_edge(real v0, real v1, real v2, real v3, real v4, real eps) {
  // candidate third-order values on the three sub-stencils
  const real q0 = (2 * v0 - 7 * v1 + 11 * v2) / 6;
  const real q1 = (-v1 + 5 * v2 + 2 * v3) / 6;
  const real q2 = (2 * v2 + 5 * v3 - v4) / 6;
  // Jiang-Shu smoothness indicators
  const real a0 = v0 - 2 * v1 + v2, b0 = v0 - 4 * v1 + 3 * v2;
  const real a1 = v1 - 2 * v2 + v3, b1 = v1 - v3;
  const real a2 = v2 - 2 * v3 + v4, b2 = 3 * v2 - 4 * v3 + v4;
  const real s0 = (13.0 / 12.0) * a0 * a0 + 0.25 * b0 * b0;
  const real s1 = (13.0 / 12.0) * a1 * a1 + 0.25 * b1 * b1;
  const real s2 = (13.0 / 12.0) * a2 * a2 + 0.25 * b2 * b2;
  // Z weights: alpha_k = d_k (1 + tau5/(beta_k + eps)), tau5 = |beta_0 - beta_2|
  const real tau5 = std::fabs(s0 - s2);
  const real w0 = 0.1 * (1 + tau5 / (s0 + eps));
  const real w1 = 0.6 * (1 + tau5 / (s1 + eps));
  const real w2 = 0.3 * (1 + tau5 / (s2 + eps));
  return (w0 * q0 + w1 * q1 + w2 * q2) / (w0 + w1 + w2);
}
// WENO5 value at the right edge of the middle cell of v[0..4] (Jiang & Shu): the same candidates and
// smoothness indicators as WENOZ, classic weights alpha_k = d_k / (beta_k + eps)^2
real weno5_edge(real v0, real v1, real v2, real v3, real v4, real eps) {
  const real q0 = (2 * v0 - 7 * v1 + 11 * v2) / 6;
  const real q1 = (-v1 + 5 * v2 + 2 * v3) / 6;
  const real q2 = (2 * v2 + 5 * v3 - v4) / 6;
  const real a0 = v0 - 2 * v1 + v2, b0 = v0 - 4 * v1 + 3 * v2;
  const real a1 = v1 - 2 * v2 + v3, b1 = v1 - v3;
  const real a2 = v2 - 2 * v3 + v4, b2 = 3 * v2 - 4 * v3 + v4;
  const real s0 = (13.0 / 12.0) * a0 * a0 + 0.25 * b0 * b0;
  const real s1 = (13.0 / 12.0) * a1 * a1 + 0.25 * b1 * b1;
  const real s2 = (13.0 / 12.0) * a2 * a2 + 0.25 * b2 * b2;
  const real w0 = 0.1 / ((s0 + eps) * (s0 + eps));
  const real w1 = 0.6 / ((s1 + eps) * (s1 + eps));
  const real w2 = 0.3 / ((s2 + eps) * (s2 + eps));
  return (w0 * q0 + w1 * q1 + w2 * q2) / (w0 + w1 + w2);
}

// PPM (reading of "PPM (Colella et al. 2011, McCorquodale & Colella 2015) as implemented in
// Athena++"): fourth-order interface values limited by the extremum-preserving criterion of Colella &
// Sekora, then the parabola of each cell limited the same way at extrema and by the monotonicity
// conditions elsewhere.  C = 1.25.
const double PPM_C = 1.25;
inline real sgn(real x) { return x > 0 ? real(1) : (x < 0 ? real(-1) : real(0)); }
inline real min3(real a, real b, real c) { return std::min(a, std::min(b, c)); }
// limited interface value between q1 and q2 (neighbours q0, q3)
real ppm_iface(real q0, real q1, real q2, real q3) {
  real qf = (7.0 / 12.0) * (q1 + q2) - (1.0 / 12.0) * (q0 + q3);
  if ((qf - q1) * (q2 - qf) < 0) {   // not between its neighbours: limit its curvature
    const real d2f = 3 * (q1 - 2 * qf + q2);
    const real d2l = q0 - 2 * q1 + q2;
    const real d2r = q1 - 2 * q2 + q3;
    real d2lim = 0;
    if (sgn(d2f) == sgn(d2l) && sgn(d2f) == sgn(d2r) && d2f != 0)
      d2lim = sgn(d2f) * min3(PPM_C * std::fabs(d2l), PPM_C * std::fabs(d2r), std::fabs(d2f));
    qf = 0.5 * (q1 + q2) - d2lim / 6;
  }
  return qf;
}
// left (qm) and right (qp) values of the limited parabola in the middle cell of v[0..4]
void ppm_cell(real v0, real v1, real v2, real v3, real v4, real* qm, real* qp) {
  real l = ppm_iface(v0, v1, v2, v3);   // interface v1|v2
  real r = ppm_iface(v1, v2, v3, v4);   // interface v2|v3
  const real q = v2;
  if ((r - q) * (q - l) <= 0 || (v1 - q) * (q - v3) <= 0) {
    // local extremum: scale the parabola's deviation by the limited curvature
    const real d2 = 6 * (l - 2 * q + r);
    const real d2c = v1 - 2 * q + v3;
    const real d2l = v0 - 2 * v1 + q;
    const real d2r = q - 2 * v3 + v4;
    real d2lim = 0;
    if (sgn(d2) == sgn(d2c) && sgn(d2) == sgn(d2l) && sgn(d2) == sgn(d2r) && d2 != 0)
      d2lim = sgn(d2) * std::min(min3(PPM_C * std::fabs(d2l), PPM_C * std::fabs(d2r), PPM_C * std::fabs(d2c)),
                                 std::fabs(d2));
    if (d2 == 0) { l = q; r = q; }
    else {
      l = q + (l - q) * d2lim / d2;
      r = q + (r - q) * d2lim / d2;
    }
  } else {
    // monotone: keep the parabola from overshooting inside the cell
    if (std::fabs(r - q) >= 2 * std::fabs(l - q)) r = q - 2 * (l - q);
    if (std::fabs(l - q) >= 2 * std::fabs(r - q)) l = q - 2 * (r - q);
  }
  *qm = l;
  *qp = r;
}

// Left/right states at the face between s[2] (left cell) and s[3] (right cell) of a 6-cell stencil
// s[0..5] = cells f-3 .. f+2.  Methods: 0 PLM, 1 WENOZ, 2 WENO5, 3 PPM (Sec. 3.4).
void recon_face(int method, const real s[6], real eps, real* L, real* R) {
  if (method == 0) {
    *L = s[2] + 0.5 * vl_slope(s[1], s[2], s[3]);
    *R = s[3] - 0.5 * vl_slope(s[2], s[3], s[4]);
  } else if (method == 1) {
    *L = wenoz_edge(s[0], s[1], s[2], s[3], s[4], eps);
    *R = wenoz_edge(s[5], s[4], s[3], s[2], s[1], eps);
  } else if (method == 2) {
    *L = weno5_edge(s[0], s[1], s[2], s[3], s[4], eps);
    *R = weno5_edge(s[5], s[4], s[3], s[2], s[1], eps);
  } else {
    real lm, lp, rm, rp;
    ppm_cell(s[0], s[1], s[2], s[3], s[4], &lm, &lp);   // left cell's parabola: its right value
    ppm_cell(s[1], s[2], s[3], s[4], s[5], &rm, &rp);   // right cell's parabola: its left value
    *L = lp;
    *R = rm;
  }
}

// ------------------------------------------------------------------------------------------------
// Vertex -> cell / face Lagrange interpolation of the metric (Sec. 3.2, reading c10)
// ------------------------------------------------------------------------------------------------
// weights and first-vertex offset of the 1D midpoint interpolant and its derivative
void mid_w(int order, real w[4], int* off, int* np) {
  if (order == 4) {
    w[0] = -1.0 / 16; w[1] = 9.0 / 16; w[2] = 9.0 / 16; w[3] = -1.0 / 16;
    *off = -1; *np = 4;
  } else {
    w[0] = 0.5; w[1] = 0.5; *off = 0; *np = 2;
  }
}

// Tensor-product interpolation at the centre of cell (i,j,k); deriv = -1 for the value, else the
// direction of the derivative.  Along the derivative direction the interpolant's derivative is
// written as differences, (f1 - f0)/dx at order 2 and (27 (f2 - f1) - (f3 - f0))/(24 dx) at order 4,
// so that it vanishes exactly on a constant field.
void interp_cell(const Blk& b, const double* const* mv, int order, int i, int j, int k, int deriv,
                 real out[16]) {
  real wi[3][4];
  int off, np;
  for (int d = 0; d < 3; ++d) mid_w(order, wi[d], &off, &np);
  for (int c = 0; c < 16; ++c) out[c] = 0;
  const int base[3] = {i + off, j + off, k + off};
  for (int c = 0; c < 16; ++c)
    for (int kk = 0; kk < np; ++kk)
      for (int jj = 0; jj < np; ++jj)
        for (int ii = 0; ii < np; ++ii) {
          const int t[3] = {ii, jj, kk};
          if (deriv < 0) {
            const real w = wi[0][ii] * wi[1][jj] * wi[2][kk];
            out[c] += w * mv[c][b.v(base[0] + ii, base[1] + jj, base[2] + kk)];
            continue;
          }
          if (t[deriv] != 0) continue;   // one pass per transverse point
          real w = 1;
          for (int d = 0; d < 3; ++d)
            if (d != deriv) w *= wi[d][t[d]];
          auto f = [&](int s) {
            int q[3] = {base[0] + ii, base[1] + jj, base[2] + kk};
            q[deriv] = base[deriv] + s;
            return mv[c][b.v(q[0], q[1], q[2])];
          };
          real diff;
          if (order == 4) diff = (27 * (f(2) - f(1)) - (f(3) - f(0))) / (24 * b.dx[deriv]);
          else diff = (f(1) - f(0)) / b.dx[deriv];
          out[c] += w * diff;
        }
}

// Interpolation at the centre of the d-face with index p (face at vertex plane p[d])
void interp_face(const Blk& b, const double* const* mv, int order, int d, const int p[3], real out[16]) {
  real wi[3][4];
  int o[3], np[3];
  for (int e = 0; e < 3; ++e) {
    if (e == d) { wi[e][0] = 1; o[e] = 0; np[e] = 1; }
    else mid_w(order, wi[e], &o[e], &np[e]);
  }
  for (int c = 0; c < 16; ++c) out[c] = 0;
  for (int c = 0; c < 16; ++c)
    for (int kk = 0; kk < np[2]; ++kk)
      for (int jj = 0; jj < np[1]; ++jj)
        for (int ii = 0; ii < np[0]; ++ii) {
          const real w = wi[0][ii] * wi[1][jj] * wi[2][kk];
          out[c] += w * mv[c][b.v(p[0] + o[0] + ii, p[1] + o[1] + jj, p[2] + o[2] + kk)];
        }
}

// ------------------------------------------------------------------------------------------------
// Geometric source terms, Eq. hydsrc_def with T^{mu nu} of Eq. EMT_MHD (Sec. 2.2).
// dm[k][c] = d_k of metric component c (only alpha, beta, gamma are used).
// ------------------------------------------------------------------------------------------------
void sources(const PM& M, const FP& F, const real dm[3][16], real s[5]) {
  const real a = M.alpha;
  // 4-velocity u^0 = W/alpha, u^i = W v~^i
  real u[4], b[4];
  u[0] = F.W / a;
  for (int i = 0; i < 3; ++i) u[1 + i] = F.W * F.vt_u[i];
  b[0] = F.b0;
  for (int i = 0; i < 3; ++i) b[1 + i] = F.b_u[i];
  // inverse 4-metric of the 3+1 split
  real gu4[4][4];
  gu4[0][0] = -1 / (a * a);
  for (int i = 0; i < 3; ++i) {
    gu4[0][1 + i] = gu4[1 + i][0] = M.beta[i] / (a * a);
    for (int j = 0; j < 3; ++j) gu4[1 + i][1 + j] = M.gu[i][j] - M.beta[i] * M.beta[j] / (a * a);
  }
  const real eb = F.rho * F.h + F.b2, pt = F.p + 0.5 * F.b2;
  real T[4][4];
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) T[m][n] = eb * u[m] * u[n] + pt * gu4[m][n] - b[m] * b[n];
  // T^0_i = T^{00} beta_i + T^{0j} gamma_ji
  real T0d[3];
  for (int i = 0; i < 3; ++i) {
    T0d[i] = T[0][0] * M.beta_d[i];
    for (int j = 0; j < 3; ++j) T0d[i] += T[0][1 + j] * M.g[j][i];
  }
  s[0] = 0;
  for (int k = 0; k < 3; ++k) {
    real t1 = 0, t2 = 0, t3 = 0, t4 = 0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const real dg = dm[k][4 + SYM[i][j]];
        t1 += 0.5 * M.beta[i] * M.beta[j] * dg;
        t2 += T[0][1 + i] * M.beta[j] * dg;
        t4 += 0.5 * T[1 + i][1 + j] * dg;
      }
    for (int i = 0; i < 3; ++i) t3 += T0d[i] * dm[k][1 + i];
    s[1 + k] = a * M.sqrtg * (T[0][0] * (t1 - a * dm[k][0]) + t2 + t3 + t4);
  }
  real e1 = 0, e2 = 0, e3 = 0;
  for (int i = 0; i < 3; ++i) {
    real bK = 0;
    for (int j = 0; j < 3; ++j) {
      e1 += M.beta[i] * M.beta[j] * M.K[i][j];
      bK += M.beta[j] * M.K[i][j];
      e3 += T[1 + i][1 + j] * M.K[i][j];
    }
    e1 -= M.beta[i] * dm[i][0];
    e2 += T[0][1 + i] * (2 * bK - dm[i][0]);
  }
  s[4] = a * M.sqrtg * (T[0][0] * e1 + e2 + e3);
}

// ------------------------------------------------------------------------------------------------
// Con2prim: KKC master function in mu = 1/(hW) with the PrimitiveSolver error policy (App. A) and
// the atmosphere of Sec. 3.5.  Readings c13-c16, c18.  Status bits:
//   1 atmosphere by threshold, 2 failure -> atmosphere, 4 W clamped (or ceiling -> atmosphere),
//   8 tau floored, 16 B^2/D limited, 32 EOS bound clamp.
// ------------------------------------------------------------------------------------------------
struct C2PIn {  // undensitised invariants
  real D, q, r2, b2, rb;  // D~, tau~/D~, r^2, calb^2, r.calb
  real ye;                // electron fraction (table)
};
struct C2PEval {
  real x, rbar2, qbar, v2, W, rho, eps, p, f, T;
  bool vcap, eclamp;
};

void c2p_eval(const oparams& Q, const C2PIn& I, real mu, C2PEval& E) {
  const real vmax2 = 1 - 1 / (Q.W_max * Q.W_max);
  E.x = 1 / (1 + mu * I.b2);
  E.rbar2 = E.x * E.x * I.r2 + mu * E.x * (1 + E.x) * I.rb * I.rb;
  E.qbar = I.q - 0.5 * I.b2 - 0.5 * mu * mu * E.x * E.x * (I.b2 * I.r2 - I.rb * I.rb);
  E.v2 = mu * mu * E.rbar2;
  E.vcap = false;
  if (E.v2 > vmax2) { E.v2 = vmax2; E.vcap = true; }
  E.W = 1 / std::sqrt(1 - E.v2);
  E.rho = I.D / E.W;
  E.eps = E.W * (E.qbar - mu * E.rbar2) + E.v2 * E.W * E.W / (1 + E.W);
  E.eclamp = false;
  if (Q.eos == 0) {
    if (E.eps < 0) { E.eps = 0; E.eclamp = true; }   // ideal-gas range eps >= 0
    E.p = eos_p(Q, E.rho, E.eps);
    E.T = E.p / E.rho;
  } else {
    // table: rho into the table's range, then the temperature of e/rho = 1 + eps (the nested
    // root), eps reset to the table's value when it lies outside the range at this rho (App. A)
    const otable& T = *Q.table;
    int i[3];
    double w[3];
    bool cl = false;
    const double lr = std::log(to_d(E.rho));
    tab_axis(T, 0, lr, &i[0], &w[0], &cl);
    if (cl) { E.rho = std::exp(T.x0[0] + (lr < T.x0[0] ? 0 : T.n[0] - 1) * T.dx[0]); E.eclamp = true; cl = false; }
    tab_axis(T, 2, to_d(I.ye), &i[2], &w[2], &cl);
    const double ope = to_d(E.eps);   // 1 + eps = e/rho, as log(1 + eps)
    const double lT = tab_inverse_T(T, TAB_LE, i, w, ope > -1 ? std::log1p(ope) : -HUGE_VAL, &cl);
    tab_axis(T, 1, lT, &i[1], &w[1], &cl);
    if (cl) { E.eps = std::expm1(tab_tri(T, TAB_LE, i, w)); E.eclamp = true; }
    E.p = E.rho * std::exp(tab_tri(T, TAB_LP, i, w));
    E.T = std::exp(lT);
  }
  const real ah = E.p / (E.rho * (1 + E.eps));
  const real nuA = (1 + ah) * (1 + E.eps) / E.W;
  const real nuB = (1 + ah) * (1 + E.qbar - mu * E.rbar2);
  const real nu = std::max(nuA, nuB);
  E.f = mu - 1 / (nu + mu * E.rbar2);
}

// Auxiliary function whose root bounds the master root from above: mu sqrt(h0^2 + rbar^2(mu)) - 1,
// h0 the minimum enthalpy of the EOS (1 for the ideal gas)
real c2p_aux(const C2PIn& I, real h0, real mu) {
  const real x = 1 / (1 + mu * I.b2);
  const real rbar2 = x * x * I.r2 + mu * x * (1 + x) * I.rb * I.rb;
  return mu * std::sqrt(h0 * h0 + rbar2) - 1;
}

// Illinois (modified regula falsi) on a sign-changing bracket [a,b].  Returns 0 on convergence,
// -1 without a sign change, -2 when max_iter is exhausted.  lo/hi receive the final bracket.
template <class Fn>
int illinois(Fn f, real a, real b, real fa, real fb, real tol, int max_iter, real* root, real* lo,
             real* hi, int* iters) {
  *iters = 0;
  if (fa == 0) { *root = *lo = *hi = a; return 0; }
  if (fb == 0) { *root = *lo = *hi = b; return 0; }
  if ((fa < 0) == (fb < 0)) return -1;
  int side = 0;
  for (int it = 1; it <= max_iter; ++it) {
    real c = (a * fb - b * fa) / (fb - fa);
    if (!(c > a && c < b)) c = 0.5 * (a + b);
    if (!(c > a && c < b)) { *root = c; *lo = a; *hi = b; *iters = it; return 0; }  // bracket at ulp
    const real fc = f(c);
    *iters = it;
    if (fc == 0) { *root = *lo = *hi = c; return 0; }
    if ((fc < 0) == (fa < 0)) {
      a = c; fa = fc;
      if (side == -1) fb *= 0.5;
      side = -1;
    } else {
      b = c; fb = fc;
      if (side == +1) fa *= 0.5;
      side = +1;
    }
    if (b - a <= tol * c) { *root = c; *lo = a; *hi = b; return 0; }
  }
  *lo = a; *hi = b;
  return -2;
}

// Atmosphere primitives (Sec. 3.5, App. A): rho_atm, p_atm, u~ = 0; B untouched.  Table:
// rho_atm, T_atm, Y_e = Y_e,atm, p from the table.
void atmosphere(const oparams& Q, real w[]) {
  w[0] = Q.rho_atm; w[1] = w[2] = w[3] = 0; w[4] = Q.p_atm;
  if (Q.eos) {
    real eps;
    eos_table_rho_T(Q, Q.rho_atm, Q.T_atm, Q.Ye_atm, &w[4], &eps);
    w[5] = Q.Ye_atm;
    w[6] = Q.T_atm;
  }
}

// One cell.  q: densitised (D, S_j, tau) in/out (rewritten when limits or atmosphere apply);
// Bdens: densitised cell-centred B^i; w: prims out.  Returns status bits; *iters = master iterations.
// Invariants and root of the last bracketed solve of con2prim_point (for the learned bracket)
struct C2PRecord {
  real q, r2, b2, rb, mu, D, ye;
  bool solved;
};

int con2prim_point(const PM& M, const oparams& Q, real q[], const real Bdens[3], real w[], int* iters,
                   C2PRecord* rec = nullptr) {
  if (rec) rec->solved = false;
  int st = 0;
  *iters = 0;
  const real sg = M.sqrtg;
  real D = q[0] / sg, tau = q[4] / sg, S[3], Bu[3], Bd[3];
  bool finite = std::isfinite(D) && std::isfinite(tau);
  for (int i = 0; i < 3; ++i) {
    S[i] = q[1 + i] / sg;
    Bu[i] = Bdens[i] / sg;
    finite = finite && std::isfinite(S[i]) && std::isfinite(Bu[i]);
  }
  // table: Y_e = (D Y_e)/D from the conserved pair, moved into the table's range (App. A)
  real ye = 0;
  bool ye_clamped = false;
  if (Q.eos) {
    finite = finite && std::isfinite(q[5]);
    const otable& T = *Q.table;
    const double ylo = T.x0[2], yhi = T.x0[2] + (T.n[2] - 1) * T.dx[2];
    ye = finite && q[0] != 0 ? q[5] / q[0] : real(ylo);
    if (ye < ylo) { ye = ylo; ye_clamped = true; }
    if (ye > yhi) { ye = yhi; ye_clamped = true; }
  }
  // Atmosphere threshold f_thr rho_atm (Sec. 3.5, App. A), widened by the relative band atm_band:
  // cells that sit at the atmosphere density up to rounding are reset deterministically.
  const real rho_thr = Q.f_thr * Q.rho_atm * (1 + Q.atm_band);
  bool atm = false, reprim = false;
  if (!finite) { st |= 2; atm = true; }
  else if (D < rho_thr) { st |= 1; atm = true; }
  if (!atm) {
    for (int i = 0; i < 3; ++i) {
      Bd[i] = 0;
      for (int j = 0; j < 3; ++j) Bd[i] += M.g[i][j] * Bu[j];
    }
    real BB = 0;
    for (int i = 0; i < 3; ++i) BB += Bu[i] * Bd[i];
    bool qmod = false;
    // B^2/D > M_max  ->  D = B^2/M_max  (App. A)
    if (BB > Q.M_max * D) { D = BB / Q.M_max; st |= 16; qmod = true; }
    // tau floor of a static cold fluid with the same field (c16): D eps(rho = D, T_min) + B^2/2,
    // eps(T=0) = 0 for the ideal gas, the table's lowest temperature for a table
    real eps_min = 0;
    if (Q.eos) {
      real pm;
      eos_table_rho_T(Q, D, std::exp(Q.table->x0[1]), ye, &pm, &eps_min);
    }
    const real tau_min = D * eps_min + 0.5 * BB;
    if (tau < tau_min) { tau = tau_min; st |= 8; qmod = true; }
    C2PIn I;
    I.D = D;
    I.q = tau / D;
    I.ye = ye;
    real r_d[3], r_u[3], bb_u[3];
    for (int i = 0; i < 3; ++i) { r_d[i] = S[i] / D; bb_u[i] = Bu[i] / std::sqrt(D); }
    I.r2 = 0; I.rb = 0;
    for (int i = 0; i < 3; ++i) {
      r_u[i] = 0;
      for (int j = 0; j < 3; ++j) r_u[i] += M.gu[i][j] * r_d[j];
    }
    for (int i = 0; i < 3; ++i) { I.r2 += r_d[i] * r_u[i]; I.rb += r_d[i] * bb_u[i]; }
    I.b2 = BB / D;
    // bracket (0, mu+], mu+ from the auxiliary function on (0, 1/h0]
    const real h0 = Q.eos ? real(Q.h0) : real(1);
    const real mu_top = 1 / h0;
    real mup = mu_top, root, lo, hi;
    int it_aux = 0;
    {
      auto fa = [&](real mu) { return c2p_aux(I, h0, mu); };
      const real f1 = fa(mu_top);
      if (f1 > 0) {
        int r = illinois(fa, 0.0, mu_top, -1.0, f1, 1e-3, Q.max_iter, &root, &lo, &hi, &it_aux);
        if (r == 0) mup = hi;
      }
    }
    C2PEval E;
    auto fm = [&](real mu) { c2p_eval(Q, I, mu, E); return E.f; };
    real f0 = fm(0.0), fp = fm(mup);
    if ((f0 < 0) == (fp < 0) && mup < mu_top) { mup = mu_top; fp = fm(mup); }
    int r = illinois(fm, 0.0, mup, f0, fp, Q.tol, Q.max_iter, &root, &lo, &hi, iters);
    if (r != 0) { st |= 2; atm = true; }
    else {
      const real mu = root;
      if (rec) { rec->q = I.q; rec->r2 = I.r2; rec->b2 = I.b2; rec->rb = I.rb; rec->mu = mu; rec->D = D;
                 rec->ye = ye; rec->solved = true; }
      c2p_eval(Q, I, mu, E);
      // v^i = mu x (r^i + mu (r.calb) calb^i)
      real v_u[3];
      for (int i = 0; i < 3; ++i) v_u[i] = mu * E.x * (r_u[i] + mu * I.rb * bb_u[i]);
      if (E.vcap) {
        st |= 4;
        const real s = std::sqrt(E.v2 / (mu * mu * E.rbar2));
        for (int i = 0; i < 3; ++i) v_u[i] *= s;
        if (Q.ceiling == 1) atm = true;
      }
      if (E.eclamp || ye_clamped) st |= 32;
      if (E.rho < rho_thr) { st |= 1; atm = true; }
      if (!atm) {
        w[0] = E.rho;
        for (int i = 0; i < 3; ++i) w[1 + i] = E.W * v_u[i];
        w[4] = E.p;
        if (Q.eos) {
          w[5] = ye;
          w[6] = E.T;
          // temperature floor (App. A): T < T_atm -> T_atm, p recomputed, conserved rebuilt
          if (E.T < Q.T_atm) {
            real eps;
            eos_table_rho_T(Q, E.rho, Q.T_atm, ye, &w[4], &eps);
            w[6] = Q.T_atm;
            st |= 32;
            reprim = true;
          }
          if (ye_clamped) qmod = true;
        }
        if (qmod) {
          q[0] = sg * D; q[4] = sg * tau;
          if (Q.eos) q[5] = q[0] * ye;
        }
      }
    }
  }
  if (atm) atmosphere(Q, w);
  if (atm || reprim) {
    FP F;
    fluid_point(M, Q, w, Bdens, F);
    cons_all(Q, M, F, q);
  }
  return st;
}

// ------------------------------------------------------------------------------------------------
// The stage on one block (steps a1-a8 of the hot path, c12 semantics)
// ------------------------------------------------------------------------------------------------
struct Arr {  // zero-initialised scratch
  std::vector<real> a;
  explicit Arr(long n) : a(n, 0.0) {}
  real& operator[](long i) { return a[i]; }
  real operator[](long i) const { return a[i]; }
};

inline void load16(const double* const* mv, long vi, real m[16]) {
  for (int c = 0; c < 16; ++c) m[c] = mv[c][vi];
}

}  // namespace

#ifndef ORACLE_COUNT_FLOPS
namespace {
// ------------------------------------------------------------------------------------------------
// Learned con2prim bracket (not in the paper): features, training target, and a 6-64-64-1 tanh
// MLP with its mean-squared-error gradient by plain backpropagation, all in FP64.
//
// Parameter vector (the layout documented for the library's gr_mlp_* calls):
//   [0..5] feature means, [6..11] feature inverse standard deviations, [12] target mean,
//   [13] target standard deviation, [14] first bracket step in log mu, [15] unused,
//   [16..]  W1 (64 x 6), b1 (64), W2 (64 x 64), b2 (64), W3 (64), b3 (1), row-major (out, in).
// Features of a solved cell: log(1+q), log(1+r^2), log(1+calb^2), (r.calb)^2 / (r^2 calb^2) (0 if
// either vanishes), and for a table log D~ and Y_e (0, 0 for the scale-free ideal gas); target:
// log mu at the root.
// ------------------------------------------------------------------------------------------------
static const int MLP_H = 64, MLP_IN = 6, MLP_OFF = 16;
static const int MLP_NW = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;
static const int MLP_MEAN = 0, MLP_ISTD = 6, MLP_TMEAN = 12, MLP_TSTD = 13;

void c2p_features(const oparams& Q, const C2PRecord& r, double f[MLP_IN]) {
  f[0] = std::log1p(to_d(r.q));
  f[1] = std::log1p(to_d(r.r2));
  f[2] = std::log1p(to_d(r.b2));
  const double den = to_d(r.r2) * to_d(r.b2);
  f[3] = den > 0 ? to_d(r.rb) * to_d(r.rb) / den : 0.0;
  f[4] = Q.eos ? std::log(to_d(r.D)) : 0.0;
  f[5] = Q.eos ? to_d(r.ye) : 0.0;
}

// z (normalised output) and hidden activations of one sample
void mlp_forward1(const double* P, const double* x, double h1[64], double h2[64], double* z) {
  const double* W1 = P + MLP_OFF;
  const double* b1 = W1 + MLP_H * MLP_IN;
  const double* W2 = b1 + MLP_H;
  const double* b2 = W2 + MLP_H * MLP_H;
  const double* W3 = b2 + MLP_H;
  const double* b3 = W3 + MLP_H;
  double xn[MLP_IN];
  for (int j = 0; j < MLP_IN; ++j) xn[j] = (x[j] - P[MLP_MEAN + j]) * P[MLP_ISTD + j];
  for (int i = 0; i < MLP_H; ++i) {
    double a = b1[i];
    for (int j = 0; j < MLP_IN; ++j) a += W1[i * MLP_IN + j] * xn[j];
    h1[i] = std::tanh(a);
  }
  for (int i = 0; i < MLP_H; ++i) {
    double a = b2[i];
    for (int j = 0; j < MLP_H; ++j) a += W2[i * MLP_H + j] * h1[j];
    h2[i] = std::tanh(a);
  }
  double a = b3[0];
  for (int j = 0; j < MLP_H; ++j) a += W3[j] * h2[j];
  *z = a;
}

}  // namespace

extern "C" {
// Features and log(mu) of the bracketed con2prim solve at np points (valid[n] = 0 when the cell was
// not solved: atmosphere, failure).
// q: np x 5 (ideal gas) or np x 6 (table).
void oracle_c2p_samples(int np, const double* metric, const double* q, const double* Bdens, const oparams* Q,
                        double* feats, double* target, uint8_t* valid) {
  const int nq = Q->eos ? 6 : 5;
  for (int n = 0; n < np; ++n) {
    PM M;
    pm_from16(metric + 16 * n, M);
    real qq[6], w[7];
    for (int v = 0; v < nq; ++v) qq[v] = q[nq * n + v];
    int it;
    C2PRecord rec;
    con2prim_point(M, *Q, qq, Bdens + 3 * n, w, &it, &rec);
    valid[n] = rec.solved ? 1 : 0;
    if (rec.solved) {
      c2p_features(*Q, rec, feats + MLP_IN * n);
      target[n] = std::log(rec.mu);
    } else {
      for (int j = 0; j < MLP_IN; ++j) feats[MLP_IN * n + j] = 0;
      target[n] = 0;
    }
  }
}

int oracle_mlp_nparam(void) { return MLP_OFF + MLP_NW; }

// Predicted log(mu) at n feature vectors
void oracle_mlp_forward(const double* P, const double* x, int n, double* t) {
  double h1[64], h2[64], z;
  for (int s = 0; s < n; ++s) {
    mlp_forward1(P, x + MLP_IN * s, h1, h2, &z);
    t[s] = P[MLP_TMEAN] + P[MLP_TSTD] * z;
  }
}

// loss = mean over samples of (z - zt)^2 / 2 with zt = (t - P[8]) / P[9]; grad (MLP_NW) with respect
// to the network weights (the normalisation entries are constants)
void oracle_mlp_loss_grad(const double* P, const double* x, const double* t, int n, double* grad, double* loss) {
  const double* W2 = P + MLP_OFF + MLP_H * MLP_IN + MLP_H;
  const double* W3 = W2 + MLP_H * MLP_H + MLP_H;
  double* gW1 = grad;
  double* gb1 = gW1 + MLP_H * MLP_IN;
  double* gW2 = gb1 + MLP_H;
  double* gb2 = gW2 + MLP_H * MLP_H;
  double* gW3 = gb2 + MLP_H;
  double* gb3 = gW3 + MLP_H;
  for (int k = 0; k < MLP_NW; ++k) grad[k] = 0;
  double L = 0;
  for (int s = 0; s < n; ++s) {
    const double* xs = x + MLP_IN * s;
    double h1[64], h2[64], z;
    mlp_forward1(P, xs, h1, h2, &z);
    const double zt = (t[s] - P[MLP_TMEAN]) / P[MLP_TSTD];
    const double dz = (z - zt) / n;
    L += 0.5 * (z - zt) * (z - zt) / n;
    double xn[MLP_IN];
    for (int j = 0; j < MLP_IN; ++j) xn[j] = (xs[j] - P[MLP_MEAN + j]) * P[MLP_ISTD + j];
    // output layer
    double g2[64];
    for (int j = 0; j < MLP_H; ++j) {
      gW3[j] += dz * h2[j];
      g2[j] = dz * W3[j] * (1 - h2[j] * h2[j]);
    }
    gb3[0] += dz;
    // second hidden layer
    double g1[64];
    for (int j = 0; j < MLP_H; ++j) g1[j] = 0;
    for (int i = 0; i < MLP_H; ++i) {
      gb2[i] += g2[i];
      for (int j = 0; j < MLP_H; ++j) {
        gW2[i * MLP_H + j] += g2[i] * h1[j];
        g1[j] += W2[i * MLP_H + j] * g2[i];
      }
    }
    // first hidden layer
    for (int i = 0; i < MLP_H; ++i) {
      const double gi = g1[i] * (1 - h1[i] * h1[i]);
      gb1[i] += gi;
      for (int j = 0; j < MLP_IN; ++j) gW1[i * MLP_IN + j] += gi * xn[j];
    }
  }
  *loss = L;
}
}  // extern "C"
#endif

#ifdef ORACLE_COUNT_FLOPS
OpCount g_ops;
namespace {
OpCount g_phase[8];
void phase_mark(int k, OpCount& last) {
  g_phase[k].add += g_ops.add - last.add; g_phase[k].mul += g_ops.mul - last.mul;
  g_phase[k].div += g_ops.div - last.div; g_phase[k].sqrt += g_ops.sqrt - last.sqrt;
  g_phase[k].cmp += g_ops.cmp - last.cmp;
  last = g_ops;
}
// con2prim of cells that take the atmosphere branch before any root find (no iteration): their
// operations are moved from phase 6 to phase 7, so the two kinds of cell can be told apart
OpCount g_c2p_cell_start, g_c2p_atm;
void c2p_cell_begin() { g_c2p_cell_start = g_ops; }
void c2p_cell_end(int iterations) {
  if (iterations != 0) return;
  g_c2p_atm.add += g_ops.add - g_c2p_cell_start.add; g_c2p_atm.mul += g_ops.mul - g_c2p_cell_start.mul;
  g_c2p_atm.div += g_ops.div - g_c2p_cell_start.div; g_c2p_atm.sqrt += g_ops.sqrt - g_c2p_cell_start.sqrt;
  g_c2p_atm.cmp += g_ops.cmp - g_c2p_cell_start.cmp;
}
void c2p_split() {
  g_phase[6].add -= g_c2p_atm.add; g_phase[6].mul -= g_c2p_atm.mul; g_phase[6].div -= g_c2p_atm.div;
  g_phase[6].sqrt -= g_c2p_atm.sqrt; g_phase[6].cmp -= g_c2p_atm.cmp;
  g_phase[7].add += g_c2p_atm.add; g_phase[7].mul += g_c2p_atm.mul; g_phase[7].div += g_c2p_atm.div;
  g_phase[7].sqrt += g_c2p_atm.sqrt; g_phase[7].cmp += g_c2p_atm.cmp;
  g_c2p_atm = OpCount();
}
}  // namespace
#define ORACLE_PHASE(k) phase_mark(k, ops_last)
#define ORACLE_C2P_CELL_BEGIN() c2p_cell_begin()
#define ORACLE_C2P_CELL_END(it) c2p_cell_end(it)
#define ORACLE_C2P_SPLIT() c2p_split()
#else
#define ORACLE_PHASE(k)
#define ORACLE_C2P_CELL_BEGIN()
#define ORACLE_C2P_CELL_END(it)
#define ORACLE_C2P_SPLIT()
#endif

extern "C" {

#ifndef ORACLE_COUNT_FLOPS
// Primitive -> conserved at np points.  metric: np x 16, Bdens: np x 3; prims np x 5 and q np x 5
// (ideal gas) or prims np x 7 (rho, u~^i, p, Y_e, T; T unread) and q np x 6 (table).
void oracle_prim2con(int np, const double* metric, const double* prims, const double* Bdens,
                     const oparams* Q, double* q) {
  const int nw = Q->eos ? 7 : 5, nq = Q->eos ? 6 : 5;
  for (int n = 0; n < np; ++n) {
    PM M;
    pm_from16(metric + 16 * n, M);
    FP F;
    fluid_point(M, *Q, prims + nw * n, Bdens + 3 * n, F);
    cons_all(*Q, M, F, q + nq * n);
  }
}

// Conserved -> primitive at np points (layouts as oracle_prim2con).  q is rewritten in place when a
// limit or the atmosphere applies.
void oracle_con2prim(int np, const double* metric, double* q, const double* Bdens, const oparams* Q,
                     double* prims, uint8_t* status, int32_t* iters) {
  const int nw = Q->eos ? 7 : 5, nq = Q->eos ? 6 : 5;
  for (int n = 0; n < np; ++n) {
    PM M;
    pm_from16(metric + 16 * n, M);
    int it;
    status[n] = (uint8_t)con2prim_point(M, *Q, q + nq * n, Bdens + 3 * n, prims + nw * n, &it);
    if (iters) iters[n] = it;
  }
}

// Table lookups at np points for the pins: out[4n..4n+3] = p(rho, T, Y_e), eps(rho, T, Y_e),
// c_s^2(rho, T, Y_e) and the temperature recovered from (rho, that p, Y_e).
void oracle_table_eval(int np, const oparams* Q, const double* rho, const double* T, const double* ye,
                       double* out) {
  for (int n = 0; n < np; ++n) {
    real p, eps;
    eos_table_rho_T(*Q, rho[n], T[n], ye[n], &p, &eps);
    Thermo th;
    eos_from_rho_p(*Q, rho[n], p, ye[n], th);
    out[4 * n + 0] = to_d(p);
    out[4 * n + 1] = to_d(eps);
    out[4 * n + 2] = to_d(th.cs2);
    out[4 * n + 3] = to_d(th.T);
  }
}

// Minimum over the table's nodes of the specific enthalpy h = (e + p)/rho (the h0 of the bracket)
double oracle_table_hmin(const otable* T) {
  double hmin = HUGE_VAL;
  for (int iy = 0; iy < T->n[2]; ++iy)
    for (int iT = 0; iT < T->n[1]; ++iT)
      for (int ir = 0; ir < T->n[0]; ++ir) {
        const long k = tab_idx(*T, ir, iT, iy);
        const double lr = T->x0[0] + ir * T->dx[0];
        const double h = std::exp(T->le[k] - lr) + std::exp(T->lp[k] - lr);
        if (h < hmin) hmin = h;
      }
  return hmin;
}

// Physical state at np points in direction d: cons U (5 + 2 transverse B), flux F (5 + 2), speeds.
void oracle_flux_points(int np, int d, const double* metric, const double* prims, const double* Bdens,
                        const oparams* Q, double* U, double* F, double* lam) {
  const int nw = Q->eos ? 7 : 5;
  for (int n = 0; n < np; ++n) {
    PM M;
    pm_from16(metric + 16 * n, M);
    FP P;
    fluid_point(M, *Q, prims + nw * n, Bdens + 3 * n, P);
    real q[7], f[7];
    cons_from_fp(M, P, q);
    q[5] = P.Bd_u[(d + 1) % 3];
    q[6] = P.Bd_u[(d + 2) % 3];
    flux_from_fp(M, P, q, d, f, f + 5);
    for (int v = 0; v < 7; ++v) { U[7 * n + v] = q[v]; F[7 * n + v] = f[v]; }
    speeds_from_fp(M, *Q, P, d, &lam[2 * n], &lam[2 * n + 1]);
  }
}

// HLLE face flux from left/right prims at np faces.  Out: F (np x 7): 5 conserved, 2 induction; with
// a table F (np x 8), the D Y_e flux last, and prims np x 7.
void oracle_face_flux(int np, int d, const double* metric, const double* wL, const double* BL,
                      const double* wR, const double* BR, const oparams* Q, double* F) {
  const int nw = Q->eos ? 7 : 5, nf = Q->eos ? 8 : 7;
  for (int n = 0; n < np; ++n) {
    PM M;
    pm_from16(metric + 16 * n, M);
    real fq[6], fb[2];
    face_flux(M, *Q, d, wL + nw * n, BL + 3 * n, wR + nw * n, BR + 3 * n, fq, fb);
    for (int v = 0; v < 5; ++v) F[nf * n + v] = to_d(fq[v]);
    F[nf * n + 5] = to_d(fb[0]);
    F[nf * n + 6] = to_d(fb[1]);
    if (Q->eos) F[nf * n + 7] = to_d(fq[5]);
  }
}

// Source terms at np points.  dmetric: np x 3 x 16 (d_k of each metric component).
void oracle_sources(int np, const double* metric, const double* dmetric, const double* prims,
                    const double* Bdens, const oparams* Q, double* s) {
  const int nw = Q->eos ? 7 : 5;
  for (int n = 0; n < np; ++n) {
    PM M;
    pm_from16(metric + 16 * n, M);
    FP P;
    fluid_point(M, *Q, prims + nw * n, Bdens + 3 * n, P);
    real dm[3][16];
    for (int k = 0; k < 3; ++k)
      for (int c = 0; c < 16; ++c) dm[k][c] = dmetric[48 * n + 16 * k + c];
    sources(M, P, dm, s + 5 * n);
  }
}

// Reconstruction along a 1D array of nc cells: faces f = 3..nc-3 (between cells f-1 and f).
void oracle_recon1d(int method, int nc, const double* w, double eps, double* L, double* R) {
  for (int f = 3; f <= nc - 3; ++f) {
    real s[6];
    for (int t = 0; t < 6; ++t) s[t] = w[f - 3 + t];
    recon_face(method, s, eps, &L[f], &R[f]);
  }
}

// Metric interpolation on one block: values at cell centres and derivatives there (cells with
// index in [lo, hi) in each direction), and values at the centres of d-faces.
void oracle_interp_cells(const ob_geom* G, const double* metric, int order, const int32_t* lo,
                         const int32_t* hi, double* val, double* dval) {
  Blk b(G);
  const double* mv[16];
  for (int c = 0; c < 16; ++c) mv[c] = metric + c * b.nvert();
  long n = 0;
  for (int k = lo[2]; k < hi[2]; ++k)
    for (int j = lo[1]; j < hi[1]; ++j)
      for (int i = lo[0]; i < hi[0]; ++i, ++n) {
        real o[16];
        interp_cell(b, mv, order, i, j, k, -1, o);
        for (int c = 0; c < 16; ++c) val[16 * n + c] = o[c];
        for (int e = 0; e < 3; ++e) {
          interp_cell(b, mv, order, i, j, k, e, o);
          for (int c = 0; c < 16; ++c) dval[48 * n + 16 * e + c] = o[c];
        }
      }
}
void oracle_interp_faces(const ob_geom* G, const double* metric, int order, int d, const int32_t* lo,
                         const int32_t* hi, double* val) {
  Blk b(G);
  const double* mv[16];
  for (int c = 0; c < 16; ++c) mv[c] = metric + c * b.nvert();
  long n = 0;
  int p[3];
  for (p[2] = lo[2]; p[2] < hi[2]; ++p[2])
    for (p[1] = lo[1]; p[1] < hi[1]; ++p[1])
      for (p[0] = lo[0]; p[0] < hi[0]; ++p[0], ++n) {
        real o[16];
        interp_face(b, mv, order, d, p, o);
        for (int c = 0; c < 16; ++c) val[16 * n + c] = o[c];
      }
}

#else
// Operation counts per phase of the stage accumulated since the last reset:
// out[5*k + {0,1,2,3,4}] = (add, mul, div, sqrt, cmp) of phase k, k = 0..7:
//   0 cell metric + cell field, 1 faces (reconstruction, face metric, HLLE), 2 cell electric field,
//   3 corner EMFs, 4 flux divergence + sources + update, 5 CT face update, 6 con2prim of the cells
//   that run the root find, 7 con2prim of the cells reset to the atmosphere without one
void oracle_flops_get(double* out, int reset) {
  for (int k = 0; k < 8; ++k) {
    out[5 * k + 0] = g_phase[k].add; out[5 * k + 1] = g_phase[k].mul; out[5 * k + 2] = g_phase[k].div;
    out[5 * k + 3] = g_phase[k].sqrt; out[5 * k + 4] = g_phase[k].cmp;
    if (reset) g_phase[k] = OpCount();
  }
}
#endif

// One Runge-Kutta stage on one MeshBlock.
//   metric: 16 vertex arrays; W: 5 cell arrays (stage-input prims, ghosts filled); B: 3 face arrays
//   (densitised, ghosts filled); U, U0: 5 cell arrays (interior read); B0: 3 face arrays.
//   With a table: W has 7 arrays (rho, u~^i, p, Y_e, T; T unread) and U, U0, Uo 6 (D Y_e last).
//   Out: Uo (interior cells), Bo (interior faces), Wo (interior prims), status (interior cells).
// Returns 0, or -1 when the ghost width is too small for the stencil.
int oracle_stage_block_ex(const ob_geom* G, const double* metric, const double* W, const double* Bx,
                          const double* By, const double* Bz, const double* U, const double* U0,
                          const double* B0x, const double* B0y, const double* B0z, double dt,
                          const oparams* Qp, double* Uo, double* Box, double* Boy, double* Boz, double* Wo,
                          uint8_t* status, int32_t* iters, double* flux_out, double* emf_out,
                          const double* flux_in, const double* emf_in);

int oracle_stage_block(const ob_geom* G, const double* metric, const double* W, const double* Bx,
                       const double* By, const double* Bz, const double* U, const double* U0,
                       const double* B0x, const double* B0y, const double* B0z, double dt,
                       const oparams* Qp, double* Uo, double* Box, double* Boy, double* Boz, double* Wo,
                       uint8_t* status, int32_t* iters) {
  return oracle_stage_block_ex(G, metric, W, Bx, By, Bz, U, U0, B0x, B0y, B0z, dt, Qp, Uo, Box, Boy, Boz, Wo, status,
                               iters, nullptr, nullptr, nullptr, nullptr);
}

// The stage of one block, with the face fluxes and corner EMFs exposed for the level-boundary
// corrections of a refined mesh (Sec. 3.3, last paragraph): flux_out / emf_out (if not NULL) receive the
// block's fluxes (for d = 0..2, for each conserved variable v, the block's d-face array) and corner
// EMFs (E_m for m = 0..2, each vertex-indexed by the edge's low corner); flux_in / emf_in (if not
// NULL, same layouts) replace them before the cell update and the CT update.
int oracle_stage_block_ex(const ob_geom* G, const double* metric, const double* W, const double* Bx,
                          const double* By, const double* Bz, const double* U, const double* U0,
                          const double* B0x, const double* B0y, const double* B0z, double dt,
                          const oparams* Qp, double* Uo, double* Box, double* Boy, double* Boz, double* Wo,
                          uint8_t* status, int32_t* iters, double* flux_out, double* emf_out,
                          const double* flux_in, const double* emf_in) {
  const oparams& Q = *Qp;
  Blk b(G);
  const int g = b.g;
  const int need = (Q.recon == 0 ? 2 : 3) + (Q.interp_order == 4 ? 1 : 0);
  if (g < need) return -1;
  const long NC = b.ncell();
  const int nq = Q.eos ? 6 : 5, nw = Q.eos ? 7 : 5;
  const int nrec = Q.eos ? 8 : 7;   // reconstructed: rho, u~^i, p, calB^{t1}, calB^{t2}[, Y_e]
  const double* mv[16];
  for (int c = 0; c < 16; ++c) mv[c] = metric + c * b.nvert();
  const double* Bf[3] = {Bx, By, Bz};
  const double* B0f[3] = {B0x, B0y, B0z};
  double* Bof[3] = {Box, Boy, Boz};
  const int lo_c = (Q.interp_order == 4) ? -g + 1 : -g;   // cells whose metric is computable
  const int hi_off = (Q.interp_order == 4) ? g - 1 : g;   // ... up to n + hi_off - 1

#ifdef ORACLE_COUNT_FLOPS
  OpCount ops_last = g_ops;
#endif
  // a1: metric at cell centres (all computable cells); sqrt(gamma) kept per cell
  std::vector<PM> cm(NC);
  for (int k = lo_c; k < b.n[2] + hi_off; ++k)
    for (int j = lo_c; j < b.n[1] + hi_off; ++j)
      for (int i = lo_c; i < b.n[0] + hi_off; ++i) {
        real m[16];
        interp_cell(b, mv, Q.interp_order, i, j, k, -1, m);
        pm_from16(m, cm[b.c(i, j, k)]);
      }
  // a2: cell-centred field, densitised mean of the two faces; calB = that / sqrt(gamma_cc)  (c8)
  Arr Bcc[3] = {Arr(NC), Arr(NC), Arr(NC)};   // densitised
  for (int k = lo_c; k < b.n[2] + hi_off; ++k)
    for (int j = lo_c; j < b.n[1] + hi_off; ++j)
      for (int i = lo_c; i < b.n[0] + hi_off; ++i) {
        const int p[3] = {i, j, k};
        for (int d = 0; d < 3; ++d) {
          int q2[3] = {i, j, k};
          q2[d] += 1;
          Bcc[d][b.c(i, j, k)] = 0.5 * (Bf[d][fidx(b, d, p)] + Bf[d][fidx(b, d, q2)]);
        }
      }

  ORACLE_PHASE(0);
  // a3 + a4: face fluxes on d-faces with normal index 0..n_d and transverse index -1..n_t
  std::vector<Arr> Fq[3], Fb[3];
  for (int d = 0; d < 3; ++d) {
    Fq[d].assign(nq, Arr(b.nface(d)));
    Fb[d].assign(2, Arr(b.nface(d)));
  }
  for (int d = 0; d < 3; ++d) {
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    int p[3];
    int lo[3], hi[3];
    for (int e = 0; e < 3; ++e) { lo[e] = -1; hi[e] = b.n[e] + 1; }
    lo[d] = 0; hi[d] = b.n[d] + 1;
    for (p[2] = lo[2]; p[2] < hi[2]; ++p[2])
      for (p[1] = lo[1]; p[1] < hi[1]; ++p[1])
        for (p[0] = lo[0]; p[0] < hi[0]; ++p[0]) {
          // stencil cells along d: p[d]-3 .. p[d]+2
          real wL[7], wR[7], cL[2], cR[2];
          real st[6];
          int q[3] = {p[0], p[1], p[2]};
          real w1[8][6];  // variables x stencil: rho, u~^3, p, calB^{t1}, calB^{t2}[, Y_e]
          for (int t = 0; t < 6; ++t) {
            q[d] = p[d] - 3 + t;
            const bool inside = (q[d] >= -g && q[d] < b.n[d] + g);
            if (!inside) { for (int v = 0; v < nrec; ++v) w1[v][t] = 0; continue; }
            const long ci = cidx(b, q);
            for (int v = 0; v < 5; ++v) w1[v][t] = W[v * NC + ci];
            const real sgc = cm[ci].sqrtg;
            w1[5][t] = Bcc[t1][ci] / sgc;
            w1[6][t] = Bcc[t2][ci] / sgc;
            if (Q.eos) w1[7][t] = W[5 * NC + ci];
          }
          real Lv[8], Rv[8];
          for (int v = 0; v < nrec; ++v) {
            for (int t = 0; t < 6; ++t) st[t] = w1[v][t];
            recon_face(Q.recon, st, Q.weno_eps, &Lv[v], &Rv[v]);
          }
          // c6: a non-physical reconstructed state (rho <= 0 or p <= 0) drops both sides of the
          // face to first order
          if (!(Lv[0] > 0) || !(Rv[0] > 0) || !(Lv[4] > 0) || !(Rv[4] > 0))
            for (int v = 0; v < nrec; ++v) { Lv[v] = w1[v][2]; Rv[v] = w1[v][3]; }
          for (int v = 0; v < 5; ++v) { wL[v] = Lv[v]; wR[v] = Rv[v]; }
          if (Q.eos) { wL[5] = Lv[7]; wR[5] = Rv[7]; }
          cL[0] = Lv[5]; cL[1] = Lv[6]; cR[0] = Rv[5]; cR[1] = Rv[6];
          real m[16];
          interp_face(b, mv, Q.interp_order, d, p, m);
          PM M;
          pm_from16(m, M);
          // c7: transverse field reconstructed undensitised, normal field is the face value
          real BL[3], BR[3];
          const real Bn = Bf[d][fidx(b, d, p)];
          BL[d] = BR[d] = Bn;
          BL[t1] = cL[0] * M.sqrtg; BL[t2] = cL[1] * M.sqrtg;
          BR[t1] = cR[0] * M.sqrtg; BR[t2] = cR[1] * M.sqrtg;
          real fq[6], fb[2];
          face_flux(M, Q, d, wL, BL, wR, BR, fq, fb);
          const long fi = fidx(b, d, p);
          for (int v = 0; v < nq; ++v) Fq[d][v][fi] = fq[v];
          Fb[d][0][fi] = fb[0];
          Fb[d][1][fi] = fb[1];
        }
  }

  ORACLE_PHASE(1);
  // a5: cell-centred E_m = alpha (v~^b B^a - v~^a B^b), (a,b,m) cyclic, on cells -1..n
  Arr Ecc[3] = {Arr(NC), Arr(NC), Arr(NC)};
  for (int k = -1; k <= b.n[2]; ++k)
    for (int j = -1; j <= b.n[1]; ++j)
      for (int i = -1; i <= b.n[0]; ++i) {
        const long ci = b.c(i, j, k);
        real w[7], Bd[3];
        for (int v = 0; v < nw; ++v) w[v] = W[v * NC + ci];
        for (int e = 0; e < 3; ++e) Bd[e] = Bcc[e][ci];
        FP F;
        fluid_point(cm[ci], Q, w, Bd, F);
        for (int m = 0; m < 3; ++m) {
          const int a = (m + 1) % 3, bb = (m + 2) % 3;
          Ecc[m][ci] = cm[ci].alpha * (F.vt_u[bb] * Bd[a] - F.vt_u[a] * Bd[bb]);
        }
      }
  ORACLE_PHASE(2);
  // a5: edge E_m at (a-face ia, b-face ib, m-cell im).  From an a-face E_m = -F^a_{B^b} (Fb[a][0]);
  // from a b-face E_m = +F^b_{B^a} (Fb[bb][1]).  Gardiner-Stone corner average (c9).
  std::vector<Arr> Ee;
  Ee.assign(3, Arr(b.nvert()));   // indexed like vertices (edge low corner), sized generously
  for (int m = 0; m < 3; ++m) {
    const int a = (m + 1) % 3, bb = (m + 2) % 3;
    int e[3];
    int hi[3];
    for (int t = 0; t < 3; ++t) hi[t] = b.n[t] + 1;
    hi[m] = b.n[m];
    for (e[2] = 0; e[2] < hi[2]; ++e[2])
      for (e[1] = 0; e[1] < hi[1]; ++e[1])
        for (e[0] = 0; e[0] < hi[0]; ++e[0]) {
          // index of the point with coordinate ja along a, jb along b and e[m] along m
          const int ia = e[a], ib = e[bb];
          auto at = [&](int ja, int jb, int r[3]) { r[a] = ja; r[bb] = jb; r[m] = e[m]; };
          int r[3];
          auto Ea = [&](int jb) { at(ia, jb, r); return -Fb[a][0][b.f(a, r[0], r[1], r[2])]; };
          auto Eb = [&](int ja) { at(ja, ib, r); return Fb[bb][1][b.f(bb, r[0], r[1], r[2])]; };
          auto Ec = [&](int ja, int jb) { at(ja, jb, r); return Ecc[m][b.c(r[0], r[1], r[2])]; };
          auto Va = [&](int jb) { at(ia, jb, r); return Fq[a][0][b.f(a, r[0], r[1], r[2])]; };
          auto Vb = [&](int ja) { at(ja, ib, r); return Fq[bb][0][b.f(bb, r[0], r[1], r[2])]; };
          const real avg = 0.25 * (Ea(ib) + Ea(ib - 1) + Eb(ia) + Eb(ia - 1));
          if (Q.emf == 1) { Ee[m][b.v(e[0], e[1], e[2])] = avg; continue; }
          auto upw = [](real vel, real lowside, real highside) {
            return vel > 0 ? lowside : (vel < 0 ? highside : 0.5 * (lowside + highside));
          };
          // (db/2) dE/db on the a-face line, upwinded by the mass flux through that a-face
          const real db_hi = upw(Va(ib), Ec(ia - 1, ib) - Eb(ia - 1), Ec(ia, ib) - Eb(ia));
          const real db_lo = upw(Va(ib - 1), Eb(ia - 1) - Ec(ia - 1, ib - 1), Eb(ia) - Ec(ia, ib - 1));
          // (da/2) dE/da on the b-face line, upwinded by the mass flux through that b-face
          const real da_hi = upw(Vb(ia), Ec(ia, ib - 1) - Ea(ib - 1), Ec(ia, ib) - Ea(ib));
          const real da_lo = upw(Vb(ia - 1), Ea(ib - 1) - Ec(ia - 1, ib - 1), Ea(ib) - Ec(ia - 1, ib));
          Ee[m][b.v(e[0], e[1], e[2])] = avg + 0.25 * (db_lo - db_hi) + 0.25 * (da_lo - da_hi);
        }
  }

  {
    long off = 0;
    for (int d = 0; d < 3; ++d)
      for (int v = 0; v < nq; ++v, off += b.nface(d))
        for (long f = 0; f < b.nface(d); ++f) {
          if (flux_out) flux_out[off + f] = to_d(Fq[d][v][f]);
          if (flux_in) Fq[d][v][f] = flux_in[off + f];
        }
    for (int m = 0; m < 3; ++m)
      for (long e = 0; e < b.nvert(); ++e) {
        if (emf_out) emf_out[m * b.nvert() + e] = to_d(Ee[m][e]);
        if (emf_in) Ee[m][e] = emf_in[m * b.nvert() + e];
      }
  }

  ORACLE_PHASE(3);
  // a6: cell update with flux divergence and sources (stage-input prims), Eq. claw
  for (int k = 0; k < b.n[2]; ++k)
    for (int j = 0; j < b.n[1]; ++j)
      for (int i = 0; i < b.n[0]; ++i) {
        const long ci = b.c(i, j, k);
        real w[7], Bd[3];
        for (int v = 0; v < nw; ++v) w[v] = W[v * NC + ci];
        for (int e = 0; e < 3; ++e) Bd[e] = Bcc[e][ci];
        FP F;
        fluid_point(cm[ci], Q, w, Bd, F);
        real dm[3][16];
        for (int e = 0; e < 3; ++e) interp_cell(b, mv, Q.interp_order, i, j, k, e, dm[e]);
        real s[6];
        sources(cm[ci], F, dm, s);
        s[5] = 0;   // D Y_e has no source (Sec. 2.2.1)
        for (int v = 0; v < nq; ++v) {
          real divF = 0;
          for (int d = 0; d < 3; ++d) {
            int p[3] = {i, j, k}, p1[3] = {i, j, k};
            p1[d] += 1;
            divF += (Fq[d][v][fidx(b, d, p1)] - Fq[d][v][fidx(b, d, p)]) / b.dx[d];
          }
          Uo[v * NC + ci] = to_d(Q.rk_g0 * U0[v * NC + ci] + Q.rk_g1 * U[v * NC + ci] +
                                 Q.rk_beta * dt * (-divF + s[v]));
        }
      }

  ORACLE_PHASE(4);
  // a7: constrained-transport face update, B'^d = g0 B0 + g1 B - beta dt (curl E)_d
  for (int d = 0; d < 3; ++d) {
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    int p[3];
    int hi[3] = {b.n[0], b.n[1], b.n[2]};
    hi[d] += 1;
    for (p[2] = 0; p[2] < hi[2]; ++p[2])
      for (p[1] = 0; p[1] < hi[1]; ++p[1])
        for (p[0] = 0; p[0] < hi[0]; ++p[0]) {
          int a1[3] = {p[0], p[1], p[2]}, a2[3] = {p[0], p[1], p[2]};
          a1[t1] += 1; a2[t2] += 1;
          // E_{t2} edges at t1 = p, p+1 ; E_{t1} edges at t2 = p, p+1
          const real dE2 = (Ee[t2][b.v(a1[0], a1[1], a1[2])] - Ee[t2][b.v(p[0], p[1], p[2])]) / b.dx[t1];
          const real dE1 = (Ee[t1][b.v(a2[0], a2[1], a2[2])] - Ee[t1][b.v(p[0], p[1], p[2])]) / b.dx[t2];
          const long fi = fidx(b, d, p);
          Bof[d][fi] = to_d(Q.rk_g0 * B0f[d][fi] + Q.rk_g1 * Bf[d][fi] - Q.rk_beta * dt * (dE2 - dE1));
        }
  }

  ORACLE_PHASE(5);
  // a8: con2prim on the updated state (cell field from the updated faces)
  for (int k = 0; k < b.n[2]; ++k)
    for (int j = 0; j < b.n[1]; ++j)
      for (int i = 0; i < b.n[0]; ++i) {
        const long ci = b.c(i, j, k);
        const int p[3] = {i, j, k};
        real Bd[3], q[6], w[7];
        for (int d = 0; d < 3; ++d) {
          int p1[3] = {i, j, k};
          p1[d] += 1;
          Bd[d] = 0.5 * (Bof[d][fidx(b, d, p)] + Bof[d][fidx(b, d, p1)]);
        }
        for (int v = 0; v < nq; ++v) q[v] = Uo[v * NC + ci];
        int it = 0;
        ORACLE_C2P_CELL_BEGIN();
        status[ci] = (uint8_t)con2prim_point(cm[ci], Q, q, Bd, w, &it);
        ORACLE_C2P_CELL_END(it);
        if (iters) iters[ci] = it;
        for (int v = 0; v < nq; ++v) Uo[v * NC + ci] = to_d(q[v]);
        for (int v = 0; v < nw; ++v) Wo[v * NC + ci] = to_d(w[v]);
      }
  ORACLE_PHASE(6);
  ORACLE_C2P_SPLIT();
  return 0;
}

// Divergence of the densitised face field on interior cells (Eq. gausslaw, discrete form):
// divB[c] = sum_d (B^d_{+} - B^d_{-}) / dx_d, written into a cell array (interior only).
void oracle_divb_block(const ob_geom* G, const double* Bx, const double* By, const double* Bz,
                       double* divb) {
  Blk b(G);
  const double* Bf[3] = {Bx, By, Bz};
  for (int k = 0; k < b.n[2]; ++k)
    for (int j = 0; j < b.n[1]; ++j)
      for (int i = 0; i < b.n[0]; ++i) {
        real s = 0;
        for (int d = 0; d < 3; ++d) {
          int p[3] = {i, j, k}, p1[3] = {i, j, k};
          p1[d] += 1;
          s += (Bf[d][fidx(b, d, p1)] - Bf[d][fidx(b, d, p)]) / b.dx[d];
        }
        divb[b.c(i, j, k)] = to_d(s);
      }
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// Matter sources of the spacetime equations (Sec. 2.1 hydro form, Sec. 2.2 MHD form) and their
// cell-to-vertex interpolation (Sec. 3.2)
// ------------------------------------------------------------------------------------------------
namespace {

// out = (rho_ADM, S_x, S_y, S_z, S_xx, S_xy, S_xz, S_yy, S_yz, S_zz) at one point:
//   rho_ADM = (rho h + b^2) W^2 - (p + b^2/2) - (alpha b^0)^2
//   S_i     = (rho h + b^2) W^2 v_i - alpha b^0 b_i
//   S_ij    = (rho h + b^2) W^2 v_i v_j + (p + b^2/2) gamma_ij - b_i b_j
// (at B = 0 these are the hydro forms rho h W^2 - p, rho h W^2 v_i, rho h W^2 v_i v_j + p gamma_ij)
void adm_point(const PM& M, const FP& F, real out[10]) {
  const real e = F.rho * F.h + F.b2, pt = F.p + F.b2 / 2, ab0 = M.alpha * F.b0;
  const real eW2 = e * F.W * F.W;
  out[0] = eW2 - pt - ab0 * ab0;
  for (int i = 0; i < 3; ++i) out[1 + i] = eW2 * F.v_d[i] - ab0 * F.b_d[i];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) out[4 + SYM[i][j]] = eW2 * F.v_d[i] * F.v_d[j] + pt * M.g[i][j] - F.b_d[i] * F.b_d[j];
}

}  // namespace

extern "C" {

#ifndef ORACLE_COUNT_FLOPS
// Matter sources at np points; prims and Bdens as oracle_prim2con; out np x 10.
void oracle_adm_points(int np, const double* metric, const double* prims, const double* Bdens, const oparams* Q,
                       double* out) {
  const int nw = Q->eos ? 7 : 5;
  for (int n = 0; n < np; ++n) {
    PM M;
    pm_from16(metric + 16 * n, M);
    FP F;
    fluid_point(M, *Q, prims + nw * n, Bdens + 3 * n, F);
    real o[10];
    adm_point(M, F, o);
    for (int c = 0; c < 10; ++c) out[10 * n + c] = to_d(o[c]);
  }
}

// Matter sources of one block at its owned vertices 0..n (per axis), interpolated from the cell
// centres with the Lagrange interpolant of order vc_order (2: the 2 nearest cells per axis, 4: the
// 4 nearest), the same midpoint weights as the metric's vertex-to-cell interpolation.  The cell
// values use the metric interpolated to the cell centre (order Q.interp_order), the cell field
// (mean of the two densitised faces) and the cell's primitives.  out: 10 x nvert (vertex layout of
// the metric); entries at other vertices are left untouched.  Returns -1 if the ghost width is too
// small for the cells the interpolation reads.
int oracle_adm_block(const ob_geom* G, const double* metric, const double* W, const double* Bx, const double* By,
                     const double* Bz, const oparams* Q, int vc_order, double* out) {
  Blk b(G);
  real wi[4];
  int off, np;
  mid_w(vc_order, wi, &off, &np);
  const int r = np / 2;                            // cells -r .. n + r - 1 per axis
  const int mg = Q->interp_order == 4 ? 1 : 0;     // extra vertices the cell metric reads
  if (b.g < r + mg) return -1;
  const int nw = Q->eos ? 7 : 5;
  const double* mv[16];
  for (int c = 0; c < 16; ++c) mv[c] = metric + c * b.nvert();
  const double* Bf[3] = {Bx, By, Bz};
  const int C[3] = {b.n[0] + 2 * r, b.n[1] + 2 * r, b.n[2] + 2 * r};
  std::vector<real> cellv((size_t)10 * C[0] * C[1] * C[2]);
  auto at = [&](int c, int i, int j, int k) -> real& {
    return cellv[(((size_t)c * C[2] + (k + r)) * C[1] + (j + r)) * C[0] + (i + r)];
  };
  for (int k = -r; k < b.n[2] + r; ++k)
    for (int j = -r; j < b.n[1] + r; ++j)
      for (int i = -r; i < b.n[0] + r; ++i) {
        real m[16];
        interp_cell(b, mv, Q->interp_order, i, j, k, -1, m);
        PM M;
        pm_from16(m, M);
        const int p[3] = {i, j, k};
        real Bc[3], w[7];
        for (int d = 0; d < 3; ++d) {
          int p1[3] = {i, j, k};
          p1[d] += 1;
          Bc[d] = (Bf[d][fidx(b, d, p)] + Bf[d][fidx(b, d, p1)]) / 2;
        }
        for (int v = 0; v < nw; ++v) w[v] = W[v * b.ncell() + cidx(b, p)];
        FP F;
        fluid_point(M, *Q, w, Bc, F);
        real o[10];
        adm_point(M, F, o);
        for (int c = 0; c < 10; ++c) at(c, i, j, k) = o[c];
      }
  // vertex (i, j, k) lies between cells i-1 and i along x (and likewise in y, z)
  for (int k = 0; k <= b.n[2]; ++k)
    for (int j = 0; j <= b.n[1]; ++j)
      for (int i = 0; i <= b.n[0]; ++i)
        for (int c = 0; c < 10; ++c) {
          real s = 0;
          for (int kk = 0; kk < np; ++kk)
            for (int jj = 0; jj < np; ++jj)
              for (int ii = 0; ii < np; ++ii)
                s += wi[ii] * wi[jj] * wi[kk] * at(c, i - 1 + off + ii, j - 1 + off + jj, k - 1 + off + kk);
          out[c * b.nvert() + b.v(i, j, k)] = to_d(s);
        }
  return 0;
}
#endif

}  // extern "C"
