// eos.cuh -- tabulated equation of state on the device (arXiv:2311.04989, Sec. 2.2.1; App. A for the
// temperature root and the bounds policy).
//
// The table holds log p, log e (e = rho (1 + eps)) and c_s^2 on a uniform grid in (log rho, log T,
// Y_e) and is interpolated trilinearly in those variables.  The device arrays store log(p/rho) and
// log(e/rho) = log(1 + eps) at each node: log rho is linear along its own axis, so the trilinear
// interpolant of (log p - log rho) is exactly the interpolant of log p minus log rho -- the same
// function -- but its values are O(1), which keeps the FP32 copy accurate.
//
// Temperature from (rho, p, Y_e) or (rho, eps, Y_e) (the nested root of App. A): at fixed (log rho,
// Y_e) the interpolant is linear in log T between T nodes, so its inverse is found exactly by a
// binary search over the node values followed by one linear solve on the bracketing interval.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace grs {

template <class R> __device__ __forceinline__ R rlog(R x);
template <> __device__ __forceinline__ double rlog(double x) { return log(x); }
template <> __device__ __forceinline__ float rlog(float x) { return logf(x); }
template <class R> __device__ __forceinline__ R rexp(R x);
template <> __device__ __forceinline__ double rexp(double x) { return exp(x); }
template <> __device__ __forceinline__ float rexp(float x) { return expf(x); }
template <class R> __device__ __forceinline__ R rlog1p(R x);
template <> __device__ __forceinline__ double rlog1p(double x) { return log1p(x); }
template <> __device__ __forceinline__ float rlog1p(float x) { return log1pf(x); }
template <class R> __device__ __forceinline__ R rexpm1(R x);
template <> __device__ __forceinline__ double rexpm1(double x) { return expm1(x); }
template <> __device__ __forceinline__ float rexpm1(float x) { return expm1f(x); }

template <class R> __device__ __forceinline__ const TabView<R>& tab_of(const KParams& kp);
template <> __device__ __forceinline__ const TabView<double>& tab_of<double>(const KParams& kp) { return kp.t64; }
template <> __device__ __forceinline__ const TabView<float>& tab_of<float>(const KParams& kp) { return kp.t32; }

// Position on one axis: cell index i in [0, n-2] and fraction in [0, 1]; x outside the axis (or NaN)
// is moved to the nearest end and *cl is set.
template <class R>
__device__ __forceinline__ R tab_locate(const TabView<R>& t, int a, R x, int* i, bool* cl) {
  if (!(x >= t.x0[a])) { x = t.x0[a]; *cl = true; }
  if (x > t.hi[a]) { x = t.hi[a]; *cl = true; }
  const R s = (x - t.x0[a]) * t.idx[a];
  int k = (int)s;
  if (k > t.n[a] - 2) k = t.n[a] - 2;
  *i = k;
  return s - R(k);
}

// (log rho, Y_e) location of a point
template <class R>
struct TabLoc {
  int base;   // node index of (ir, T node 0, iy)
  R wr, wy;
};

template <class R>
__device__ __forceinline__ TabLoc<R> tab_loc(const TabView<R>& t, R lrho, R ye, bool* cl) {
  TabLoc<R> L;
  int ir, iy;
  L.wr = tab_locate(t, 0, lrho, &ir, cl);
  L.wy = tab_locate(t, 2, ye, &iy, cl);
  L.base = iy * t.n[1] * t.n[0] + ir;
  return L;
}

// interpolant of node field f at T node k (bilinear in log rho, Y_e)
template <class R>
__device__ __forceinline__ R tab_at(const TabView<R>& t, const R* __restrict__ f, const TabLoc<R>& L, int k) {
  const int o = L.base + k * t.n[0];
  const int sy = t.n[1] * t.n[0];
  const R a = __ldg(f + o), b = __ldg(f + o + 1), c = __ldg(f + o + sy), d = __ldg(f + o + sy + 1);
  return (R(1) - L.wy) * ((R(1) - L.wr) * a + L.wr * b) + L.wy * ((R(1) - L.wr) * c + L.wr * d);
}

// log T at which the interpolant of f (increasing in T) equals y; y beyond the values at the table's
// T ends gives that end and sets *cl.  *k and *wT receive the T interval and fraction of the result.
// hint >= 0: an interval to try first (the previous result of a root iteration); if it brackets y
// (g(hint) <= y < g(hint+1)) it is the interval the search would find, since g is increasing.
template <class R>
__device__ __forceinline__ R tab_inverse_T(const TabView<R>& t, const R* __restrict__ f, const TabLoc<R>& L,
                                           R y, bool* cl, int* k, R* wT, int hint = -1) {
  if (hint >= 0 && hint < t.n[1] - 1) {
    const R gk = tab_at(t, f, L, hint), gk1 = tab_at(t, f, L, hint + 1);
    if (gk <= y && y < gk1) {
      const R fr = (y - gk) / (gk1 - gk);
      *k = hint;
      *wT = fr;
      return t.x0[1] + t.dx[1] * (R(hint) + fr);
    }
  }
  int lo = 0, hi = t.n[1] - 1;
  R glo = tab_at(t, f, L, lo);
  if (!(y > glo)) {
    if (!(y == glo)) *cl = true;
    *k = 0; *wT = R(0);
    return t.x0[1];
  }
  R ghi = tab_at(t, f, L, hi);
  if (y >= ghi) {
    if (y > ghi) *cl = true;
    *k = hi - 1; *wT = R(1);
    return t.hi[1];
  }
  while (hi - lo > 1) {   // g(lo) < y < g(hi); at most log2(n_T) steps
    const int mid = (lo + hi) >> 1;
    const R gm = tab_at(t, f, L, mid);
    if (gm <= y) { lo = mid; glo = gm; }
    else { hi = mid; ghi = gm; }
  }
  const R fr = (y - glo) / (ghi - glo);
  *k = lo;
  *wT = fr;
  return t.x0[1] + t.dx[1] * (R(lo) + fr);
}

// interpolant of f at T interval k, fraction wT
template <class R>
__device__ __forceinline__ R tab_T(const TabView<R>& t, const R* __restrict__ f, const TabLoc<R>& L, int k, R wT) {
  const R a = tab_at(t, f, L, k), b = tab_at(t, f, L, k + 1);
  return a + wT * (b - a);
}

// Thermodynamics of a point from (rho, p, Y_e): rho h = rho (1 + eps) + p, c_s^2 and (optionally) T.
template <class R>
__device__ __forceinline__ void tab_thermo_p(const TabView<R>& t, R rho, R p, R ye, R* rhoh, R* cs2, R* T) {
  bool cl = false;
  const TabLoc<R> L = tab_loc(t, rlog(rho), ye, &cl);
  int k;
  R wT;
  const R lT = tab_inverse_T(t, t.f[0], L, rlog(p / rho), &cl, &k, &wT);
  const R l1e = tab_T(t, t.f[1], L, k, wT);       // log(1 + eps)
  *rhoh = rho * rexp(l1e) + p;
  *cs2 = tab_T(t, t.f[2], L, k, wT);
  if (T) *T = rexp(lT);
}

// p and eps at (rho, T, Y_e) (atmosphere, temperature floor, tau floor)
template <class R>
__device__ __forceinline__ void tab_p_eps_T(const TabView<R>& t, R rho, R lT, R ye, R* p, R* eps) {
  bool cl = false;
  const TabLoc<R> L = tab_loc(t, rlog(rho), ye, &cl);
  int k;
  const R wT = tab_locate(t, 1, lT, &k, &cl);
  *p = rho * rexp(tab_T(t, t.f[0], L, k, wT));
  *eps = rexpm1(tab_T(t, t.f[1], L, k, wT));
}

}  // namespace grs
