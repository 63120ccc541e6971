// physics.cuh -- device arithmetic of the GRMHD stage (arXiv:2311.04989, Sec. 2-3).
//
// Templated on the arithmetic type R of the reconstruction / Riemann / EMF path (double for the
// FP64 path, float for the mixed path).  Con2prim, the sources and all accumulation are FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "eos.cuh"
#include "internal.h"
#include "mlp.cuh"

namespace grs {

// ------------------------------------------------------------------------------------------------
// small helpers
// ------------------------------------------------------------------------------------------------
// square root in precision R: the IEEE square root in FP64; in FP32 (the mixed path) the hardware's
// approximate square root (PTX sqrt.approx.f32, relative error of the order of one FP32 ulp), a single
// instruction instead of the correctly rounded sequence
template <class R> __device__ __forceinline__ R sqrt_r(R x);
template <> __device__ __forceinline__ double sqrt_r(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float sqrt_r(float x) {
  float y;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// the Lorentz factor W = sqrt(1 + u~^2), correctly rounded in both precisions: tau is formed as
// (rho h + b^2) W^2 - rho W - ..., where the rest mass cancels, so an ulp of W costs an ulp of rho
// against the much smaller tau
template <class R> __device__ __forceinline__ R sqrt_w(R x) { return sqrt(x); }
template <> __device__ __forceinline__ float sqrt_w(float x) { return sqrtf(x); }

// a/b: IEEE division in FP64; the fast approximate FP32 division (2 ulp) on the mixed path
template <class R> __device__ __forceinline__ R rdiv(R a, R b);
template <> __device__ __forceinline__ double rdiv(double a, double b) { return a / b; }
template <> __device__ __forceinline__ float rdiv(float a, float b) { return __fdividef(a, b); }

template <class R> __device__ __forceinline__ R rabs(R x) { return x < R(0) ? -x : x; }

// whether x is finite, from the exponent bits of its high word (integer operations only: on GB300 an
// FP64 comparison is an instruction of the narrow FP64 pipe)
__device__ __forceinline__ bool finite64(double x) { return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000; }

// Precision conversions without the FP64 pipe (on GB300 an F2F conversion is an FP64-pipe
// instruction, ~1/64 of the FP32 rate), in integer arithmetic on the IEEE-754 encodings.
// FP64 -> FP32: round to nearest, ties to even, with gradual underflow (float subnormals) and
// overflow to infinity, i.e. the IEEE conversion; NaN becomes the canonical quiet NaN of its sign.
// FP32 -> FP64 is exact.
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned long long sgn = u & 0x8000000000000000ull;
  const unsigned long long a = u ^ sgn;
  const unsigned int s32 = (unsigned int)(sgn >> 32);
  if (a >= 0x7FF0000000000000ull) return __uint_as_float(s32 | (a > 0x7FF0000000000000ull ? 0x7FC00000u : 0x7F800000u));
  const int e = (int)(a >> 52);                                 // biased binary exponent of |x|
  if (e >= 1151) return __uint_as_float(s32 | 0x7F800000u);     // |x| >= 2^128
  if (e >= 897) {                                               // |x| >= 2^-126: a normal float
    // drop the low 29 significand bits, rounding to nearest even; a carry out of the significand
    // steps the exponent (and turns 2^128 into infinity); rebias the exponent by 1023 - 127
    const unsigned long long r = a + 0x0FFFFFFFull + ((a >> 29) & 1ull);
    return __uint_as_float(s32 | (unsigned int)((r >> 29) - (896ull << 23)));
  }
  if (e < 873) return __uint_as_float(s32);                     // |x| < 2^-150: rounds to zero
  // a float subnormal: |x| = M 2^(e - 1075) with the 53-bit significand M, in units of 2^-149 that is
  // M / 2^s with s = 926 - e in [30, 53]; round the quotient to nearest even (2^23 is the smallest normal)
  const int s = 926 - e;
  const unsigned long long M = (a & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  unsigned long long q = M >> s;
  const unsigned long long rem = M & ((1ull << s) - 1ull), half = 1ull << (s - 1);
  if (rem > half || (rem == half && (q & 1ull))) ++q;
  return __uint_as_float(s32 | (unsigned int)q);
}

__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int sgn = u & 0x80000000u;
  const unsigned int a = u ^ sgn;
  if (a == 0u) return __longlong_as_double((long long)((unsigned long long)sgn << 32));
  if (a < 0x00800000u || a >= 0x7F800000u) return (double)f;    // subnormal, inf, nan (rare)
  const unsigned long long bits = ((unsigned long long)sgn << 32) |
                                  ((unsigned long long)((a >> 23) + 896u) << 52) |
                                  ((unsigned long long)(a & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}

template <class R> __device__ __forceinline__ double to64(R x);
template <> __device__ __forceinline__ double to64(double x) { return x; }
template <> __device__ __forceinline__ double to64(float x) { return f2d_exact(x); }

// a - b in FP64.  For two FP32 values the difference is exact in FP64; it is formed in FP32 when it is
// exact there too (Knuth's two-sum of a and -b has a zero error term, as for values within a factor 2
// of each other by Sterbenz's lemma) and widened by integer operations, else by an FP64 subtraction:
// the same value either way, mostly without the narrow FP64 pipe.
template <class R> __device__ __forceinline__ double diff64(R a, R b);
template <> __device__ __forceinline__ double diff64(double a, double b) { return a - b; }
template <> __device__ __forceinline__ double diff64(float a, float b) {
  const float s = __fsub_rn(a, b);
  const float bp = __fsub_rn(s, a);               // the part of s that came from -b
  const float ap = __fsub_rn(s, bp);              // the part of s that came from a
  const float err = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(__fsub_rn(0.f, b), bp));
  if (err == 0.f && isfinite(s)) return f2d_exact(s);
  return f2d_exact(a) - f2d_exact(b);
}
template <class R> __device__ __forceinline__ R rmax(R a, R b) { return a > b ? a : b; }
template <class R> __device__ __forceinline__ R rmin(R a, R b) { return a < b ? a : b; }

// symmetric 3x3 packed as xx, xy, xz, yy, yz, zz
__device__ __forceinline__ int sidx(int i, int j) {
  // (0,0)0 (0,1)1 (0,2)2 (1,1)3 (1,2)4 (2,2)5
  return (i <= j) ? (i == 0 ? j : (i == 1 ? 2 + j : 5)) : (j == 0 ? i : (j == 1 ? 2 + i : 5));
}

// lower an index with gamma_ij
template <class R>
__device__ __forceinline__ void lower3(const R g[6], const R u[3], R l[3]) {
  l[0] = g[0] * u[0] + g[1] * u[1] + g[2] * u[2];
  l[1] = g[1] * u[0] + g[3] * u[1] + g[4] * u[2];
  l[2] = g[2] * u[0] + g[4] * u[1] + g[5] * u[2];
}

template <class R>
__device__ __forceinline__ R det3(const R g[6]) {
  return g[0] * (g[3] * g[5] - g[4] * g[4]) - g[1] * (g[1] * g[5] - g[4] * g[2]) +
         g[2] * (g[1] * g[4] - g[3] * g[2]);
}

// gamma^{dd} = cofactor_dd / det
template <class R>
__device__ __forceinline__ R inv_dd(const R g[6], int d, R det) {
  R c;
  if (d == 0) c = g[3] * g[5] - g[4] * g[4];
  else if (d == 1) c = g[0] * g[5] - g[2] * g[2];
  else c = g[0] * g[3] - g[1] * g[1];
  return rdiv(c, det);
}

// full inverse
template <class R>
__device__ __forceinline__ void inv3_id(const R g[6], R id, R gi[6]) {
  gi[0] = (g[3] * g[5] - g[4] * g[4]) * id;
  gi[1] = (g[2] * g[4] - g[1] * g[5]) * id;
  gi[2] = (g[1] * g[4] - g[2] * g[3]) * id;
  gi[3] = (g[0] * g[5] - g[2] * g[2]) * id;
  gi[4] = (g[1] * g[2] - g[0] * g[4]) * id;
  gi[5] = (g[0] * g[3] - g[1] * g[1]) * id;
}

template <class R>
__device__ __forceinline__ void inv3(const R g[6], R det, R gi[6]) {
  const R id = rdiv(R(1), det);
  gi[0] = (g[3] * g[5] - g[4] * g[4]) * id;
  gi[1] = (g[2] * g[4] - g[1] * g[5]) * id;
  gi[2] = (g[1] * g[4] - g[2] * g[3]) * id;
  gi[3] = (g[0] * g[5] - g[2] * g[2]) * id;
  gi[4] = (g[1] * g[2] - g[0] * g[4]) * id;
  gi[5] = (g[0] * g[3] - g[1] * g[1]) * id;
}

// ------------------------------------------------------------------------------------------------
// Layout helpers (ghost-padded, x fastest)
// ------------------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ long long cix(const DBlock& b, int i, int j, int k) {
  return ((long long)(k + b.g) * b.N[1] + (j + b.g)) * b.N[0] + (i + b.g);
}
__host__ __device__ __forceinline__ long long fix(const DBlock& b, int d, int i, int j, int k) {
  const int sx = b.N[0] + (d == 0), sy = b.N[1] + (d == 1);
  return ((long long)(k + b.g) * sy + (j + b.g)) * sx + (i + b.g);
}
__host__ __device__ __forceinline__ long long vix(const DBlock& b, int i, int j, int k) {
  return ((long long)(k + b.g) * (b.N[1] + 1) + (j + b.g)) * (b.N[0] + 1) + (i + b.g);
}

// ------------------------------------------------------------------------------------------------
// Metric interpolation from vertices (Sec. 3.2): tensor-product Lagrange, order 2 or 4, at the
// centre of a d-face (face plane = vertex plane p[d]) and at cell centres (with derivatives).
// ------------------------------------------------------------------------------------------------
// vertex index within a block (32-bit: a block has fewer than 2^31 vertices)
__device__ __forceinline__ int vix32(const DBlock& b, int i, int j, int k) {
  return ((k + b.g) * (b.N[1] + 1) + (j + b.g)) * (b.N[0] + 1) + (i + b.g);
}

template <class R>
__device__ __forceinline__ void face_metric(const DBlock& b, const InView<R>& m, int order, int d,
                                            const int p[3], R out[10]) {
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  const long long base = b.vert;
  if (order == 2) {
    // the four vertices of the face: offsets within the block, one pointer per component
    const int v00 = vix32(b, p[0], p[1], p[2]);
    const int s1 = t1 == 0 ? 1 : (t1 == 1 ? b.N[0] + 1 : (b.N[0] + 1) * (b.N[1] + 1));
    const int s2 = t2 == 0 ? 1 : (t2 == 1 ? b.N[0] + 1 : (b.N[0] + 1) * (b.N[1] + 1));
#pragma unroll
    for (int c = 0; c < 10; ++c) {
      const R* a = m.M[c] + base + v00;
      out[c] = R(0.25) * ((a[0] + a[s1]) + (a[s2] + a[s1 + s2]));
    }
  } else {
    const R w[4] = {R(-1.0 / 16), R(9.0 / 16), R(9.0 / 16), R(-1.0 / 16)};
#pragma unroll
    for (int c = 0; c < 10; ++c) out[c] = R(0);
    for (int s2 = 0; s2 < 4; ++s2)
      for (int s1 = 0; s1 < 4; ++s1) {
        int q[3] = {p[0], p[1], p[2]};
        q[t1] += s1 - 1;
        q[t2] += s2 - 1;
        const long long vi = base + vix(b, q[0], q[1], q[2]);
        const R ww = w[s1] * w[s2];
#pragma unroll
        for (int c = 0; c < 10; ++c) out[c] += ww * m.M[c][vi];
      }
  }
}

// Cell-centre value of components [c0, nc) and, if dv != nullptr, derivatives d_k of components
// [0, 10) (alpha, beta, gamma), computed in R from the FP64 vertex pools.  The derivative along k is
// written as vertex differences so that it vanishes exactly on a constant field.
template <class R>
__device__ __forceinline__ void cell_metric(const DBlock& b, const InView<R>& m, int order, int i,
                                            int j, int k, int c0, int nc, R* val, R (*dv)[10]) {
  const long long base = b.vert;
  if (order == 2) {
    long long v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = base + vix(b, i + (t & 1), j + ((t >> 1) & 1), k + (t >> 2));
    const R ix = R(0.25 * b.idx[0]), iy = R(0.25 * b.idx[1]), iz = R(0.25 * b.idx[2]);
#pragma unroll
    for (int c = c0; c < nc; ++c) {
      const R* a = m.M[c];
      R f[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) f[t] = a[v[t]];
      val[c] = R(0.125) * (((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])));
      if (dv && c < 10) {
        dv[0][c] = (((f[1] - f[0]) + (f[3] - f[2])) + ((f[5] - f[4]) + (f[7] - f[6]))) * ix;
        dv[1][c] = (((f[2] - f[0]) + (f[3] - f[1])) + ((f[6] - f[4]) + (f[7] - f[5]))) * iy;
        dv[2][c] = (((f[4] - f[0]) + (f[5] - f[1])) + ((f[6] - f[2]) + (f[7] - f[3]))) * iz;
      }
    }
  } else {
    const R w[4] = {R(-1.0 / 16), R(9.0 / 16), R(9.0 / 16), R(-1.0 / 16)};
    for (int c = c0; c < nc; ++c) {
      const R* a = m.M[c];
      R s = 0, d0 = 0;
      for (int kk = 0; kk < 4; ++kk)
        for (int jj = 0; jj < 4; ++jj) {
          const long long r = base + vix(b, i - 1, j - 1 + jj, k - 1 + kk);
          const R f0 = a[r], f1 = a[r + 1], f2 = a[r + 2], f3 = a[r + 3];
          const R wjk = w[jj] * w[kk];
          s += wjk * (w[0] * f0 + w[1] * f1 + w[2] * f2 + w[3] * f3);
          if (dv && c < 10) d0 += wjk * (R(27) * (f2 - f1) - (f3 - f0));
        }
      val[c] = s;
      if (dv && c < 10) {
        dv[0][c] = d0 * R(1.0 / (24.0 * b.dx[0]));
        for (int ax = 1; ax < 3; ++ax) {
          R acc = 0;
          for (int u = 0; u < 4; ++u)
            for (int t = 0; t < 4; ++t) {
              auto at = [&](int s4) {
                int q[3] = {i - 1 + t, j - 1 + (ax == 2 ? u : 0), k - 1 + (ax == 1 ? u : 0)};
                q[ax] = (ax == 1 ? j : k) - 1 + s4;
                return a[base + vix(b, q[0], q[1], q[2])];
              };
              acc += w[t] * w[u] * (R(27) * (at(2) - at(1)) - (at(3) - at(0)));
            }
          dv[ax][c] = acc * R(1.0 / (24.0 * b.dx[ax]));
        }
      }
    }
  }
}

// ------------------------------------------------------------------------------------------------
// Reconstruction (Sec. 3.4): van Leer PLM and WENOZ (Borges et al.).
// s[0..5] = cells f-3 .. f+2 around the face f (between s[2] and s[3]).
// ------------------------------------------------------------------------------------------------
// Arithmetic of the PLM, WENO5 and PPM reconstructions.  FP32 (mixed path): explicit round-to-nearest
// operations that the compiler never fuses into an FMA, so a stencil evaluates to the same bits in every
// kernel that reconstructs it (a fused multiply-add is otherwise chosen per kernel, where a common
// subexpression of the two face states can change which product gets fused).  FP64: the plain operators
// in the oracle's order.
template <class R> __device__ __forceinline__ R xm(R a, R b) { return a * b; }
template <> __device__ __forceinline__ float xm(float a, float b) { return __fmul_rn(a, b); }
template <class R> __device__ __forceinline__ R xa(R a, R b) { return a + b; }
template <> __device__ __forceinline__ float xa(float a, float b) { return __fadd_rn(a, b); }
template <class R> __device__ __forceinline__ R xs(R a, R b) { return a - b; }
template <> __device__ __forceinline__ float xs(float a, float b) { return __fsub_rn(a, b); }

template <class R>
__device__ __forceinline__ R vl_slope(R wm, R w0, R wp) {
  const R dL = xs(w0, wm), dR = xs(wp, w0);
  const R pr = xm(dL, dR);
  return pr > R(0) ? xm(R(2), pr) / xa(dL, dR) : R(0);
}

// smoothness indicators and candidate values shared by both weight forms
template <class R>
__device__ __forceinline__ void wenoz_parts(R v0, R v1, R v2, R v3, R v4, R q[3], R bk[3]) {
  q[0] = xm(xa(xs(xm(R(2), v0), xm(R(7), v1)), xm(R(11), v2)), R(1.0 / 6.0));
  q[1] = xm(xa(xa(-v1, xm(R(5), v2)), xm(R(2), v3)), R(1.0 / 6.0));
  q[2] = xm(xs(xa(xm(R(2), v2), xm(R(5), v3)), v4), R(1.0 / 6.0));
  const R a0 = xa(xs(v0, xm(R(2), v1)), v2), c0 = xa(xs(v0, xm(R(4), v1)), xm(R(3), v2));
  const R a1 = xa(xs(v1, xm(R(2), v2)), v3), c1 = xs(v1, v3);
  const R a2 = xa(xs(v2, xm(R(2), v3)), v4), c2 = xa(xs(xm(R(3), v2), xm(R(4), v3)), v4);
  bk[0] = xa(xm(xm(R(13.0 / 12.0), a0), a0), xm(xm(R(0.25), c0), c0));
  bk[1] = xa(xm(xm(R(13.0 / 12.0), a1), a1), xm(xm(R(0.25), c1), c1));
  bk[2] = xa(xm(xm(R(13.0 / 12.0), a2), a2), xm(xm(R(0.25), c2), c2));
}

// WENOZ value at the right edge of the middle cell of v0..v4.
// FP64: the weights alpha_k = d_k (1 + tau5/e_k), e_k = beta_k + eps, are multiplied through by
// e_0 e_1 e_2 so that one division normalises them (same weights, one FP64 division instead of
// four).  FP32: per-weight fast divisions on the power-of-two scaled stencil.
template <class R>
__device__ __forceinline__ R wenoz(R v0, R v1, R v2, R v3, R v4, R eps);

template <>
__device__ __forceinline__ double wenoz<double>(double v0, double v1, double v2, double v3, double v4,
                                                double eps) {
  double q[3], bk[3];
  wenoz_parts(v0, v1, v2, v3, v4, q, bk);
  const double t5 = fabs(bk[0] - bk[2]);
  const double e0 = bk[0] + eps, e1 = bk[1] + eps, e2 = bk[2] + eps;
  const double P = e0 * e1 * e2;
  const double w0 = 0.1 * (P + t5 * (e1 * e2));
  const double w1 = 0.6 * (P + t5 * (e0 * e2));
  const double w2 = 0.3 * (P + t5 * (e0 * e1));
  return (w0 * q[0] + w1 * q[1] + w2 * q[2]) / (w0 + w1 + w2);
}

// FP32: per-weight fast divisions on the power-of-two scaled stencil (|v| < 2), eps = 1e-30.  A
// product form with one division would need a much larger eps to keep e0 e1 e2 a normal float,
// which lets rough sub-stencils leak into faces between cells ~1e11 apart in density (star
// surface against atmosphere).
template <>
__device__ __forceinline__ float wenoz<float>(float v0, float v1, float v2, float v3, float v4, float eps) {
  float q[3], bk[3];
  wenoz_parts(v0, v1, v2, v3, v4, q, bk);
  const float t5 = fabsf(bk[0] - bk[2]);
  const float w0 = 0.1f * (1.f + __fdividef(t5, bk[0] + eps));
  const float w1 = 0.6f * (1.f + __fdividef(t5, bk[1] + eps));
  const float w2 = 0.3f * (1.f + __fdividef(t5, bk[2] + eps));
  return __fdividef(w0 * q[0] + w1 * q[1] + w2 * q[2], w0 + w1 + w2);
}

// FP32: the stencil is scaled by a power of two near its largest magnitude before the smoothness
// indicators are formed, so that squares of tiny densities/pressures (atmosphere p ~ 1e-30) do not
// underflow; the scaling is exact and is undone on the result.
// 2^-e and 2^e for the binary exponent e of m > 0 (normal, finite), by bit manipulation
__device__ __forceinline__ void pow2_pair(float m, float* sc, float* isc) {
  const int e = (int)((__float_as_uint(m) >> 23) & 0xFFu) - 127;   // m in [2^e, 2^(e+1))
  *sc = __uint_as_float((unsigned)(127 - e) << 23);                 // 2^-e
  *isc = __uint_as_float((unsigned)(127 + e) << 23);                // 2^e
}

// WENO5 (Jiang & Shu) value at the right edge of the middle cell: weights d_k / (beta_k + eps)^2.
// FP64: multiplied through by the product of the squares so that one division normalises them;
// FP32: per-weight fast divisions with eps = 1e-18 on the scaled stencil (eps^2 stays a normal float).
template <class R>
__device__ __forceinline__ R weno5(R v0, R v1, R v2, R v3, R v4, R eps);

template <>
__device__ __forceinline__ double weno5<double>(double v0, double v1, double v2, double v3, double v4,
                                                double eps) {
  double q[3], bk[3];
  wenoz_parts(v0, v1, v2, v3, v4, q, bk);
  const double e0 = (bk[0] + eps) * (bk[0] + eps), e1 = (bk[1] + eps) * (bk[1] + eps);
  const double e2 = (bk[2] + eps) * (bk[2] + eps);
  const double w0 = 0.1 * (e1 * e2), w1 = 0.6 * (e0 * e2), w2 = 0.3 * (e0 * e1);
  return (w0 * q[0] + w1 * q[1] + w2 * q[2]) / (w0 + w1 + w2);
}

template <>
__device__ __forceinline__ float weno5<float>(float v0, float v1, float v2, float v3, float v4, float eps) {
  (void)eps;
  float q[3], bk[3];
  wenoz_parts(v0, v1, v2, v3, v4, q, bk);
  const float e = 1e-18f;
  const float w0 = __fdividef(0.1f, xm(xa(bk[0], e), xa(bk[0], e)));
  const float w1 = __fdividef(0.6f, xm(xa(bk[1], e), xa(bk[1], e)));
  const float w2 = __fdividef(0.3f, xm(xa(bk[2], e), xa(bk[2], e)));
  return __fdividef(xa(xa(xm(w0, q[0]), xm(w1, q[1])), xm(w2, q[2])), xa(xa(w0, w1), w2));
}

// PPM: fourth-order interface values limited by the extremum-preserving criterion of Colella & Sekora,
// then each cell's parabola limited at extrema (curvature) and elsewhere by monotonicity; C = 1.25.
template <class R> __device__ __forceinline__ R rsgn(R x) { return x > R(0) ? R(1) : (x < R(0) ? R(-1) : R(0)); }

template <class R>
__device__ __forceinline__ R ppm_iface(R q0, R q1, R q2, R q3) {
  R qf = xs(xm(R(7.0 / 12.0), xa(q1, q2)), xm(R(1.0 / 12.0), xa(q0, q3)));
  if (xm(xs(qf, q1), xs(q2, qf)) < R(0)) {
    const R d2f = xm(R(3), xa(xs(q1, xm(R(2), qf)), q2));
    const R d2l = xa(xs(q0, xm(R(2), q1)), q2);
    const R d2r = xa(xs(q1, xm(R(2), q2)), q3);
    const R sf = rsgn(d2f);
    R d2lim = R(0);
    if (sf == rsgn(d2l) && sf == rsgn(d2r) && d2f != R(0))
      d2lim = xm(sf, rmin(rmin(xm(R(1.25), rabs(d2l)), xm(R(1.25), rabs(d2r))), rabs(d2f)));
    qf = xs(xm(R(0.5), xa(q1, q2)), xm(d2lim, R(1.0 / 6.0)));
  }
  return qf;
}

template <class R>
__device__ __forceinline__ void ppm_cell(R v0, R v1, R v2, R v3, R v4, R* qm, R* qp) {
  R l = ppm_iface(v0, v1, v2, v3), r = ppm_iface(v1, v2, v3, v4);
  const R q = v2;
  if (xm(xs(r, q), xs(q, l)) <= R(0) || xm(xs(v1, q), xs(q, v3)) <= R(0)) {
    const R d2 = xm(R(6), xa(xs(l, xm(R(2), q)), r));
    const R d2c = xa(xs(v1, xm(R(2), q)), v3);
    const R d2l = xa(xs(v0, xm(R(2), v1)), q);
    const R d2r = xa(xs(q, xm(R(2), v3)), v4);
    const R s2 = rsgn(d2);
    R d2lim = R(0);
    if (s2 == rsgn(d2c) && s2 == rsgn(d2l) && s2 == rsgn(d2r) && d2 != R(0))
      d2lim = xm(s2, rmin(rmin(rmin(xm(R(1.25), rabs(d2l)), xm(R(1.25), rabs(d2r))), xm(R(1.25), rabs(d2c))),
                          rabs(d2)));
    if (d2 == R(0)) {
      l = q;
      r = q;
    } else {
      const R ratio = d2lim / d2;
      l = xa(q, xm(xs(l, q), ratio));
      r = xa(q, xm(xs(r, q), ratio));
    }
  } else {
    if (rabs(xs(r, q)) >= xm(R(2), rabs(xs(l, q)))) r = xs(q, xm(R(2), xs(l, q)));
    if (rabs(xs(l, q)) >= xm(R(2), rabs(xs(r, q)))) l = xs(q, xm(R(2), xs(r, q)));
  }
  *qm = l;
  *qp = r;
}

// WENOZ of both face states at once in FP32 (packed FP32x2 arithmetic: one instruction per operation
// for both).  Lane x: the L state, wenoz of cells f-3 .. f+1; lane y: the R state, wenoz of the mirror
// image f+2 .. f-2.  Both lanes take the same operations, so a mirror-symmetric stencil still gives
// L == R bitwise.  Weights d_k (1 + tau5/(beta_k + eps)) from the fast reciprocal of beta_k + eps.
__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 pk1(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 prcp(float2 a) { return make_float2(__fdividef(1.f, a.x), __fdividef(1.f, a.y)); }

__device__ __forceinline__ void wenoz_pair(const float s[6], float eps, float* L, float* Rr) {
  const float2 v0 = pk(s[0], s[5]), v1 = pk(s[1], s[4]), v2 = pk(s[2], s[3]);
  const float2 v3 = pk(s[3], s[2]), v4 = pk(s[4], s[1]);
  const float2 sixth = pk1(1.f / 6.f);
  // candidates (2 v0 - 7 v1 + 11 v2)/6, (-v1 + 5 v2 + 2 v3)/6, (2 v2 + 5 v3 - v4)/6
  const float2 q0 = __fmul2_rn(__ffma2_rn(pk1(11.f), v2, __ffma2_rn(pk1(-7.f), v1, __fmul2_rn(pk1(2.f), v0))), sixth);
  const float2 q1 = __fmul2_rn(__ffma2_rn(pk1(2.f), v3, __ffma2_rn(pk1(5.f), v2, __fmul2_rn(pk1(-1.f), v1))), sixth);
  const float2 q2 = __fmul2_rn(__ffma2_rn(pk1(-1.f), v4, __ffma2_rn(pk1(5.f), v3, __fmul2_rn(pk1(2.f), v2))), sixth);
  // smoothness indicators 13/12 a^2 + 1/4 c^2
  const float2 a0 = __fadd2_rn(__ffma2_rn(pk1(-2.f), v1, v0), v2);
  const float2 c0 = __ffma2_rn(pk1(3.f), v2, __ffma2_rn(pk1(-4.f), v1, v0));
  const float2 a1 = __fadd2_rn(__ffma2_rn(pk1(-2.f), v2, v1), v3);
  const float2 c1 = __ffma2_rn(pk1(-1.f), v3, v1);
  const float2 a2 = __fadd2_rn(__ffma2_rn(pk1(-2.f), v3, v2), v4);
  const float2 c2 = __ffma2_rn(pk1(3.f), v2, __ffma2_rn(pk1(-4.f), v3, v4));
  const float2 k13 = pk1(13.f / 12.f), k14 = pk1(0.25f);
  const float2 b0 = __ffma2_rn(__fmul2_rn(k13, a0), a0, __fmul2_rn(__fmul2_rn(k14, c0), c0));
  const float2 b1 = __ffma2_rn(__fmul2_rn(k13, a1), a1, __fmul2_rn(__fmul2_rn(k14, c1), c1));
  const float2 b2 = __ffma2_rn(__fmul2_rn(k13, a2), a2, __fmul2_rn(__fmul2_rn(k14, c2), c2));
  const float2 d02 = __fadd2_rn(b0, __fmul2_rn(pk1(-1.f), b2));
  const float2 t5 = pk(fabsf(d02.x), fabsf(d02.y));
  const float2 e2 = pk1(eps);
  const float2 r0 = __fmul2_rn(t5, prcp(__fadd2_rn(b0, e2)));
  const float2 r1 = __fmul2_rn(t5, prcp(__fadd2_rn(b1, e2)));
  const float2 r2 = __fmul2_rn(t5, prcp(__fadd2_rn(b2, e2)));
  const float2 w0 = __ffma2_rn(pk1(0.1f), r0, pk1(0.1f));
  const float2 w1 = __ffma2_rn(pk1(0.6f), r1, pk1(0.6f));
  const float2 w2 = __ffma2_rn(pk1(0.3f), r2, pk1(0.3f));
  const float2 num = __ffma2_rn(w2, q2, __ffma2_rn(w1, q1, __fmul2_rn(w0, q0)));
  const float2 den = __fadd2_rn(__fadd2_rn(w0, w1), w2);
  *L = __fdividef(num.x, den.x);
  *Rr = __fdividef(num.y, den.y);
}

// Face states of the 6-cell stencil s[0..5] = cells f-3 .. f+2 by method (Sec. 3.4)
template <class R, int METHOD>
__device__ __forceinline__ void recon_plain(const R s[6], R eps, R* L, R* Rr) {
  constexpr int method = METHOD;
  if constexpr (method == GR_RECON_PLM) {
    *L = xa(s[2], xm(R(0.5), vl_slope(s[1], s[2], s[3])));
    *Rr = xs(s[3], xm(R(0.5), vl_slope(s[2], s[3], s[4])));
  } else if constexpr (method == GR_RECON_WENOZ) {
    if constexpr (sizeof(R) == sizeof(float)) {
      wenoz_pair(s, eps, L, Rr);
    } else {
      *L = wenoz(s[0], s[1], s[2], s[3], s[4], eps);
      *Rr = wenoz(s[5], s[4], s[3], s[2], s[1], eps);
    }
  } else if constexpr (method == GR_RECON_WENO5) {
    *L = weno5(s[0], s[1], s[2], s[3], s[4], eps);
    *Rr = weno5(s[5], s[4], s[3], s[2], s[1], eps);
  } else {
    R lm, lp, rm, rp;
    ppm_cell(s[0], s[1], s[2], s[3], s[4], &lm, &lp);
    ppm_cell(s[1], s[2], s[3], s[4], s[5], &rm, &rp);
    *L = lp;
    *Rr = rm;
  }
}

// SCALE (FP32 only): for the WENO and PPM methods, scale the stencil by a power of two near its
// largest magnitude first (exact, undone on the result).  Needed for variables whose values can be so
// small that their squared differences underflow (density and pressure near the atmosphere);
// velocities, the cell field and Y_e are O(1e-10) or larger where they matter and skip it.
template <class R, int METHOD, bool SCALE = true>
__device__ __forceinline__ void recon(const R s[6], R eps, R* L, R* Rr) {
  if constexpr (sizeof(R) == sizeof(float) && SCALE && METHOD != GR_RECON_PLM) {
    {
      float mx = 0.f;
#pragma unroll
      for (int t = 0; t < 6; ++t) mx = fmaxf(mx, fabsf(s[t]));
      // all zero, subnormal or non-finite: nothing to scale (2^e must stay a normal float)
      if (mx >= 1.2e-38f && mx < 1e38f) {
        float sc, isc;
        pow2_pair(mx, &sc, &isc);
        float t[6];
#pragma unroll
        for (int u = 0; u < 6; ++u) t[u] = s[u] * sc;
        recon_plain<float, METHOD>(t, eps, L, Rr);
        *L *= isc;
        *Rr *= isc;
        return;
      }
    }
  }
  recon_plain<R, METHOD>(s, eps, L, Rr);
}

// ------------------------------------------------------------------------------------------------
// EOS at a point from (rho, p[, Y_e]) (Sec. 2.2.1): rho h and c_s^2.  Ideal gas (reading c3 for c_s):
// rho h = rho + Gamma p/(Gamma - 1), c_s^2 = Gamma p/(rho h); table: interpolated (eos.cuh).
// ------------------------------------------------------------------------------------------------
template <class R, int EOS>
__device__ __forceinline__ void eos_rhoh_cs2(const KParams& kp, R rho, R p, R ye, R* rhoh, R* cs2) {
  if constexpr (EOS == GR_EOS_IDEAL) {
    R gam;
    if constexpr (sizeof(R) == sizeof(float)) gam = kp.gamma_f;
    else gam = kp.gamma_ad;
    *rhoh = rho + gam * rdiv(p, gam - R(1));
    *cs2 = rdiv(gam * p, *rhoh);
  } else {
    tab_thermo_p<R>(tab_of<R>(kp), rho, p, ye, rhoh, cs2, (R*)nullptr);
  }
}

// ------------------------------------------------------------------------------------------------
// One side of a face: conserved U (D, S_j, tau, B^{t1}, B^{t2}), flux F^d of Eq. fluxB_def and
// fast speeds (lam-, lam+) (Sec. 2.2, approximate quadratic dispersion relation).
//   met: alpha, beta^i, gamma_ij at the face; sg = sqrt(gamma); gdd = gamma^{dd}
//   w: (rho, u~^i, p[, Y_e]); Bd: densitised B^i at the face state.
// ------------------------------------------------------------------------------------------------
template <class R, int EOS>
__device__ __forceinline__ void face_state(int d, const R met[10], R sg, R gdd, const KParams& kp, const R w[6],
                                           const R Bd[3], R U[7], R F[7], R* lm, R* lp) {
  const R alpha = met[0];
  const R* beta = met + 1;
  const R* g = met + 4;
  const R rho = w[0], p = w[4];
  const R ut[3] = {w[1], w[2], w[3]};
  R utl[3];
  lower3(g, ut, utl);
  const R W = sqrt_w(R(1) + ut[0] * utl[0] + ut[1] * utl[1] + ut[2] * utl[2]);
  const R iW = rdiv(R(1), W);
  const R ia = rdiv(R(1), alpha);
  const R isg = rdiv(R(1), sg);
  R v[3], vl[3], vt[3], Bu[3], Bl[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    v[i] = ut[i] * iW;
    vl[i] = utl[i] * iW;
    vt[i] = v[i] - beta[i] * ia;
    Bu[i] = Bd[i] * isg;
  }
  lower3(g, Bu, Bl);
  const R Bv = Bu[0] * vl[0] + Bu[1] * vl[1] + Bu[2] * vl[2];
  const R BB = Bu[0] * Bl[0] + Bu[1] * Bl[1] + Bu[2] * Bl[2];
  const R ab0 = W * Bv;                          // alpha b^0
  const R b2 = (ab0 * ab0 + BB) * iW * iW;       // b^2
  R bl[3];                                       // b_i = calB_i / W + alpha b^0 v_i
#pragma unroll
  for (int i = 0; i < 3; ++i) bl[i] = Bl[i] * iW + ab0 * vl[i];
  R rhoh, cs2;
  eos_rhoh_cs2<R, EOS>(kp, rho, p, EOS ? w[5] : R(0), &rhoh, &cs2);
  const R e = rhoh + b2;
  const R pt = p + R(0.5) * b2;
  // Eq. consB_def
  U[0] = sg * rho * W;
#pragma unroll
  for (int j = 0; j < 3; ++j) U[1 + j] = sg * (e * W * utl[j] - ab0 * bl[j]);
  U[4] = sg * (e * W * W - rho * W - pt - ab0 * ab0);
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  U[5] = Bd[t1];
  U[6] = Bd[t2];
  // Eq. fluxB_def
  const R avd = alpha * vt[d];
  const R asg = alpha * sg;
  const R BdW = Bu[d] * iW;
  F[0] = U[0] * avd;
#pragma unroll
  for (int j = 0; j < 3; ++j) F[1 + j] = U[1 + j] * avd - asg * bl[j] * BdW;
  F[1 + d] += pt * asg;
  F[4] = U[4] * avd + asg * (pt * v[d] - ab0 * BdW);
  F[5] = alpha * (Bd[t1] * vt[d] - Bd[d] * vt[t1]);
  F[6] = alpha * (Bd[t2] * vt[d] - Bd[d] * vt[t2]);
  // fast speeds
  const R ca2 = rdiv(b2, e);
  const R c2 = cs2 + ca2 - cs2 * ca2;
  const R v2 = v[0] * vl[0] + v[1] * vl[1] + v[2] * vl[2];
  R disc = (R(1) - v2) * (gdd * (R(1) - v2 * c2) - v[d] * v[d] * (R(1) - c2));
  disc = disc > R(0) ? disc : R(0);
  const R cr = sqrt_r(c2) * sqrt_r(disc);
  const R iden = rdiv(R(1), R(1) - v2 * c2);
  const R vc = v[d] * (R(1) - c2);
  *lp = alpha * (vc + cr) * iden - beta[d];
  *lm = alpha * (vc - cr) * iden - beta[d];
}

// HLLE (lam+ = max(0, ...), lam- = min(0, ...); equal speeds give the mean flux)
template <class R>
__device__ __forceinline__ void hlle(const R UL[7], const R UR[7], const R FL[7], const R FR[7], R lmL,
                                     R lpL, R lmR, R lpR, R out[7]) {
  const R lp = rmax(R(0), rmax(lpL, lpR));
  const R lm = rmin(R(0), rmin(lmL, lmR));
  const R den = lp - lm;
  if (den == R(0)) {
#pragma unroll
    for (int v = 0; v < 7; ++v) out[v] = R(0.5) * (FL[v] + FR[v]);
    return;
  }
  const R iden = rdiv(R(1), den);
  const R lpm = lp * lm;
#pragma unroll
  for (int v = 0; v < 7; ++v) out[v] = (lp * FL[v] - lm * FR[v] + lpm * (UR[v] - UL[v])) * iden;
}

// ------------------------------------------------------------------------------------------------
// Cell physics in R: prim -> cons, stress tensor and sources (Eq. EMT_MHD, Eq. hydsrc_def)
// ------------------------------------------------------------------------------------------------
template <class R>
struct CellMet {
  R alpha, beta[3], g[6], K[6], gi[6], sg, det;
};

template <class R>
__device__ __forceinline__ void cellmet_from(const R val[16], bool kzero, CellMet<R>& M) {
  M.alpha = val[0];
  #pragma unroll
  for (int i = 0; i < 3; ++i) M.beta[i] = val[1 + i];
  #pragma unroll
  for (int c = 0; c < 6; ++c) {
    M.g[c] = val[4 + c];
    M.K[c] = kzero ? R(0) : val[10 + c];
  }
  M.det = det3(M.g);
  M.sg = sqrt_r(M.det);
  inv3(M.g, M.det, M.gi);
}

template <class R>
struct CellFluid {
  R rho, p, W, rhoh, b2, ab0;
  R ut[3], utl[3], v[3], vl[3], vt[3];
  R Bu[3], bl[3];
};

template <class R, int EOS>
__device__ __forceinline__ void cell_fluid(const CellMet<R>& M, const KParams& kp, const R w[6], const R Bd[3],
                                           CellFluid<R>& f) {
  f.rho = w[0];
  f.p = w[4];
  #pragma unroll
  for (int i = 0; i < 3; ++i) f.ut[i] = w[1 + i];
  lower3(M.g, f.ut, f.utl);
  f.W = sqrt_w(R(1) + f.ut[0] * f.utl[0] + f.ut[1] * f.utl[1] + f.ut[2] * f.utl[2]);
  const R iW = rdiv(R(1), f.W), ia = rdiv(R(1), M.alpha), isg = rdiv(R(1), M.sg);
  #pragma unroll
  for (int i = 0; i < 3; ++i) {
    f.v[i] = f.ut[i] * iW;
    f.vl[i] = f.utl[i] * iW;
    f.vt[i] = f.v[i] - M.beta[i] * ia;
    f.Bu[i] = Bd[i] * isg;
  }
  R Bl[3];
  lower3(M.g, f.Bu, Bl);
  const R Bv = f.Bu[0] * f.vl[0] + f.Bu[1] * f.vl[1] + f.Bu[2] * f.vl[2];
  const R BB = f.Bu[0] * Bl[0] + f.Bu[1] * Bl[1] + f.Bu[2] * Bl[2];
  f.ab0 = f.W * Bv;
  f.b2 = (f.ab0 * f.ab0 + BB) * iW * iW;
  #pragma unroll
  for (int i = 0; i < 3; ++i) f.bl[i] = Bl[i] * iW + f.ab0 * f.vl[i];
  R cs2;
  eos_rhoh_cs2<R, EOS>(kp, f.rho, f.p, EOS ? w[5] : R(0), &f.rhoh, &cs2);
}

template <class R>
__device__ __forceinline__ void cell_cons(const CellMet<R>& M, const CellFluid<R>& f, R q[5]) {
  const R e = f.rhoh + f.b2, pt = f.p + R(0.5) * f.b2;
  q[0] = M.sg * f.rho * f.W;
  #pragma unroll
  for (int j = 0; j < 3; ++j) q[1 + j] = M.sg * (e * f.W * f.utl[j] - f.ab0 * f.bl[j]);
  q[4] = M.sg * (e * f.W * f.W - f.rho * f.W - pt - f.ab0 * f.ab0);
}

// Eq. hydsrc_def; dm[k][c] = d_k of alpha (c=0), beta^i (1..3), gamma_ij (4..9)
template <class R>
__device__ __forceinline__ void cell_sources(const CellMet<R>& M, const CellFluid<R>& f, const R dm[3][10],
                                             bool kzero, R s[5]) {
  const R a = M.alpha, ia2 = rdiv(R(1), a * a);
  // u^mu, b^mu
  R u[4], b[4];
  u[0] = f.W * rdiv(R(1), a);
  #pragma unroll
  for (int i = 0; i < 3; ++i) u[1 + i] = f.W * f.vt[i];
  b[0] = f.ab0 * rdiv(R(1), a);
  const R iW = rdiv(R(1), f.W);
  #pragma unroll
  for (int i = 0; i < 3; ++i) b[1 + i] = f.Bu[i] * iW + f.ab0 * f.vt[i];
  const R e = f.rhoh + f.b2, pt = f.p + R(0.5) * f.b2;
  // T^{mu nu} = e u u + pt g^{mu nu} - b b, with g^{00} = -1/a^2, g^{0i} = beta^i/a^2,
  // g^{ij} = gamma^{ij} - beta^i beta^j / a^2
  const R T00 = e * u[0] * u[0] - pt * ia2 - b[0] * b[0];
  R T0i[3], Tij[6];
  #pragma unroll
  for (int i = 0; i < 3; ++i) T0i[i] = e * u[0] * u[1 + i] + pt * M.beta[i] * ia2 - b[0] * b[1 + i];
  #pragma unroll
  for (int i = 0; i < 3; ++i)
    #pragma unroll
    for (int j = i; j < 3; ++j) {
      const int c = sidx(i, j);
      Tij[c] = e * u[1 + i] * u[1 + j] + pt * (M.gi[c] - M.beta[i] * M.beta[j] * ia2) - b[1 + i] * b[1 + j];
    }
  // T^0_i = T^{00} beta_i + T^{0j} gamma_ji
  R betal[3], T0l[3];
  lower3(M.g, M.beta, betal);
  lower3(M.g, T0i, T0l);
  #pragma unroll
  for (int i = 0; i < 3; ++i) T0l[i] += T00 * betal[i];
  const R asg = a * M.sg;
  s[0] = R(0);
  #pragma unroll
  for (int k = 0; k < 3; ++k) {
    const R* dg = dm[k] + 4;
    R bbdg = 0, T0bdg = 0, Tdg = 0;
    #pragma unroll
    for (int i = 0; i < 3; ++i)
      #pragma unroll
      for (int j = 0; j < 3; ++j) {
        const R dgij = dg[sidx(i, j)];
        bbdg += M.beta[i] * M.beta[j] * dgij;
        T0bdg += T0i[i] * M.beta[j] * dgij;
        Tdg += Tij[sidx(i, j)] * dgij;
      }
    const R Tdb = T0l[0] * dm[k][1] + T0l[1] * dm[k][2] + T0l[2] * dm[k][3];
    s[1 + k] = asg * (T00 * (R(0.5) * bbdg - a * dm[k][0]) + T0bdg + Tdb + R(0.5) * Tdg);
  }
  R st = 0;
  #pragma unroll
  for (int i = 0; i < 3; ++i) st -= (T00 * M.beta[i] + T0i[i]) * dm[i][0];
  if (!kzero) {
    R bKb = 0, TK = 0;
    #pragma unroll
    for (int i = 0; i < 3; ++i) {
      R bK = 0;
      #pragma unroll
      for (int j = 0; j < 3; ++j) {
        const R Kij = M.K[sidx(i, j)];
        bK += M.beta[j] * Kij;
        TK += Tij[sidx(i, j)] * Kij;
      }
      bKb += M.beta[i] * bK;
      st += R(2) * T0i[i] * bK;
    }
    st += T00 * bKb + TK;
  }
  s[4] = asg * st;
}

// FP64 spatial metric at a cell centre for con2prim: gamma_ij and sqrt(gamma); the inverse is
// formed only for cells that are solved
struct C2PMet {
  double g[6], sg, det;
  double isg;   // 1/sqrt(gamma), formed only by the FAST form
};

// FAST (the mixed stage's con2prim): sqrt(gamma) and its inverse from one reciprocal square root,
// sg = det rsqrt(det), in place of a square root and a division
template <bool FAST = false>
__device__ __forceinline__ void c2pmet_from(const double g6[6], C2PMet& M) {
  for (int c = 0; c < 6; ++c) M.g[c] = g6[c];
  M.det = det3(M.g);
  if constexpr (FAST) {
    M.isg = rsqrt(M.det);
    M.sg = M.det * M.isg;
  } else {
    M.sg = sqrt(M.det);
  }
}

// ------------------------------------------------------------------------------------------------
// Con2prim (Sec. 3.5, App. A): KKC master function in mu = 1/(hW), Illinois bracketing.
// Templated so that an FP32 pre-solve can narrow the FP64 bracket.
// ------------------------------------------------------------------------------------------------
template <class R>
struct C2PInv {
  R D, q, r2, b2, rb;
  R ye;     // table: electron fraction (already inside the table's range)
};
template <class R>
struct C2PVal {
  R x, rbar2, v2, iW, eps, f;
  R rho, p, lT;   // table: density (inside the table), pressure, log T at mu
  R en, ed;       // c2p_master_fast: eps = en / ed, formed only where eps itself is needed
  bool vcap, eclamp;
};

// f(mu) = mu - 1/(nu + mu rbar^2), nu = max(nu_A, nu_B).  For the ideal gas (1 + a)(1 + eps) =
// 1 + Gamma eps, so nu_A = (1 + Gamma eps)/W and nu_B = (1 + Gamma eps)(1 + qbar - mu rbar^2)/(1 + eps);
// eps = W (qbar - mu rbar^2) + v^2 W^2/(1 + W) is formed over the common denominator iW (1 + iW),
// iW = 1/W = sqrt(1 - v^2).
template <class R>
__device__ __forceinline__ void c2p_master(R gam, R vmax2, const C2PInv<R>& I, R mu, C2PVal<R>& E) {
  E.x = rdiv(R(1), R(1) + mu * I.b2);
  E.rbar2 = E.x * E.x * I.r2 + mu * E.x * (R(1) + E.x) * I.rb * I.rb;
  const R qbar = I.q - R(0.5) * I.b2 - R(0.5) * mu * mu * E.x * E.x * (I.b2 * I.r2 - I.rb * I.rb);
  E.v2 = mu * mu * E.rbar2;
  E.vcap = E.v2 > vmax2;
  if (E.vcap) E.v2 = vmax2;
  E.iW = sqrt_r(R(1) - E.v2);
  const R qm = qbar - mu * E.rbar2;
  E.eps = rdiv(qm * (R(1) + E.iW) + E.v2, E.iW * (R(1) + E.iW));
  E.eclamp = E.eps < R(0);
  if (E.eclamp) E.eps = R(0);
  const R ge = R(1) + gam * E.eps;
  const R nuA = ge * E.iW;
  const R nuB = rdiv(ge * (R(1) + qm), R(1) + E.eps);
  const R nu = nuA > nuB ? nuA : nuB;
  E.f = mu - rdiv(R(1), nu + mu * E.rbar2);
}

// The same f(mu) for the ideal gas with two FP64 divisions instead of four (the mixed stage's
// con2prim): eps = n/d with n = qm (1 + iW) + v^2, d = iW (1 + iW) > 0, so eps < 0 iff n < 0,
// 1 + Gamma eps = G/d with G = d + Gamma n, 1 + eps = (d + n)/d, and
//   nu_A = G iW / d,  nu_B = G (1 + qm) / (d + n),  nu_A > nu_B  iff  iW (d + n) > (1 + qm) d;
// with nu = G P / Q for the larger one, f = mu - 1/(nu + mu rbar^2) = mu - Q / (G P + mu rbar^2 Q).
// The same function as c2p_master up to rounding; eps itself (needed only at the root) is left as
// E.en / E.ed.
template <class R>
__device__ __forceinline__ void c2p_master_fast(R gam, R vmax2, const C2PInv<R>& I, R mu, C2PVal<R>& E) {
  E.x = rdiv(R(1), R(1) + mu * I.b2);
  E.rbar2 = E.x * E.x * I.r2 + mu * E.x * (R(1) + E.x) * I.rb * I.rb;
  const R qbar = I.q - R(0.5) * I.b2 - R(0.5) * mu * mu * E.x * E.x * (I.b2 * I.r2 - I.rb * I.rb);
  E.v2 = mu * mu * E.rbar2;
  E.vcap = E.v2 > vmax2;
  if (E.vcap) E.v2 = vmax2;
  E.iW = sqrt_r(R(1) - E.v2);
  const R qm = qbar - mu * E.rbar2;
  const R d = E.iW * (R(1) + E.iW);
  R n = qm * (R(1) + E.iW) + E.v2;
  E.eclamp = n < R(0);
  if (E.eclamp) n = R(0);
  E.en = n;
  E.ed = d;
  const R G = d + gam * n;
  const R dn = d + n, q1 = R(1) + qm;
  const bool a_wins = E.iW * dn > q1 * d;
  const R P = a_wins ? E.iW : q1, Q = a_wins ? d : dn;
  E.f = mu - rdiv(Q, G * P + mu * E.rbar2 * Q);
}

// The same master function with the tabulated EOS (Sec. 2.2.1, App. A): rho = D/W moved into the
// table, the temperature of e/rho = 1 + eps by the exact inverse of the interpolant (eps reset to the
// table's value at the nearest end when outside), p from the table; (1 + a)(1 + eps) = h =
// 1 + eps + p/rho.
template <class R>
__device__ __forceinline__ void c2p_master_tab(const TabView<R>& t, R vmax2, const C2PInv<R>& I, R mu,
                                               C2PVal<R>& E, int* khint) {
  E.x = rdiv(R(1), R(1) + mu * I.b2);
  E.rbar2 = E.x * E.x * I.r2 + mu * E.x * (R(1) + E.x) * I.rb * I.rb;
  const R qbar = I.q - R(0.5) * I.b2 - R(0.5) * mu * mu * E.x * E.x * (I.b2 * I.r2 - I.rb * I.rb);
  E.v2 = mu * mu * E.rbar2;
  E.vcap = E.v2 > vmax2;
  if (E.vcap) E.v2 = vmax2;
  E.iW = sqrt_r(R(1) - E.v2);
  const R qm = qbar - mu * E.rbar2;
  E.eps = rdiv(qm * (R(1) + E.iW) + E.v2, E.iW * (R(1) + E.iW));
  E.rho = I.D * E.iW;
  E.eclamp = false;
  bool cl = false;
  const R lr = rlog(E.rho);
  const TabLoc<R> L = tab_loc(t, lr, I.ye, &cl);
  if (cl) { E.rho = rexp(lr < t.x0[0] ? t.x0[0] : t.hi[0]); E.eclamp = true; cl = false; }
  int k;
  R wT;
  const R y = E.eps > R(-1) ? rlog1p(E.eps) : R(-INFINITY);
  E.lT = tab_inverse_T(t, t.f[1], L, y, &cl, &k, &wT, *khint);
  *khint = k;
  if (cl) { E.eps = rexpm1(tab_T(t, t.f[1], L, k, wT)); E.eclamp = true; }
  E.p = E.rho * rexp(tab_T(t, t.f[0], L, k, wT));
  const R h = (R(1) + E.eps) + rdiv(E.p, E.rho);
  const R nuA = h * E.iW;
  const R nuB = rdiv(h * (R(1) + qm), R(1) + E.eps);
  const R nu = nuA > nuB ? nuA : nuB;
  E.f = mu - rdiv(R(1), nu + mu * E.rbar2);
}

// Auxiliary function mu sqrt(h0^2 + rbar^2(mu)) - 1 whose root bounds the master root from above;
// h0 = minimum enthalpy of the EOS (1 for the ideal gas), passed squared
template <class R>
__device__ __forceinline__ R c2p_aux(const C2PInv<R>& I, R h0sq, R mu) {
  const R x = rdiv(R(1), R(1) + mu * I.b2);
  const R rbar2 = x * x * I.r2 + mu * x * (R(1) + x) * I.rb * I.rb;
  return mu * sqrt_r(h0sq + rbar2) - R(1);
}

// Illinois on [a,b] (f(a) < 0 < f(b) or reverse).  Returns 0 (root), -1 (no sign change), -2 (cap).
// *fresh (optional): whether the root is the point f was last evaluated at.
template <class R, class Fn>
__device__ __forceinline__ int illinois(Fn f, R a, R b, R fa, R fb, R tol, int max_iter, R* root, R* hi_out,
                                        int* iters, bool* fresh = nullptr) {
  *iters = 0;
  if (fresh) *fresh = false;
  if (fa == R(0)) { *root = a; *hi_out = a; return 0; }
  if (fb == R(0)) { *root = b; *hi_out = b; return 0; }
  if ((fa < R(0)) == (fb < R(0))) return -1;
  int side = 0;
  for (int it = 1; it <= max_iter; ++it) {
    R c = rdiv(a * fb - b * fa, fb - fa);
    if (!(c > a && c < b)) c = R(0.5) * (a + b);
    if (!(c > a && c < b)) {
      *root = c; *hi_out = b; *iters = it;
      if (fresh) *fresh = false;   // c itself was not evaluated
      return 0;
    }
    const R fc = f(c);
    *iters = it;
    if (fresh) *fresh = true;
    if (fc == R(0)) { *root = c; *hi_out = c; return 0; }
    if ((fc < R(0)) == (fa < R(0))) {
      a = c; fa = fc;
      if (side == -1) fb *= R(0.5);
      side = -1;
    } else {
      b = c; fb = fc;
      if (side == +1) fa *= R(0.5);
      side = +1;
    }
    if (b - a <= tol * c) { *root = c; *hi_out = b; return 0; }
  }
  *hi_out = b;
  return -2;
}

// FP32 pre-solve: the bracket (0, mu+] of the master root narrowed by Illinois steps in FP32 until its
// width is below 1e-4 of its upper end (at most 12 steps; FP32 evaluations of f carry rounding noise of
// ~1e-7 of their terms, so a tighter FP32 tolerance would only spend steps on noise).  Returns false when
// the FP32 invariants are not finite or f shows no sign change; else [*lo, *hi] with f32(lo) <= 0 <=
// f32(hi), which the FP64 solve widens slightly and verifies by the signs of the FP64 f.
template <int EOS>
__device__ __forceinline__ bool c2p_presolve32(const KParams& P, const C2PInv<double>& I64, float* lo, float* hi) {
  C2PInv<float> I;
  I.D = d2f_rn(I64.D); I.q = d2f_rn(I64.q); I.r2 = d2f_rn(I64.r2); I.b2 = d2f_rn(I64.b2); I.rb = d2f_rn(I64.rb);
  I.ye = d2f_rn(I64.ye);
  if (!(I.D > 0.f) || !isfinite(I.q) || !isfinite(I.r2) || !isfinite(I.b2) || !isfinite(I.rb * I.rb)) return false;
  const float gam = P.gamma_f, vmax2 = P.vmax2_f;
  const float top = EOS ? P.top_f : 1.f, h0sq = EOS ? P.h0sq_f : 1.f;
  float mup = top, root, hiv;
  int it;
  const float f1 = c2p_aux<float>(I, h0sq, top);
  if (f1 > 0.f) {
    auto fa = [&](float mu) { return c2p_aux<float>(I, h0sq, mu); };
    if (illinois<float>(fa, 0.f, top, -1.f, f1, 1e-3f, 40, &root, &hiv, &it) == 0) mup = hiv;
  }
  C2PVal<float> E;
  int kh = -1;   // temperature interval of the last evaluation (table)
  auto fm = [&](float mu) {
    if constexpr (EOS == GR_EOS_IDEAL) c2p_master_fast<float>(gam, vmax2, I, mu, E);
    else c2p_master_tab<float>(P.t32, vmax2, I, mu, E, &kh);
    return E.f;
  };
  float a = 0.f, b = mup;
  float fa = fm(a), fb = fm(b);
  if (!(fb >= 0.f) && mup < top) { b = top; fb = fm(b); }
  if (!(fa < 0.f) || !(fb >= 0.f)) return false;
  int side = 0;
  for (int k = 0; k < 12 && b - a > 1e-4f * b; ++k) {
    float c = __fdividef(a * fb - b * fa, fb - fa);
    if (!(c > a && c < b)) c = 0.5f * (a + b);
    if (!(c > a && c < b)) break;
    const float fc = fm(c);
    if (fc == 0.f) { a = c; b = c; break; }
    if (fc < 0.f) {
      a = c; fa = fc;
      if (side == -1) fb *= 0.5f;
      side = -1;
    } else {
      b = c; fb = fc;
      if (side == +1) fa *= 0.5f;
      side = +1;
    }
  }
  *lo = a;
  *hi = b;
  return true;
}

// Invariants and root of a bracketed solve (training samples for the learned bracket)
struct C2PRecord {
  double q, r2, b2, rb, mu, D, ye;
  bool solved;
};

// Conserved variables of a primitive state at a point with spatial metric M (Eq. consB_def needs
// only gamma_ij): used to rebuild q after a temperature floor.  w: (rho, u~^i, p[, Y_e]).
template <int EOS>
__device__ __forceinline__ void cons_at(const C2PMet& M, const KParams& P, const double w[6], const double Bd[3],
                                        double q[6]) {
  CellMet<double> Mc;
  Mc.alpha = 1.0;
  for (int i = 0; i < 3; ++i) Mc.beta[i] = 0.0;
  for (int c = 0; c < 6; ++c) { Mc.g[c] = M.g[c]; Mc.K[c] = 0.0; }
  Mc.det = M.det;
  Mc.sg = M.sg;
  inv3(Mc.g, Mc.det, Mc.gi);
  CellFluid<double> f;
  cell_fluid<double, EOS>(Mc, P, w, Bd, f);
  cell_cons<double>(Mc, f, q);
  if (EOS) q[5] = q[0] * w[5];
}

// Atmosphere primitives (Sec. 3.5, App. A) and their conserved variables, Eq. consB_def at u~ = 0:
// W = 1, b^0 = 0, b^2 = calB^2, so D = sqrt(gamma) rho, S_j = 0,
// tau = sqrt(gamma) (rho eps + calB^2 / 2) = sqrt(gamma) rho eps + gamma_ij B^i B^j/(2 sqrt(gamma))
template <int EOS>
__device__ __forceinline__ void atm_cell(const C2PMet& M, const KParams& P, const double Bd[3], double q[6],
                                         double w[7]) {
  w[0] = P.rho_atm;
  w[1] = w[2] = w[3] = 0.0;
  w[4] = P.p_atm;
  double Bl[3];
  lower3(M.g, Bd, Bl);
  const double BBd = Bd[0] * Bl[0] + Bd[1] * Bl[1] + Bd[2] * Bl[2];
  q[0] = M.sg * P.rho_atm;
  q[1] = q[2] = q[3] = 0.0;
  q[4] = M.sg * P.eint_atm + (BBd == 0.0 ? 0.0 : 0.5 * BBd / M.sg);
  if constexpr (EOS == GR_EOS_TABLE) {
    w[5] = P.Ye_atm;
    w[6] = P.T_atm;
    q[5] = q[0] * P.Ye_atm;
  }
}

// Full con2prim of one cell.  q: densitised conserved (in/out; q[5] = D Y_e with a table), Bd:
// densitised cell field, w: primitives out (w[5], w[6] = Y_e, T with a table).
// guess: GR_GUESS_NONE (bracket (0, mu+]), GR_GUESS_FP32 (c2p_presolve32's FP32 bracket widened by 4e-6
// of its ends; it is used only if the FP64 master function changes sign across it, else the full bracket
// is used and GR_ST_GUESS_REJECTED is set) or GR_GUESS_MLP (GR_GUESS_AUTO is resolved on the host).
// FAST (the mixed stage): the upper end mu+ of the bracket from the auxiliary function in FP32 (its
// tolerance is 1e-3; a bound that turns out too low is caught by the sign test and replaced by 1/h0),
// and for the ideal gas the two-division form of the master function (c2p_master_fast).  The root is
// still bracketed in FP64 to the same tolerance; only the bracket's upper end and the rounding of f
// differ from the plain form.
template <int EOS, bool FAST = false>
__device__ __forceinline__ int con2prim_cell(const C2PMet& M, const KParams& P, double q[6],
                                             const double Bd[3], double w[7], int* iters,
                                             C2PRecord* rec = nullptr) {
  int st = 0;
  *iters = 0;
  if (rec) rec->solved = false;
  bool finite = isfinite(q[0]) && isfinite(q[4]);
  for (int i = 0; i < 3; ++i) finite = finite && isfinite(q[1 + i]) && isfinite(Bd[i]);
  // table: Y_e = (D Y_e)/D moved into the table's range (App. A)
  double ye = 0.0;
  bool ye_clamped = false;
  if constexpr (EOS == GR_EOS_TABLE) {
    finite = finite && isfinite(q[5]);
    const double ylo = P.t64.x0[2], yhi = P.t64.hi[2];
    ye = (finite && q[0] != 0.0) ? q[5] / q[0] : ylo;
    if (ye < ylo) { ye = ylo; ye_clamped = true; }
    if (ye > yhi) { ye = yhi; ye_clamped = true; }
  }
  // atmosphere threshold f_thr rho_atm (1 + atm_band); values within the band count as having reached it
  const double rho_thr = P.rho_thr;
  bool atm = false, reprim = false;
  if (!finite) { st |= GR_ST_FAILED; atm = true; }
  else if (q[0] < rho_thr * M.sg) { st |= GR_ST_ATM_THRESHOLD; atm = true; }   // D~ < rho_thr
  double isg = 0.0;
  if (!atm) {
    if constexpr (FAST) isg = M.isg;
    else isg = 1.0 / M.sg;
    double D = q[0] * isg, tau = q[4] * isg, S[3], Bu[3];
    for (int i = 0; i < 3; ++i) {
      S[i] = q[1 + i] * isg;
      Bu[i] = Bd[i] * isg;
    }
    double Bl[3];
    lower3(M.g, Bu, Bl);
    const double BB = Bu[0] * Bl[0] + Bu[1] * Bl[1] + Bu[2] * Bl[2];
    bool qmod = false;
    if (BB > P.M_max * D) { D = BB / P.M_max; st |= GR_ST_BD_LIMIT; qmod = true; }
    // tau floor of a static cold fluid with the same field: D eps(rho = D, T_min) + B^2/2
    double eps_min = 0.0;
    if constexpr (EOS == GR_EOS_TABLE) {
      double pm;
      tab_p_eps_T<double>(P.t64, D, P.t64.x0[1], ye, &pm, &eps_min);
    }
    const double tau_min = D * eps_min + 0.5 * BB;
    if (tau < tau_min) { tau = tau_min; st |= GR_ST_TAU_FLOOR; qmod = true; }
    double gi[6];
    if constexpr (FAST) inv3_id(M.g, isg * isg, gi);   // 1/det = (1/sqrt(gamma))^2
    else inv3(M.g, M.det, gi);
    C2PInv<double> I;
    I.D = D;
    I.ye = ye;
    double iD, isD;
    if constexpr (FAST) {   // 1/sqrt(D) from one reciprocal square root, 1/D its square
      isD = rsqrt(D);
      iD = isD * isD;
    } else {
      iD = 1.0 / D;
      isD = sqrt(iD);
    }
    I.q = tau * iD;
    double rl[3], ru[3], bu[3];
    for (int i = 0; i < 3; ++i) { rl[i] = S[i] * iD; bu[i] = Bu[i] * isD; }
    ru[0] = gi[0] * rl[0] + gi[1] * rl[1] + gi[2] * rl[2];
    ru[1] = gi[1] * rl[0] + gi[3] * rl[1] + gi[4] * rl[2];
    ru[2] = gi[2] * rl[0] + gi[4] * rl[1] + gi[5] * rl[2];
    I.r2 = rl[0] * ru[0] + rl[1] * ru[1] + rl[2] * ru[2];
    I.rb = rl[0] * bu[0] + rl[1] * bu[1] + rl[2] * bu[2];
    I.b2 = BB * iD;
    const double gam = P.gamma_ad, vmax2 = P.vmax2;
    // upper end of the bracket search: mu <= 1/h0
    const double top = EOS ? P.top : 1.0, h0sq = EOS ? P.h0sq : 1.0;
    C2PVal<double> E;
    int nevals = 0;   // FP64 master-function evaluations (reported through *iters)
    int kh = -1;      // temperature interval of the last evaluation (table)
    bool fresh = false;   // E holds f's values at the root (the solve's last evaluation was there)
    auto fm = [&](double mu) {
      ++nevals;
      if constexpr (EOS == GR_EOS_IDEAL && FAST) c2p_master_fast<double>(gam, vmax2, I, mu, E);
      else if constexpr (EOS == GR_EOS_IDEAL) c2p_master<double>(gam, vmax2, I, mu, E);
      else c2p_master_tab<double>(P.t64, vmax2, I, mu, E, &kh);
      return E.f;
    };
    double root = 0.0, hi;
    int r = -1;
    int it_master = 0;
    if (P.c2p_guess == GR_GUESS_FP32) {
      float lo32, hi32;
      if (c2p_presolve32<EOS>(P, I, &lo32, &hi32)) {
        // the FP32 bracket widened by 4e-6 of its ends (a few FP32 roundings of f near the root)
        const double lo = f2d_exact(lo32) * (1.0 - 4e-6), up = fmin(f2d_exact(hi32) * (1.0 + 4e-6), top);
        const double flo = fm(lo), fup = fm(up);
        if (flo <= 0.0 && fup >= 0.0) r = illinois<double>(fm, lo, up, flo, fup, P.tol, P.max_iter, &root, &hi, &it_master, &fresh);
      }
      if (r != 0) st |= GR_ST_GUESS_REJECTED;
    } else if (P.c2p_guess == GR_GUESS_MLP && P.mlp) {
      // learned bracket: start at the network's prediction mu_hat of the root and step outwards
      // geometrically (factor exp(delta 2^k), k = 0..5) in the direction the sign of f points,
      // until f changes sign; that bracket, verified by the sign change, goes to the Illinois solve
      float f[kMlpIn];
      c2p_features(I.q, I.r2, I.b2, I.rb, f);
      f[4] = EOS ? (float)log(D) : 0.f;
      f[5] = EOS ? (float)ye : 0.f;
      const float th = __ldg(P.mlp + kMlpTMean) + __ldg(P.mlp + kMlpTStd) * mlp_z(P.mlp, f);
      const double dl = (double)__ldg(P.mlp + kMlpStep);
      double m0 = fmin((double)__expf(th), top);
      if (m0 > 0.0) {
        double f0 = fm(m0);
        if (f0 == 0.0) {
          root = m0;
          r = 0;
          fresh = true;
        } else {
          const double dir = f0 < 0.0 ? 1.0 : -1.0;   // f < 0 below the root
          double step = dl;
          for (int k = 0; k < 6 && r != 0; ++k, step *= 2.0) {
            const double m1 = fmin(m0 * exp(dir * step), top);
            if (!(m1 > 0.0) || m1 == m0) break;
            const double f1 = fm(m1);
            if ((f1 < 0.0) != (f0 < 0.0) || f1 == 0.0) {
              const double a = fmin(m0, m1), bnd = fmax(m0, m1);
              const double fa = (a == m0) ? f0 : f1, fb = (a == m0) ? f1 : f0;
              r = illinois<double>(fm, a, bnd, fa, fb, P.tol, P.max_iter, &root, &hi, &it_master, &fresh);
              break;
            }
            m0 = m1;
            f0 = f1;
          }
        }
      }
      if (r != 0) st |= GR_ST_GUESS_REJECTED;
    }
    if (r != 0) {
      // bracket (0, mu+], mu+ from the auxiliary function on (0, 1/h0]
      double mup = top;
      int it_aux;
      bool aux_done = false;
      if constexpr (FAST) {
        C2PInv<float> If;
        If.D = d2f_rn(I.D); If.q = d2f_rn(I.q); If.r2 = d2f_rn(I.r2); If.b2 = d2f_rn(I.b2); If.rb = d2f_rn(I.rb);
        If.ye = 0.f;
        if (isfinite(If.r2) && isfinite(If.b2) && isfinite(If.rb * If.rb)) {
          const float topf = EOS ? P.top_f : 1.f, h0sqf = EOS ? P.h0sq_f : 1.f;
          const float f1 = c2p_aux<float>(If, h0sqf, topf);
          float rootf, hif;
          if (f1 > 0.f) {
            auto fa = [&](float mu) { return c2p_aux<float>(If, h0sqf, mu); };
            if (illinois<float>(fa, 0.f, topf, -1.f, f1, 1e-3f, P.max_iter, &rootf, &hif, &it_aux) == 0)
              mup = fmin(f2d_exact(hif), top);
          }
          aux_done = true;
        }
      }
      if (!aux_done) {
        const double f1 = c2p_aux<double>(I, h0sq, top);
        if (f1 > 0.0) {
          auto fa = [&](double mu) { return c2p_aux<double>(I, h0sq, mu); };
          if (illinois<double>(fa, 0.0, top, -1.0, f1, 1e-3, P.max_iter, &root, &hi, &it_aux) == 0) mup = hi;
        }
      }
      const double f0 = fm(0.0);
      double fp = fm(mup);
      if ((f0 < 0.0) == (fp < 0.0) && mup < top) { mup = top; fp = fm(mup); }
      r = illinois<double>(fm, 0.0, mup, f0, fp, P.tol, P.max_iter, &root, &hi, &it_master, &fresh);
    }
    *iters = nevals;
    if (r != 0) {
      st |= GR_ST_FAILED;
      atm = true;
    } else {
      const double mu = root;
      if (rec) {
        rec->q = I.q; rec->r2 = I.r2; rec->b2 = I.b2; rec->rb = I.rb; rec->mu = mu; rec->D = D; rec->ye = ye;
        rec->solved = true;
      }
      // E at the root: the solve's last evaluation is usually there already (the ideal-gas master
      // function is a pure function of mu, so the values are the ones a new evaluation would give)
      if constexpr (EOS == GR_EOS_IDEAL && FAST) {
        if (!fresh) c2p_master_fast<double>(gam, vmax2, I, mu, E);
        E.eps = E.en / E.ed;
      } else if constexpr (EOS == GR_EOS_IDEAL) {
        if (!fresh) c2p_master<double>(gam, vmax2, I, mu, E);
      } else {
        c2p_master_tab<double>(P.t64, vmax2, I, mu, E, &kh);
      }
      double vu[3];
      for (int i = 0; i < 3; ++i) vu[i] = mu * E.x * (ru[i] + mu * I.rb * bu[i]);
      if (E.vcap) {
        st |= GR_ST_W_CLAMPED;
        const double s = sqrt(E.v2 / (mu * mu * E.rbar2));
        for (int i = 0; i < 3; ++i) vu[i] *= s;
        if (P.ceiling == GR_CEIL_ATMOSPHERE) atm = true;
      }
      if (E.eclamp || ye_clamped) st |= GR_ST_EOS_CLAMP;
      const double rho = EOS ? E.rho : D * E.iW;
      if (rho < rho_thr) { st |= GR_ST_ATM_THRESHOLD; atm = true; }
      if (!atm) {
        const double W = 1.0 / E.iW;
        w[0] = rho;
        for (int i = 0; i < 3; ++i) w[1 + i] = W * vu[i];
        if constexpr (EOS == GR_EOS_IDEAL) {
          w[4] = (P.gamma_ad - 1.0) * rho * E.eps;
        } else {
          w[4] = E.p;
          w[5] = ye;
          w[6] = exp(E.lT);
          // temperature floor (App. A): T below T_atm -> T_atm, p recomputed, conserved rebuilt
          if (w[6] < P.T_atm) {
            double eps;
            tab_p_eps_T<double>(P.t64, rho, log(P.T_atm), ye, &w[4], &eps);
            w[6] = P.T_atm;
            st |= GR_ST_EOS_CLAMP;
            reprim = true;
          }
          if (ye_clamped) qmod = true;
        }
        if (qmod) {
          q[0] = M.sg * D; q[4] = M.sg * tau;
          if (EOS) q[5] = q[0] * ye;
        }
      }
    }
  }
  if (atm) {
    atm_cell<EOS>(M, P, Bd, q, w);
  } else if (reprim) {
    cons_at<EOS>(M, P, w, Bd, q);
  }
  return st;
}

}  // namespace grs
