// amr.cu -- level-boundary operators of a refined mesh (Sec. 3.3, last paragraph: divergence- and
// curl-preserving restriction and prolongation of the face field, flux and electric-field corrections
// at refinement boundaries), refinement ratio 2.
//
//   k_restrict_cells  coarse cell = mean of its 8 fine cells (densitised conserved variables: conservative)
//   k_restrict_faces  coarse face = mean of the 4 fine faces on it (same flux through the face)
//   k_prolong_cells   limited linear: u_c + (s_x dx + s_y dy + s_z dz)/4, d_ = minmod of the one-sided
//                     coarse differences, s_ = +-1 the fine cell's side
//   k_prolong_faces   a fine face on a coarse face: the coarse value plus the limited transverse slopes
//                     of the coarse face plane; a fine face inside a coarse cell: the mean of the two
//                     opposite outer fine faces plus the minimal-norm correction that makes the 8 fine
//                     cells divergence-free (solved on fluxes, value x face area)
//   k_level_fix       inside the stage, after the corner EMFs: a coarse face on a level boundary takes
//                     the mean of the 4 fine-face fluxes on it, a coarse edge the mean of the 2 fine
//                     edge EMFs along it
// A fine cell i along an axis covers half of coarse cell off + floor(i/2).
#include "internal.h"
#include "physics.cuh"
#include "stage_common.cuh"

namespace grs {

__device__ __forceinline__ double minmod(double a, double b) {
  return a * b <= 0.0 ? 0.0 : (fabs(a) < fabs(b) ? a : b);
}

__device__ __forceinline__ int floor2(int i) { return i >= 0 ? i >> 1 : -((-i + 1) >> 1); }

// coordinates of element e of the box lo..hi-1 (x fastest)
__device__ __forceinline__ void box_decode(int e, const int lo[3], const int ext[3], int p[3]) {
  p[0] = lo[0] + e % ext[0];
  p[1] = lo[1] + (e / ext[0]) % ext[1];
  p[2] = lo[2] + e / (ext[0] * ext[1]);
}

struct AmrArgs {
  double* cells[8];   // cell pools to restrict / prolong
  int nvar;
  double* B[3];       // face pools, or NULL
};

// ---- restriction -----------------------------------------------------------------------------
// Work: block = map index, dir = element kind (0 cells, 1 + d: d-faces), start
__global__ void __launch_bounds__(kTile) k_restrict(const DBlock* __restrict__ blocks, const LevelMap* __restrict__ maps,
                                                    const Work* __restrict__ work, const __grid_constant__ AmrArgs a) {
  const Work w = work[blockIdx.x];
  const LevelMap mp = maps[w.block];
  const DBlock c = blocks[mp.coarse], f = blocks[mp.fine];
  const int D = w.dir - 1;
  int ext[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) ext[t] = mp.hi[t] - mp.lo[t] + (t == D);
  const int e = w.start + threadIdx.x;
  if (e >= ext[0] * ext[1] * ext[2]) return;
  int p[3], q[3];
  box_decode(e, mp.lo, ext, p);
#pragma unroll
  for (int t = 0; t < 3; ++t) q[t] = 2 * (p[t] - mp.off[t]);
  if (D < 0) {
    const long long cc = c.cell + cix(c, p[0], p[1], p[2]);
    const long long f0 = f.cell + cix(f, q[0], q[1], q[2]);
    const long long sy = f.N[0], sz = (long long)f.N[0] * f.N[1];
    for (int v = 0; v < a.nvar; ++v) {
      const double* u = a.cells[v] + f0;
      const double s = ((u[0] + u[1]) + (u[sy] + u[sy + 1])) + ((u[sz] + u[sz + 1]) + (u[sz + sy] + u[sz + sy + 1]));
      a.cells[v][cc] = 0.125 * s;
    }
  } else {
    // a range wholly outside the block along D (a ghost slab) leaves the block's own face planes 0, n
    if ((mp.hi[D] <= 0 || mp.lo[D] >= c.n[D]) && (p[D] == 0 || p[D] == c.n[D])) return;
    const int t1 = (D + 1) % 3, t2 = (D + 2) % 3;
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        int r[3] = {q[0], q[1], q[2]};
        r[t1] += u;
        r[t2] += v;
        s = s + a.B[D][f.face[D] + fix(f, D, r[0], r[1], r[2])];
      }
    a.B[D][c.face[D] + fix(c, D, p[0], p[1], p[2])] = 0.25 * s;
  }
}

// ---- prolongation ----------------------------------------------------------------------------
// the 4 fine d-faces on coarse d-face cf: value at transverse sides (s1, s2) in {-1, +1}
__device__ __forceinline__ double outer_face(const DBlock& c, const double* __restrict__ B, int d, const int cf[3],
                                             int s1, int s2) {
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  const double b0 = B[c.face[d] + fix(c, d, cf[0], cf[1], cf[2])];
  double sl[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int t = q == 0 ? t1 : t2;
    int m[3] = {cf[0], cf[1], cf[2]}, pp[3] = {cf[0], cf[1], cf[2]};
    m[t] -= 1;
    pp[t] += 1;
    const double bm = B[c.face[d] + fix(c, d, m[0], m[1], m[2])];
    const double bp = B[c.face[d] + fix(c, d, pp[0], pp[1], pp[2])];
    sl[q] = minmod(bp - b0, b0 - bm);
  }
  return b0 + 0.25 * s1 * sl[0] + 0.25 * s2 * sl[1];
}

// an interior fine d-face of coarse cell cc at transverse sides (s1, s2): mean of the two opposite outer
// fine faces plus the minimal-norm divergence correction (fluxes: value x fine face area)
__device__ double inner_face(const DBlock& c, const AmrArgs& a, const double dxf[3], const int cc[3], int d, int s1,
                             int s2) {
  const double area[3] = {dxf[1] * dxf[2], dxf[0] * dxf[2], dxf[0] * dxf[1]};
  // Dd at the transverse position of each fine cell: high outer minus low outer flux
  // Dd[dd][x][y]: (x, y) = the transverse sides (along (dd+1)%3, (dd+2)%3) as 0 / 1
  double Dd[3][2][2], lo_out[2][2] = {{0, 0}, {0, 0}}, hi_out[2][2] = {{0, 0}, {0, 0}};
#pragma unroll
  for (int dd = 0; dd < 3; ++dd) {
    int cl[3] = {cc[0], cc[1], cc[2]}, ch[3] = {cc[0], cc[1], cc[2]};
    ch[dd] += 1;
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int y = 0; y < 2; ++y) {
        const double l = outer_face(c, a.B[dd], dd, cl, 2 * x - 1, 2 * y - 1) * area[dd];
        const double h = outer_face(c, a.B[dd], dd, ch, 2 * x - 1, 2 * y - 1) * area[dd];
        Dd[dd][x][y] = h - l;
        if (dd == d) { lo_out[x][y] = l; hi_out[x][y] = h; }
      }
  }
  // R at fine cell (a, b, c) (sides as 0/1 along x, y, z): (Dx(b,c) + Dy(c,a) + Dz(a,b)) / 2, with the
  // transverse order of Dd[dd] = ((dd+1)%3, (dd+2)%3): x -> (y, z), y -> (z, x), z -> (x, y)
  double r[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // monomials 1, a, b, c, ab, ac, bc, abc
#pragma unroll
  for (int ia = 0; ia < 2; ++ia)
#pragma unroll
    for (int ib = 0; ib < 2; ++ib)
#pragma unroll
      for (int ic = 0; ic < 2; ++ic) {
        const double R = 0.5 * (Dd[0][ib][ic] + Dd[1][ic][ia] + Dd[2][ia][ib]);
        const double sa = 2 * ia - 1, sb = 2 * ib - 1, sc = 2 * ic - 1;
        r[1] += R * sa;
        r[2] += R * sb;
        r[3] += R * sc;
        r[4] += R * sa * sb;
        r[5] += R * sa * sc;
        r[6] += R * sb * sc;
        r[7] += R * sa * sb * sc;
      }
#pragma unroll
  for (int m = 1; m < 8; ++m) r[m] = r[m] / 8.0;
  // correction of the interior face; (s1, s2) are its sides along (d+1)%3, (d+2)%3
  double corr;
  if (d == 0) {        // X_bc, b = s1 (y), c = s2 (z)
    corr = r[1] + 0.5 * r[4] * s1 + 0.5 * r[5] * s2 + r[7] / 3.0 * s1 * s2;
  } else if (d == 1) { // Y_ac, c = s1 (z), a = s2 (x)
    corr = r[2] + 0.5 * r[4] * s2 + 0.5 * r[6] * s1 + r[7] / 3.0 * s2 * s1;
  } else {             // Z_ab, a = s1 (x), b = s2 (y)
    corr = r[3] + 0.5 * r[5] * s1 + 0.5 * r[6] * s2 + r[7] / 3.0 * s1 * s2;
  }
  const int x = (s1 + 1) / 2, y = (s2 + 1) / 2;
  return (0.5 * (lo_out[x][y] + hi_out[x][y]) + corr) / area[d];
}

__global__ void __launch_bounds__(kTile) k_prolong(const DBlock* __restrict__ blocks, const LevelMap* __restrict__ maps,
                                                   const Work* __restrict__ work, const __grid_constant__ AmrArgs a) {
  const Work w = work[blockIdx.x];
  const LevelMap mp = maps[w.block];
  const DBlock c = blocks[mp.coarse], f = blocks[mp.fine];
  const int D = w.dir - 1;
  int ext[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) ext[t] = mp.hi[t] - mp.lo[t] + (t == D);
  const int e = w.start + threadIdx.x;
  if (e >= ext[0] * ext[1] * ext[2]) return;
  int p[3];
  box_decode(e, mp.lo, ext, p);
  if (D < 0) {
    int cc[3], side[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int q = floor2(p[t]);
      cc[t] = q + mp.off[t];
      side[t] = p[t] - 2 * q ? 1 : -1;
    }
    const long long c0 = c.cell + cix(c, cc[0], cc[1], cc[2]);
    const long long st[3] = {1, c.N[0], (long long)c.N[0] * c.N[1]};
    const long long fc = f.cell + cix(f, p[0], p[1], p[2]);
    for (int v = 0; v < a.nvar; ++v) {
      const double* u = a.cells[v];
      const double u0 = u[c0];
      double val = u0;
#pragma unroll
      for (int t = 0; t < 3; ++t) val = val + 0.25 * side[t] * minmod(u[c0 + st[t]] - u0, u0 - u[c0 - st[t]]);
      a.cells[v][fc] = val;
    }
    return;
  }
  if ((mp.hi[D] <= 0 || mp.lo[D] >= f.n[D]) && (p[D] == 0 || p[D] == f.n[D])) return;   // as in k_restrict
  const int t1 = (D + 1) % 3, t2 = (D + 2) % 3;
  double val;
  if ((p[D] & 1) == 0) {   // on a coarse face plane
    int cf[3];
    cf[D] = floor2(p[D]) + mp.off[D];
    const int q1 = floor2(p[t1]), q2 = floor2(p[t2]);
    cf[t1] = q1 + mp.off[t1];
    cf[t2] = q2 + mp.off[t2];
    val = outer_face(c, a.B[D], D, cf, p[t1] - 2 * q1 ? 1 : -1, p[t2] - 2 * q2 ? 1 : -1);
  } else {                 // inside a coarse cell
    int cc[3];
    cc[D] = floor2(p[D]) + mp.off[D];
    const int q1 = floor2(p[t1]), q2 = floor2(p[t2]);
    cc[t1] = q1 + mp.off[t1];
    cc[t2] = q2 + mp.off[t2];
    val = inner_face(c, a, f.dx, cc, D, p[t1] - 2 * q1 ? 1 : -1, p[t2] - 2 * q2 ? 1 : -1);
  }
  a.B[D][f.face[D] + fix(f, D, p[0], p[1], p[2])] = val;
}

// ---- flux and EMF corrections (inside the stage) ---------------------------------------------
template <class R>
__global__ void __launch_bounds__(kTile) k_level_fix(const DBlock* __restrict__ blocks,
                                                     const LevelFace* __restrict__ lf,
                                                     const __grid_constant__ Workspace ws, int table) {
  const LevelFace r = lf[blockIdx.x];
  const DBlock c = blocks[r.coarse], f = blocks[r.fine];
  const int d = r.dir, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  const int n1 = f.n[t1] / 2, n2 = f.n[t2] / 2;
  const int pc = r.side > 0 ? c.n[d] : 0, pf = r.side > 0 ? 0 : f.n[d];
  auto at = [&](int pd, int a1, int a2, int q[3]) { q[d] = pd; q[t1] = a1; q[t2] = a2; };
  // fluxes of the conserved variables (components 0..4, 7 = D Y_e with a table)
  R* F = reinterpret_cast<R*>(ws.flux[d]);
  const long long sf = ws.fstride[d];
  for (int e = threadIdx.x; e < n1 * n2; e += blockDim.x) {
    const int J = r.o1 + e % n1, K = r.o2 + e / n1;
    int q[3];
    at(pc, J, K, q);
    const long long co = c.wface[d] + fix(c, d, q[0], q[1], q[2]);
    long long fo[4];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        at(pf, 2 * (J - r.o1) + u, 2 * (K - r.o2) + v, q);
        fo[2 * u + v] = f.wface[d] + fix(f, d, q[0], q[1], q[2]);
      }
    for (int k = 0; k < (table ? 6 : 5); ++k) {
      const int comp = k < 5 ? k : 7;
      const R* s = F + comp * sf;
      F[comp * sf + co] = R(0.25) * ((s[fo[0]] + s[fo[1]]) + (s[fo[2]] + s[fo[3]]));
    }
  }
  // corner EMFs on the face plane: E_t1 at (cell J along t1, vertex K along t2), E_t2 likewise
  R* E1 = reinterpret_cast<R*>(ws.edge[t1]);
  R* E2 = reinterpret_cast<R*>(ws.edge[t2]);
  const int ne1 = n1 * (n2 + 1), ne2 = (n1 + 1) * n2;
  for (int e = threadIdx.x; e < ne1 + ne2; e += blockDim.x) {
    int q[3];
    if (e < ne1) {
      const int J = r.o1 + e % n1, K = r.o2 + e / n1;
      at(pf, 2 * (J - r.o1), 2 * (K - r.o2), q);
      const long long fa = f.wvert + vix(f, q[0], q[1], q[2]);
      const long long fb = fa + (t1 == 0 ? 1 : (t1 == 1 ? (long long)(f.N[0] + 1) : (long long)(f.N[0] + 1) * (f.N[1] + 1)));
      at(pc, J, K, q);
      E1[c.wvert + vix(c, q[0], q[1], q[2])] = R(0.5) * (E1[fa] + E1[fb]);
    } else {
      const int e2 = e - ne1;
      const int J = r.o1 + e2 % (n1 + 1), K = r.o2 + e2 / (n1 + 1);
      at(pf, 2 * (J - r.o1), 2 * (K - r.o2), q);
      const long long fa = f.wvert + vix(f, q[0], q[1], q[2]);
      const long long fb = fa + (t2 == 0 ? 1 : (t2 == 1 ? (long long)(f.N[0] + 1) : (long long)(f.N[0] + 1) * (f.N[1] + 1)));
      at(pc, J, K, q);
      E2[c.wvert + vix(c, q[0], q[1], q[2])] = R(0.5) * (E2[fa] + E2[fb]);
    }
  }
}

cudaError_t launch_level_fix(int precision, const DBlock* blocks, const LevelFace* lf, int nlf, const Workspace& ws,
                             int table, cudaStream_t st) {
  if (!nlf) return cudaSuccess;
  if (precision == GR_PREC_MIXED) k_level_fix<float><<<nlf, kTile, 0, st>>>(blocks, lf, ws, table);
  else k_level_fix<double><<<nlf, kTile, 0, st>>>(blocks, lf, ws, table);
  return cudaGetLastError();
}

cudaError_t launch_amr(bool prolong, const DBlock* blocks, const LevelMap* maps, const Work* work, int nwork,
                       double* const cells[8], int nvar, double* const B[3], cudaStream_t st) {
  if (!nwork) return cudaSuccess;
  AmrArgs a;
  for (int v = 0; v < 8; ++v) a.cells[v] = v < nvar ? cells[v] : nullptr;
  a.nvar = nvar;
  for (int d = 0; d < 3; ++d) a.B[d] = B ? B[d] : nullptr;
  if (prolong) k_prolong<<<nwork, kTile, 0, st>>>(blocks, maps, work, a);
  else k_restrict<<<nwork, kTile, 0, st>>>(blocks, maps, work, a);
  return cudaGetLastError();
}

}  // namespace grs
