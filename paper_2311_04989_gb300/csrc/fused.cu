// fused.cu -- k_fused: the mixed path's reconstruction (Sec. 3.4), HLLE face fluxes (Eq. fluxB_def),
// upwinded corner EMFs and CT face update (Sec. 3.3) and flux divergence with the atmosphere test
// (Eq. claw, Sec. 3.5) of a block in one pass, the fluxes and EMFs never leaving shared memory.
//
// One CTA per block walks it along z.  Shared memory holds rings of planes: the FP32 primitives and cell
// field of six cell planes (the z-faces' stencil), three vertex planes of the metric, three planes of the
// cell electric field, the face fluxes of two cell planes (x, y faces) and three vertex planes (z faces),
// the corner EMFs of two planes, and the cell metric of two planes.  Step t of the walk:
//   faces     x- and y-faces of cell plane t - 1 and z-faces of vertex plane t (one list, all threads)
//   prefetch  (cp.async) the planes step t + 1 adds, overlapping the three phases below
//   edges     E_x, E_y on vertex plane t - 1, E_z and the cell metric of cell plane t - 1
//   CT        B' on the x- and y-faces of cell plane t - 2 and the z-faces of vertex plane t - 1
//   update    D' of cell plane t - 2, the atmosphere test and reset; U' of the other cells, queued for
//             con2prim (k_c2p on the compacted job list, as on the separate-kernel path)
// Every face, edge and cell is computed with the operations, in the order, of the separate kernels
// (face_body, edge_body, ct_body, update_cell with k_c2p's U'), so the two paths agree bitwise.  Made for
// blocks of up to 16 x 16 cells in x-y with 3 ghosts (any length in z), the ideal-gas EOS and the order-2
// metric; the host uses it only where every block of the mesh qualifies.
#include "faces_core.cuh"
#include "internal.h"
#include "physics.cuh"
#include "stage_common.cuh"
#include "update_common.cuh"

namespace grs {

constexpr int kFT = 512;                       // threads per CTA
constexpr int kFM = 16;                        // largest interior extent along x and y
constexpr int kFP = kFM + 6;                   // side of a stored cell plane (cells -3 .. n + 2)
constexpr int kFPA = kFP * kFP;
constexpr int kFVS = kFM + 3;                  // side of a stored vertex plane (vertices -1 .. n + 1)
constexpr int kFVA = kFVS * kFVS;
constexpr int kFES = kFM + 2;                  // side of the ring -1 .. n (cell E, z-faces)
constexpr int kFEA = kFES * kFES;
constexpr int kFXF = (kFM + 1) * (kFM + 2);    // x-faces of a plane (i 0..n, j -1..n); as many y-faces
constexpr int kFXY = 2 * kFXF;
constexpr int kFG = kFM * kFM;                 // interior cells of a plane
constexpr int kFEd = (kFM + 1) * (kFM + 1);    // corner EMFs of a plane

// shared-memory layout, in floats
constexpr int oW = 0;                          // [6][7][kFPA]   rho, u~^x, u~^y, u~^z, p, calB^x, calB^y
constexpr int oBz = oW + 6 * 7 * kFPA;         // [2][kFPA]      calB^z
constexpr int oM = oBz + 2 * kFPA;             // [3][10][kFVA]  alpha, beta^i, gamma_ij on vertices
constexpr int oE = oM + 3 * 10 * kFVA;         // [3][3][kFEA]   cell electric field E_x, E_y, E_z
constexpr int oG = oE + 3 * 3 * kFEA;          // [2][7][kFG]    cell gamma_ij and sqrt(gamma)
constexpr int oFxy = oG + 2 * 7 * kFG;         // [2][7][kFXY]   x-face then y-face fluxes
constexpr int oFz = oFxy + 2 * 7 * kFXY;       // [3][7][kFEA]   z-face fluxes
constexpr int oEz = oFz + 3 * 7 * kFEA;        // [2][kFEd]      corner EMFs
constexpr int oEx = oEz + 2 * kFEd;
constexpr int oEy = oEx + 2 * kFEd;
constexpr int kFFloats = oEy + 2 * kFEd;
constexpr size_t kFSmem = sizeof(float) * kFFloats;
static_assert(kFSmem <= 227 * 1024, "fused sweep: shared memory above the per-CTA limit");

__device__ __forceinline__ int fring(int p, int r) {
  const int m = p % r;
  return m < 0 ? m + r : m;
}
__device__ __forceinline__ int wix(int x, int y) { return (y + 3) * kFP + (x + 3); }
__device__ __forceinline__ int mix_(int x, int y) { return (y + 1) * kFVS + (x + 1); }
__device__ __forceinline__ int eix(int x, int y) { return (y + 1) * kFES + (x + 1); }
__device__ __forceinline__ int xfix(int i, int j) { return (j + 1) * (kFM + 1) + i; }
__device__ __forceinline__ int yfix(int i, int j) { return kFXF + j * (kFM + 2) + (i + 1); }
__device__ __forceinline__ int edix(int i, int j) { return j * (kFM + 1) + i; }

__device__ __forceinline__ void fcopy4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void fcopy16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void fcommit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void fwait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// A cell plane (all N0 x N1 cells of padded plane index p + g) of one pool into a kFP-strided smem plane:
// 16-byte copies when a padded row is exactly kFP cells and the plane is 16-byte aligned, else 4-byte.
__device__ __forceinline__ void load_cell_plane(float* dst, const float* pool, const DBlock& b, long long off, int p) {
  const int N0 = b.N[0], N1 = b.N[1];
  const float* src = pool + off + (long long)(p + b.g) * N0 * N1;
  if (N0 == kFP && ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) && ((N0 * N1) & 3) == 0) {
    for (int q = threadIdx.x; q < (N0 * N1) / 4; q += kFT) fcopy16(dst + 4 * q, src + 4 * q);
  } else {
    for (int q = threadIdx.x; q < N0 * N1; q += kFT) {
      const int y = q / N0, x = q - y * N0;
      fcopy4(dst + y * kFP + x, src + q);
    }
  }
}

// Vertex plane v (vertices -1 .. n + 1 in x and y) of the 10 metric components
__device__ __forceinline__ void load_metric_plane(float* dst, const InView<float>& in, const DBlock& b, int v) {
  const int W0 = b.N[0] + 1, W1 = b.N[1] + 1;
  const int nx = b.n[0] + 3, ny = b.n[1] + 3;
  const long long base = b.vert + (long long)(v + b.g) * W0 * W1;
  for (int q = threadIdx.x; q < 10 * nx * ny; q += kFT) {
    const int c = q / (nx * ny), r = q - c * nx * ny;
    const int y = r / nx, x = r - y * nx;   // vertex (x - 1, y - 1)
    fcopy4(dst + c * kFVA + y * kFVS + x, in.M[c] + base + (long long)(y - 1 + b.g) * W0 + (x - 1 + b.g));
  }
}

// Cell plane p of the cell electric field (cells -1 .. n in x and y), the three components
__device__ __forceinline__ void load_efield_plane(float* dst, const Workspace& ws, const DBlock& b, int p) {
  const int N0 = b.N[0], N1 = b.N[1];
  const int nx = b.n[0] + 2, ny = b.n[1] + 2;
  const long long base = b.wcell + (long long)(p + b.g) * N0 * N1;
  for (int q = threadIdx.x; q < 3 * nx * ny; q += kFT) {
    const int c = q / (nx * ny), r = q - c * nx * ny;
    const int y = r / nx, x = r - y * nx;   // cell (x - 1, y - 1)
    fcopy4(dst + c * kFEA + y * kFES + x,
           reinterpret_cast<const float*>(ws.ecc[c]) + base + (long long)(y - 1 + b.g) * N0 + (x - 1 + b.g));
  }
}

// One face of direction D: x- and y-faces at (i, j) of cell plane p, z-faces at (i, j) of vertex plane p.
// The arithmetic of face_body (faces_impl.cuh) on the stencil and metric held in shared memory.
template <int EOS, int METHOD, int D>
__device__ __forceinline__ void fused_face(const float* sm, const DBlock& b, const InView<float>& in, const KParams& kp,
                                           int i, int j, int p, float* out, int ostride) {
  constexpr int NV = 7;
  float st[NV][6];
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const float* wp;
    int c;
    const float* bz = sm + oBz + fring(p, 2) * kFPA;
    if constexpr (D == 0) { wp = sm + oW + fring(p, 6) * 7 * kFPA; c = wix(i - 3 + t, j); }
    else if constexpr (D == 1) { wp = sm + oW + fring(p, 6) * 7 * kFPA; c = wix(i, j - 3 + t); }
    else { wp = sm + oW + fring(p - 3 + t, 6) * 7 * kFPA; c = wix(i, j); }
#pragma unroll
    for (int v = 0; v < 5; ++v) st[v][t] = wp[v * kFPA + c];
    if constexpr (D == 0) { st[5][t] = wp[6 * kFPA + c]; st[6][t] = bz[c]; }
    else if constexpr (D == 1) { st[5][t] = bz[c]; st[6][t] = wp[5 * kFPA + c]; }
    else { st[5][t] = wp[5 * kFPA + c]; st[6][t] = wp[6 * kFPA + c]; }
  }
  float L[NV], Rr[NV];
  face_recon<float, EOS, METHOD>(st, kp, L, Rr);
  // face metric: the mean of the face's four vertices in face_metric's order
  float met[10];
  {
    int a0, a1, a2, a3;   // vertex indices of (0, s1, s2, s1 + s2)
    const float* m0;
    const float* m1;
    if constexpr (D == 0) {   // t1 = y, t2 = z
      m0 = sm + oM + fring(p, 3) * 10 * kFVA; m1 = sm + oM + fring(p + 1, 3) * 10 * kFVA;
      a0 = mix_(i, j); a1 = mix_(i, j + 1); a2 = a0; a3 = a1;
    } else if constexpr (D == 1) {   // t1 = z, t2 = x
      m0 = sm + oM + fring(p, 3) * 10 * kFVA; m1 = sm + oM + fring(p + 1, 3) * 10 * kFVA;
      a0 = mix_(i, j); a1 = a0; a2 = mix_(i + 1, j); a3 = a2;
    } else {   // t1 = x, t2 = y, one vertex plane
      m0 = sm + oM + fring(p, 3) * 10 * kFVA; m1 = m0;
      a0 = mix_(i, j); a1 = mix_(i + 1, j); a2 = mix_(i, j + 1); a3 = mix_(i + 1, j + 1);
    }
#pragma unroll
    for (int c = 0; c < 10; ++c) {
      float f0, f1, f2, f3;
      if constexpr (D == 0) { f0 = m0[c * kFVA + a0]; f1 = m0[c * kFVA + a1]; f2 = m1[c * kFVA + a2]; f3 = m1[c * kFVA + a3]; }
      else if constexpr (D == 1) { f0 = m0[c * kFVA + a0]; f1 = m1[c * kFVA + a1]; f2 = m0[c * kFVA + a2]; f3 = m1[c * kFVA + a3]; }
      else { f0 = m0[c * kFVA + a0]; f1 = m0[c * kFVA + a1]; f2 = m0[c * kFVA + a2]; f3 = m0[c * kFVA + a3]; }
      met[c] = 0.25f * ((f0 + f1) + (f2 + f3));
    }
  }
  const float Bn = in.B[D][b.face[D] + fix(b, D, i, j, p)];
  float F[7], ye_up;
  face_flux<float, EOS, D>(L, Rr, met, Bn, kp, F, &ye_up);
#pragma unroll
  for (int v = 0; v < 7; ++v) out[v * ostride] = F[v];
}

// upwind selection of edge_body
__device__ __forceinline__ float fupw(float vel, float lowside, float highside) {
  return vel > 0.f ? lowside : (vel < 0.f ? highside : 0.5f * (lowside + highside));
}

// Corner EMF from its four faces (a-faces at b-cells ib-1, ib; b-faces at a-cells ia-1, ia) and four cells,
// in edge_body's order: F = (mass flux, F_5, F_6) of each face, C = cell E_m
__device__ __forceinline__ float fused_edge(const float* Fa1, const float* Fa0, const float* Fb1, const float* Fb0,
                                            int sa, int sb, float C11, float C01, float C10, float C00, int emf) {
  const float Ea1 = -Fa1[5 * sa], Ea0 = -Fa0[5 * sa];
  const float Eb1 = Fb1[6 * sb], Eb0 = Fb0[6 * sb];
  float E = 0.25f * (Ea1 + Ea0 + Eb1 + Eb0);
  if (emf == GR_EMF_UPWIND) {
    const float va1 = Fa1[0], va0 = Fa0[0], vb1 = Fb1[0], vb0 = Fb0[0];
    const float db_hi = fupw(va1, C01 - Eb0, C11 - Eb1);
    const float db_lo = fupw(va0, Eb0 - C00, Eb1 - C10);
    const float da_hi = fupw(vb1, C10 - Ea0, C11 - Ea1);
    const float da_lo = fupw(vb0, Ea0 - C00, Ea1 - C01);
    E += 0.25f * (db_lo - db_hi) + 0.25f * (da_lo - da_hi);
  }
  return E;
}

// CT of one face (ct_body's operations): curl = idx1 dE2 - idx2 dE1, B' = g1 B - beta dt curl (+ g0 B0)
__device__ __forceinline__ void fused_ct(const StateView& s, const KParams& kp, int D, long long f, double idx1,
                                         double idx2, float E2hi, float E2lo, float E1hi, float E1lo) {
  const double dE2 = diff64(E2hi, E2lo);
  const double dE1 = diff64(E1hi, E1lo);
  const double curl = fma(idx1, dE2, -(idx2 * dE1));
  const double B = s.B[D][f];
  double Bn = fma(-stage_bdt(kp), curl, (kp.rk_form & RK_G1) ? kp.rk_g1 * B : B);
  if (kp.rk_form & RK_G0) Bn = fma(kp.rk_g0, s.B0[D][f], Bn);
  s.Bo[D][f] = Bn;
  if (s.Bo32[D]) s.Bo32[D][f] = d2f_rn(Bn);
}

template <int EOS, int METHOD>
__global__ void __launch_bounds__(kFT, 1) k_fused(const DBlock* __restrict__ blocks,
                                                  const __grid_constant__ InView<float> in,
                                                  const __grid_constant__ StateView s,
                                                  const __grid_constant__ Workspace ws,
                                                  const __grid_constant__ KParams kp) {
  extern __shared__ __align__(16) float sm[];
  const DBlock b = blocks[blockIdx.x];
  const int n0 = b.n[0], n1 = b.n[1], n2 = b.n[2];
  const int tid = threadIdx.x;
  auto load_w = [&](int p) {   // W plane p: the 7 ring variables, into slot fring(p, 6)
    float* d = sm + oW + fring(p, 6) * 7 * kFPA;
#pragma unroll 1
    for (int v = 0; v < 5; ++v) load_cell_plane(d + v * kFPA, in.W[v], b, b.cell, p);
    load_cell_plane(d + 5 * kFPA, reinterpret_cast<const float*>(ws.bcc[0]), b, b.wcell, p);
    load_cell_plane(d + 6 * kFPA, reinterpret_cast<const float*>(ws.bcc[1]), b, b.wcell, p);
  };
  auto load_bz = [&](int p) {
    load_cell_plane(sm + oBz + fring(p, 2) * kFPA, reinterpret_cast<const float*>(ws.bcc[2]), b, b.wcell, p);
  };
  // prologue: the planes of step 0
  for (int p = -3; p <= 2; ++p) load_w(p);
  load_bz(-1);
  load_metric_plane(sm + oM + fring(-1, 3) * 10 * kFVA, in, b, -1);
  load_metric_plane(sm + oM + fring(0, 3) * 10 * kFVA, in, b, 0);
  load_efield_plane(sm + oE + fring(-1, 3) * 3 * kFEA, ws, b, -1);
  fcommit();
  const unsigned lane = tid & 31u;
  for (int t = 0; t <= n2 + 1; ++t) {
    fwait_all();
    __syncthreads();
    // ---- faces: x, y of cell plane t - 1; z of vertex plane t --------------------------------------
    {
      const int pf = t - 1;
      const int nx = (n0 + 1) * (n1 + 2), ny = (n0 + 2) * (n1 + 1), nz = t <= n2 ? (n0 + 2) * (n1 + 2) : 0;
      const int ax = (nx + 31) & ~31, ay = (ny + 31) & ~31;
      float* fxy = sm + oFxy + fring(pf, 2) * 7 * kFXY;
      float* fz = sm + oFz + fring(t, 3) * 7 * kFEA;
      for (int q = tid; q < ax + ay + nz; q += kFT) {
        if (q < ax) {
          if (q < nx) {
            const int i = q % (n0 + 1), j = q / (n0 + 1) - 1;
            fused_face<EOS, METHOD, 0>(sm, b, in, kp, i, j, pf, fxy + xfix(i, j), kFXY);
          }
        } else if (q < ax + ay) {
          const int e = q - ax;
          if (e < ny) {
            const int i = e % (n0 + 2) - 1, j = e / (n0 + 2);
            fused_face<EOS, METHOD, 1>(sm, b, in, kp, i, j, pf, fxy + yfix(i, j), kFXY);
          }
        } else {
          const int e = q - ax - ay;
          const int i = e % (n0 + 2) - 1, j = e / (n0 + 2) - 1;
          fused_face<EOS, METHOD, 2>(sm, b, in, kp, i, j, t, fz + eix(i, j), kFEA);
        }
      }
    }
    __syncthreads();
    // ---- prefetch of the planes step t + 1 adds (slots read no more in this step) ------------------
    if (t + 3 <= n2 + 2) load_w(t + 3);
    if (t <= n2) load_bz(t);
    if (t + 1 <= n2 + 1) load_metric_plane(sm + oM + fring(t + 1, 3) * 10 * kFVA, in, b, t + 1);
    if (t <= n2) load_efield_plane(sm + oE + fring(t, 3) * 3 * kFEA, ws, b, t);
    fcommit();
    // ---- edges on vertex plane t - 1, E_z and the cell metric of cell plane t - 1 --------------------
    if (t >= 1) {
      const int ve = t - 1;
      const bool inner = ve <= n2 - 1;   // cell plane ve is interior
      const int cx = n0 * (n1 + 1), cy = (n0 + 1) * n1, cz = inner ? (n0 + 1) * (n1 + 1) : 0;
      const int cg = inner ? n0 * n1 : 0;
      const float* fxy1 = sm + oFxy + fring(ve, 2) * 7 * kFXY;       // x, y faces of cell plane ve
      const float* fxy0 = sm + oFxy + fring(ve - 1, 2) * 7 * kFXY;   // ... of cell plane ve - 1
      const float* fzv = sm + oFz + fring(ve, 3) * 7 * kFEA;         // z faces of vertex plane ve
      const float* e1 = sm + oE + fring(ve, 3) * 3 * kFEA;           // cell E of planes ve, ve - 1
      const float* e0 = sm + oE + fring(ve - 1, 3) * 3 * kFEA;
      for (int q = tid; q < cx + cy + cz + cg; q += kFT) {
        if (q < cx) {   // E_x at (i, j, ve): a = y-faces (planes ve, ve - 1), b = z-faces (j, j - 1)
          const int i = q % n0, j = q / n0;
          const float E = fused_edge(fxy1 + yfix(i, j), fxy0 + yfix(i, j), fzv + eix(i, j), fzv + eix(i, j - 1), kFXY,
                                     kFEA, e1[0 * kFEA + eix(i, j)], e1[0 * kFEA + eix(i, j - 1)],
                                     e0[0 * kFEA + eix(i, j)], e0[0 * kFEA + eix(i, j - 1)], kp.emf);
          sm[oEx + fring(ve, 2) * kFEd + edix(i, j)] = E;
        } else if (q < cx + cy) {   // E_y at (i, j, ve): a = z-faces (i, i - 1), b = x-faces (planes ve, ve - 1)
          const int e = q - cx;
          const int i = e % (n0 + 1), j = e / (n0 + 1);
          const float E = fused_edge(fzv + eix(i, j), fzv + eix(i - 1, j), fxy1 + xfix(i, j), fxy0 + xfix(i, j), kFEA,
                                     kFXY, e1[1 * kFEA + eix(i, j)], e0[1 * kFEA + eix(i, j)],
                                     e1[1 * kFEA + eix(i - 1, j)], e0[1 * kFEA + eix(i - 1, j)], kp.emf);
          sm[oEy + fring(ve, 2) * kFEd + edix(i, j)] = E;
        } else if (q < cx + cy + cz) {   // E_z at (i, j) of cell plane ve: a = x-faces (j, j - 1), b = y-faces (i, i - 1)
          const int e = q - cx - cy;
          const int i = e % (n0 + 1), j = e / (n0 + 1);
          const float E = fused_edge(fxy1 + xfix(i, j), fxy1 + xfix(i, j - 1), fxy1 + yfix(i, j), fxy1 + yfix(i - 1, j),
                                     kFXY, kFXY, e1[2 * kFEA + eix(i, j)], e1[2 * kFEA + eix(i - 1, j)],
                                     e1[2 * kFEA + eix(i, j - 1)], e1[2 * kFEA + eix(i - 1, j - 1)], kp.emf);
          sm[oEz + fring(ve, 2) * kFEd + edix(i, j)] = E;
        } else {   // cell metric of (i, j, ve): the eight vertices summed in cell_metric's order
          const int e = q - cx - cy - cz;
          const int i = e % n0, j = e / n0;
          const float* m0 = sm + oM + fring(ve, 3) * 10 * kFVA;
          const float* m1 = sm + oM + fring(ve + 1, 3) * 10 * kFVA;
          float gam[6];
#pragma unroll
          for (int c = 4; c < 10; ++c) {
            const float* a0 = m0 + c * kFVA;
            const float* a1 = m1 + c * kFVA;
            const float f0 = a0[mix_(i, j)], f1 = a0[mix_(i + 1, j)], f2 = a0[mix_(i, j + 1)], f3 = a0[mix_(i + 1, j + 1)];
            const float f4 = a1[mix_(i, j)], f5 = a1[mix_(i + 1, j)], f6 = a1[mix_(i, j + 1)], f7 = a1[mix_(i + 1, j + 1)];
            gam[c - 4] = 0.125f * (((f0 + f1) + (f2 + f3)) + ((f4 + f5) + (f6 + f7)));
          }
          float* g = sm + oG + fring(ve, 2) * 7 * kFG + j * kFM + i;
#pragma unroll
          for (int c = 0; c < 6; ++c) g[c * kFG] = gam[c];
          g[6 * kFG] = sqrt_r(det3(gam));
        }
      }
    }
    __syncthreads();
    // ---- CT: x-, y-faces of cell plane t - 2, z-faces of vertex plane t - 1 ---------------------------
    {
      const int pc = t - 2, vc = t - 1;
      const bool cells = pc >= 0 && pc <= n2 - 1;
      const int cx = cells ? (n0 + 1) * n1 : 0, cy = cells ? n0 * (n1 + 1) : 0;
      const int cz = (vc >= 0 && vc <= n2) ? n0 * n1 : 0;
      for (int q = tid; q < cx + cy + cz; q += kFT) {
        if (q < cx) {   // x-face (i, j, pc): dE_z along y, dE_y along z
          const int i = q % (n0 + 1), j = q / (n0 + 1);
          const float* ez = sm + oEz + fring(pc, 2) * kFEd;
          fused_ct(s, kp, 0, b.face[0] + fix(b, 0, i, j, pc), b.idx[1], b.idx[2], ez[edix(i, j + 1)], ez[edix(i, j)],
                   sm[oEy + fring(pc + 1, 2) * kFEd + edix(i, j)], sm[oEy + fring(pc, 2) * kFEd + edix(i, j)]);
        } else if (q < cx + cy) {   // y-face (i, j, pc): dE_x along z, dE_z along x
          const int e = q - cx;
          const int i = e % n0, j = e / n0;
          const float* ez = sm + oEz + fring(pc, 2) * kFEd;
          fused_ct(s, kp, 1, b.face[1] + fix(b, 1, i, j, pc), b.idx[2], b.idx[0],
                   sm[oEx + fring(pc + 1, 2) * kFEd + edix(i, j)], sm[oEx + fring(pc, 2) * kFEd + edix(i, j)],
                   ez[edix(i + 1, j)], ez[edix(i, j)]);
        } else {   // z-face (i, j, vc): dE_y along x, dE_x along y
          const int e = q - cx - cy;
          const int i = e % n0, j = e / n0;
          const float* ey = sm + oEy + fring(vc, 2) * kFEd;
          const float* ex = sm + oEx + fring(vc, 2) * kFEd;
          fused_ct(s, kp, 2, b.face[2] + fix(b, 2, i, j, vc), b.idx[0], b.idx[1], ey[edix(i + 1, j)], ey[edix(i, j)],
                   ex[edix(i, j + 1)], ex[edix(i, j)]);
        }
      }
    }
    __syncthreads();
    // ---- update of cell plane t - 2 -----------------------------------------------------------------
    {
      const int pu = t - 2;
      const int cu = (pu >= 0 && pu <= n2 - 1) ? n0 * n1 : 0;
      const float* fxy = sm + oFxy + fring(pu, 2) * 7 * kFXY;
      const float* fz0 = sm + oFz + fring(pu, 3) * 7 * kFEA;
      const float* fz1 = sm + oFz + fring(pu + 1, 3) * 7 * kFEA;
      for (int q0 = 0; q0 < cu; q0 += kFT) {   // uniform trip count: the job append is warp-collective
        const int q = q0 + tid;
        bool queued = false;
        int i = 0, j = 0;
        if (q < cu) {
          i = q % n0;
          j = q / n0;
          const long long c = b.cell + cix(b, i, j, pu);
          const int x0 = xfix(i, j), x1 = xfix(i + 1, j), y0 = yfix(i, j), y1 = yfix(i, j + 1), z = eix(i, j);
          const double d0 = accumulate_vals<float>(b, s, kp, c, 0, 0.f, fxy[x0], fxy[x1], fxy[y0], fxy[y1], fz0[z], fz1[z]);
          const float* g = sm + oG + fring(pu, 2) * 7 * kFG + j * kFM + i;
          float gam[6];
#pragma unroll
          for (int cc = 0; cc < 6; ++cc) gam[cc] = g[cc * kFG];
          const float sg = g[6 * kFG];
          if (isfinite(d0) && d0 < kp.rho_thr * to64(sg)) {
            bool finite = true;
#pragma unroll
            for (int v = 1; v < 5; ++v) {
              const int o = v * kFXY, oz = v * kFEA;
              const float tt = fxy[o + x1] - fxy[o + x0] + fxy[o + y1] - fxy[o + y0] + fz1[oz + z] - fz0[oz + z];
              finite = finite && isfinite(tt) && isfinite(s.U[v][c]);
            }
            mixed_atm_reset<float, EOS>(b, s, kp, i, j, pu, c, gam, sg, finite);
          } else {
            float src[6];
            CellMet<float> M;
            cell_sources_at<float, EOS>(b, in, kp, i, j, pu, c, src, M);
#pragma unroll
            for (int v = 0; v < 5; ++v) {
              const int o = v * kFXY, oz = v * kFEA;
              s.Uo[v][c] = accumulate_vals<float>(b, s, kp, c, v, src[v], fxy[o + x0], fxy[o + x1], fxy[o + y0],
                                                  fxy[o + y1], fz0[oz + z], fz1[oz + z]);
            }
            queued = true;
          }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, queued);
        int base = 0;
        if (lane == 0 && mask) base = atomicAdd(ws.njobs, __popc(mask));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (queued) ws.jobs[base + __popc(mask & ((1u << lane) - 1u))] = make_int2(blockIdx.x, (pu * n1 + j) * n0 + i);
      }
    }
  }
  fwait_all();
}

template <int METHOD>
static cudaError_t launch_fused_m(const DBlock* blocks, int nblocks, const InView<float>& in, const StateView& s,
                                  const Workspace& ws, const KParams& kp, cudaStream_t st) {
  // above the default 48 KB: the opt-in is per device (set once on each, one bit per device)
  static unsigned long long attr = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev < 64 && !((attr >> dev) & 1ull)) {
    const cudaError_t e = cudaFuncSetAttribute(k_fused<GR_EOS_IDEAL, METHOD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kFSmem);
    if (e != cudaSuccess) return e;
    attr |= 1ull << dev;
  }
  k_fused<GR_EOS_IDEAL, METHOD><<<nblocks, kFT, kFSmem, st>>>(blocks, in, s, ws, kp);
  return cudaGetLastError();
}

cudaError_t launch_fused(const DBlock* blocks, int nblocks, const InView<float>& in, const StateView& s,
                         const Workspace& ws, const KParams& kp, cudaStream_t st) {
  switch (kp.recon) {
    case GR_RECON_PLM: return launch_fused_m<GR_RECON_PLM>(blocks, nblocks, in, s, ws, kp, st);
    case GR_RECON_WENO5: return launch_fused_m<GR_RECON_WENO5>(blocks, nblocks, in, s, ws, kp, st);
    case GR_RECON_PPM: return launch_fused_m<GR_RECON_PPM>(blocks, nblocks, in, s, ws, kp, st);
    default: return launch_fused_m<GR_RECON_WENOZ>(blocks, nblocks, in, s, ws, kp, st);
  }
}

bool fused_block_ok(const DBlock& b) { return b.g == 3 && b.n[0] <= kFM && b.n[1] <= kFM; }

}  // namespace grs
