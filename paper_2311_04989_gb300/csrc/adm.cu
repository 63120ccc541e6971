// adm.cu -- matter sources of the spacetime equations at the vertices: rho_ADM, S_i, S_ij (the hydro
// forms of Sec. 2.1 and the MHD forms of Sec. 2.2), carried from the cell centres to the vertex grid
// of the spacetime solver by Lagrange interpolation (Sec. 3.2).
//
//   k_adm_cells   per cell of the ring the interpolation reads (-r .. n+r-1 per axis, r = order/2):
//                 gamma_ij at the cell centre (the metric's vertex-to-cell interpolant), cell field
//                 (mean of the two densitised faces) and primitives -> the ten sources, written in
//                 the cell layout of the caller's pools to a workspace
//   k_adm_verts   per (block, slab of vertex planes) and component: the slab's cells staged in shared
//                 memory, then the tensor-product interpolant applied one axis at a time (x, y, z),
//                 so an order-4 vertex costs 12 FMAs per component instead of 64; writes the owned
//                 vertices 0..n of the caller's vertex pools
// Arithmetic type R: double (GR_PREC_FP64), or float (GR_PREC_MIXED: FP64 inputs rounded on load,
// FP32 arithmetic and workspace, FP64 output).  The FP64 pipe of this GPU runs ~1/64 of the FP32
// rate, and both kernels are FP64-pipe bound in double.
#include "internal.h"
#include "physics.cuh"
#include "stage_common.cuh"

namespace grs {

struct AdmCellArgs {
  const double* W[6];   // rho, u~^i, p[, Y_e]
  const double* B[3];
  const double* g[6];   // gamma_ij at the vertices (xx, xy, xz, yy, yz, zz)
  void* cv[10];         // workspace, cell layout, element type R
  double gfac;          // Gamma / (Gamma - 1) (ideal gas)
  int r;                // cell ring of the interpolation
  int morder;           // vertex-to-cell order of the metric
};

template <class R> __device__ __forceinline__ R cvt(double x);
template <> __device__ __forceinline__ double cvt<double>(double x) { return x; }
template <> __device__ __forceinline__ float cvt<float>(double x) { return d2f_rn(x); }
template <class R> __device__ __forceinline__ R rrsqrt(R x);
template <> __device__ __forceinline__ double rrsqrt<double>(double x) { return rsqrt(x); }
template <> __device__ __forceinline__ float rrsqrt<float>(float x) { return rsqrtf(x); }

// Coordinates of t, t + S, t + 2S, ... in a row-major (W, H, *) box without a division per step
// (an integer division by a run-time divisor costs FP64-pipe conversions on this GPU): t and S are
// decomposed once, and each step carries at most one unit into the next coordinate.
struct Walk3 {
  int x, y, z, sx, sy, sz, W, H;
  __device__ __forceinline__ Walk3(int t, int S, int W_, int H_) : W(W_), H(H_) {
    int q = t / W;
    x = t - q * W;
    y = q % H;
    z = q / H;
    q = S / W;
    sx = S - q * W;
    sy = q % H;
    sz = q / H;
  }
  __device__ __forceinline__ void step() {
    x += sx;
    int c = 0;
    if (x >= W) { x -= W; c = 1; }
    y += sy + c;
    c = 0;
    if (y >= H) { y -= H; c = 1; }
    z += sz + c;
  }
};

// gamma_ij at the centre of cell (i, j, k): the metric's vertex-to-cell Lagrange interpolant (2 or
// 4 vertices per axis, midpoint weights 1/2 or (-1, 9, 9, -1)/16)
template <class R>
__device__ __forceinline__ void adm_gamma(const DBlock& b, const AdmCellArgs& a, int i, int j, int k, R g[6]) {
  if (a.morder == 2) {
    long long v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = b.vert + vix(b, i + (t & 1), j + ((t >> 1) & 1), k + (t >> 2));
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      R f[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) f[t] = cvt<R>(__ldg(a.g[c] + v[t]));
      g[c] = R(0.125) * (((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])));
    }
  } else {
    const R w[4] = {R(-1.0 / 16), R(9.0 / 16), R(9.0 / 16), R(-1.0 / 16)};
    for (int c = 0; c < 6; ++c) {
      R s = 0;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const double* row = a.g[c] + b.vert + vix(b, i - 1, j - 1 + jj, k - 1 + kk);
          const R x = w[0] * cvt<R>(__ldg(row)) + w[1] * cvt<R>(__ldg(row + 1)) + w[2] * cvt<R>(__ldg(row + 2)) +
                      w[3] * cvt<R>(__ldg(row + 3));
          s += (w[jj] * w[kk]) * x;
        }
      g[c] = s;
    }
  }
}

// The ten sources at the centre of cell (i, j, k), in the order rho_ADM, S_i, S_ij (xx xy xz yy yz zz).
// Lapse and shift do not enter: alpha b^0 = W calB^i v_i, and the projections carry no alpha, beta.
template <class R, int EOS>
__device__ __forceinline__ void adm_cell(const DBlock& b, const AdmCellArgs& a, const KParams& kp, int i, int j,
                                         int k, R out[10]) {
  R g[6];
  adm_gamma<R>(b, a, i, j, k, g);
  const R isg = rrsqrt<R>(det3(g));             // 1 / sqrt(gamma)
  const long long c = b.cell + cix(b, i, j, k);
  const R rho = cvt<R>(a.W[0][c]), p = cvt<R>(a.W[4][c]);
  const R ut[3] = {cvt<R>(a.W[1][c]), cvt<R>(a.W[2][c]), cvt<R>(a.W[3][c])};
  R utl[3];
  lower3(g, ut, utl);
  const R x = R(1) + (ut[0] * utl[0] + ut[1] * utl[1] + ut[2] * utl[2]);   // W^2
  const R iW = rrsqrt<R>(x), W = x * iW;
  R vl[3], Bu[3], Bl[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) vl[t] = utl[t] * iW;
  {
    const long long f0 = b.face[0] + fix(b, 0, i, j, k), f1 = b.face[1] + fix(b, 1, i, j, k);
    const long long f2 = b.face[2] + fix(b, 2, i, j, k);
    const R h = R(0.5) * isg;
    Bu[0] = (cvt<R>(a.B[0][f0]) + cvt<R>(a.B[0][f0 + 1])) * h;
    Bu[1] = (cvt<R>(a.B[1][f1]) + cvt<R>(a.B[1][f1 + b.N[0]])) * h;
    Bu[2] = (cvt<R>(a.B[2][f2]) + cvt<R>(a.B[2][f2 + (long long)b.N[0] * b.N[1]])) * h;
  }
  lower3(g, Bu, Bl);
  const R Bv = Bu[0] * vl[0] + Bu[1] * vl[1] + Bu[2] * vl[2];
  const R BB = Bu[0] * Bl[0] + Bu[1] * Bl[1] + Bu[2] * Bl[2];
  const R ab0 = W * Bv;
  const R b2 = (ab0 * ab0 + BB) * (iW * iW);
  R bl[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) bl[t] = Bl[t] * iW + ab0 * vl[t];
  R rhoh;
  if constexpr (EOS == GR_EOS_IDEAL) {
    rhoh = rho + R(a.gfac) * p;
  } else {
    R cs2;
    eos_rhoh_cs2<R, EOS>(kp, rho, p, cvt<R>(a.W[5][c]), &rhoh, &cs2);
  }
  const R pt = p + R(0.5) * b2;
  const R eW2 = (rhoh + b2) * x;
  out[0] = eW2 - pt - ab0 * ab0;
#pragma unroll
  for (int t = 0; t < 3; ++t) out[1 + t] = eW2 * vl[t] - ab0 * bl[t];
  const int I[6] = {0, 0, 0, 1, 1, 2}, J[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int t = 0; t < 6; ++t) out[4 + t] = eW2 * vl[I[t]] * vl[J[t]] + pt * g[t] - bl[I[t]] * bl[J[t]];
}

// Work: block, start = cell plane k (-r .. n_z + r - 1); the CTA's threads walk the plane's cells.
template <class R, int EOS>
__global__ void __launch_bounds__(kTile) k_adm_cells(const DBlock* __restrict__ blocks, const Work* __restrict__ work,
                                                     const __grid_constant__ KParams kp,
                                                     const __grid_constant__ AdmCellArgs a) {
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  const int r = a.r;
  const int C0 = b.n[0] + 2 * r, C1 = b.n[1] + 2 * r;
  const int k = w.start;
  Walk3 it((int)threadIdx.x, kTile, C0, C1);
  for (; it.z == 0; it.step()) {
    const int i = it.x - r, j = it.y - r;
    R out[10];
    adm_cell<R, EOS>(b, a, kp, i, j, k, out);
    const long long c = b.cell + cix(b, i, j, k);
#pragma unroll
    for (int t = 0; t < 10; ++t) static_cast<R*>(a.cv[t])[c] = out[t];
  }
}

struct AdmVertArgs {
  const void* cv[10];
  double* out[10];
};

// midpoint weights of the 2- and 4-point Lagrange interpolants
template <class R, int NP> __device__ __forceinline__ R mid_weight(int s);
template <> __device__ __forceinline__ double mid_weight<double, 2>(int) { return 0.5; }
template <> __device__ __forceinline__ float mid_weight<float, 2>(int) { return 0.5f; }
template <> __device__ __forceinline__ double mid_weight<double, 4>(int s) {
  return (s == 1 || s == 2) ? 9.0 / 16 : -1.0 / 16;
}
template <> __device__ __forceinline__ float mid_weight<float, 4>(int s) {
  return (s == 1 || s == 2) ? 9.0f / 16 : -1.0f / 16;
}

// Work: block, dir = number of vertex planes Z of the slab, start = first vertex plane z0.
// Vertex v along an axis lies between cells v-1 and v; its NP-point stencil is cells v-r .. v+r-1,
// i.e. entries v .. v+NP-1 of a cell row that starts at cell -r.
template <class R, int NP>
__global__ void __launch_bounds__(kAdmThreads) k_adm_verts(const DBlock* __restrict__ blocks,
                                                           const Work* __restrict__ work,
                                                           const __grid_constant__ AdmVertArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* smem = reinterpret_cast<R*>(smem_raw);
  constexpr int r = NP / 2;
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  const R* __restrict__ cv = static_cast<const R*>(a.cv[blockIdx.y]);
  const int C0 = b.n[0] + 2 * r, C1 = b.n[1] + 2 * r;
  const int V0 = b.n[0] + 1, V1 = b.n[1] + 1;
  const int Z = w.dir, z0 = w.start, CZ = Z + NP - 1;
  R* A = smem;                          // cells (C0, C1, CZ); later the y pass (V0, V1, CZ)
  R* X = smem + (size_t)C0 * C1 * CZ;   // x pass (V0, C1, CZ)
  // asynchronous copies straight into shared memory: each thread issues all of its loads at once
  // instead of waiting for each before the next
  const int ncells = C0 * C1 * CZ;
  Walk3 wc((int)threadIdx.x, kAdmThreads, C0, C1);
  for (int t = threadIdx.x; t < ncells; t += kAdmThreads, wc.step()) {
    const R* src = cv + b.cell + cix(b, wc.x - r, wc.y - r, z0 - r + wc.z);
    const unsigned dst = (unsigned)__cvta_generic_to_shared(A + t);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(dst), "l"(src), "n"(sizeof(R)) : "memory");
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  const int nx = V0 * C1 * CZ;
  Walk3 wx((int)threadIdx.x, kAdmThreads, V0, C1);
  for (int t = threadIdx.x; t < nx; t += kAdmThreads, wx.step()) {
    const R* src = A + ((size_t)wx.z * C1 + wx.y) * C0 + wx.x;
    R s = 0;
#pragma unroll
    for (int q = 0; q < NP; ++q) s = fma(mid_weight<R, NP>(q), src[q], s);
    X[t] = s;
  }
  __syncthreads();
  const int ny = V0 * V1 * CZ;
  Walk3 wy((int)threadIdx.x, kAdmThreads, V0, V1);
  for (int t = threadIdx.x; t < ny; t += kAdmThreads, wy.step()) {
    const R* src = X + ((size_t)wy.z * C1 + wy.y) * V0 + wy.x;
    R s = 0;
#pragma unroll
    for (int q = 0; q < NP; ++q) s = fma(mid_weight<R, NP>(q), src[(size_t)q * V0], s);
    A[t] = s;
  }
  __syncthreads();
  double* __restrict__ out = a.out[blockIdx.y];
  const int nz = V0 * V1 * Z;
  Walk3 wz((int)threadIdx.x, kAdmThreads, V0, V1);
  for (int t = threadIdx.x; t < nz; t += kAdmThreads, wz.step()) {
    const int vi = wz.x, vj = wz.y, vk = wz.z;
    const R* src = A + ((size_t)vk * V1 + vj) * V0 + vi;
    R s = 0;
#pragma unroll
    for (int q = 0; q < NP; ++q) s = fma(mid_weight<R, NP>(q), src[(size_t)q * V0 * V1], s);
    out[b.vert + vix(b, vi, vj, z0 + vk)] = to64(s);
  }
}

size_t adm_smem_bytes(const int n[3], int Z, int np, size_t elem) {
  const int r = np / 2;
  const size_t C0 = n[0] + 2 * r, C1 = n[1] + 2 * r, V0 = n[0] + 1, CZ = Z + np - 1;
  return elem * CZ * C1 * (C0 + V0);
}

template <class R, int NP>
static cudaError_t launch_verts(const DBlock* blocks, const Work* vw, int nvw, size_t smem, const AdmVertArgs& va,
                                cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_adm_verts<R, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_adm_verts<R, NP><<<dim3(nvw, 10), kAdmThreads, smem, st>>>(blocks, vw, va);
  return cudaGetLastError();
}

template <class R>
static cudaError_t launch_adm_r(const DBlock* blocks, const Work* cw, int ncw, const Work* vw, int nvw, size_t smem,
                                const MetricView& m, const double* const W[7], const double* const B[3],
                                const KParams& kp, int vc_order, void* const cv[10], double* const out[10],
                                cudaStream_t st) {
  AdmCellArgs ca;
  for (int v = 0; v < 6; ++v) ca.W[v] = W[v];
  for (int d = 0; d < 3; ++d) ca.B[d] = B[d];
  for (int c = 0; c < 6; ++c) ca.g[c] = m.v[4 + c];
  for (int c = 0; c < 10; ++c) ca.cv[c] = cv[c];
  ca.gfac = kp.gamma_ad / (kp.gamma_ad - 1.0);
  ca.r = vc_order / 2;
  ca.morder = m.order;
  if (ncw) {
    if (kp.eos == GR_EOS_TABLE) k_adm_cells<R, GR_EOS_TABLE><<<ncw, kTile, 0, st>>>(blocks, cw, kp, ca);
    else k_adm_cells<R, GR_EOS_IDEAL><<<ncw, kTile, 0, st>>>(blocks, cw, kp, ca);
  }
  AdmVertArgs va;
  for (int c = 0; c < 10; ++c) {
    va.cv[c] = cv[c];
    va.out[c] = out[c];
  }
  if (!nvw) return cudaGetLastError();
  return vc_order == 4 ? launch_verts<R, 4>(blocks, vw, nvw, smem, va, st)
                       : launch_verts<R, 2>(blocks, vw, nvw, smem, va, st);
}

cudaError_t launch_adm(int precision, const DBlock* blocks, const Work* cw, int ncw, const Work* vw, int nvw,
                       size_t smem, const MetricView& m, const double* const W[7], const double* const B[3],
                       const KParams& kp, int vc_order, void* const cv[10], double* const out[10], cudaStream_t st) {
  if (precision == GR_PREC_MIXED)
    return launch_adm_r<float>(blocks, cw, ncw, vw, nvw, smem, m, W, B, kp, vc_order, cv, out, st);
  return launch_adm_r<double>(blocks, cw, ncw, vw, nvw, smem, m, W, B, kp, vc_order, cv, out, st);
}

}  // namespace grs
