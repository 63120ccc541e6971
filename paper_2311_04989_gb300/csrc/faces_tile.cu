// faces_tile.cu -- k_faces_tile: the face fluxes of the mixed path (reconstruction, Sec. 3.4; face metric,
// Sec. 3.2; HLLE flux, Eq. fluxB_def) with the stencils and the metric staged in shared memory.
//
// One CTA per tile of at most kTY interior rows (y) of a block walks the block along z.  Shared memory
// holds a ring of six cell planes of the FP32 primitives and cell field (the tile's rows with their
// 3-cell halo: the z-faces' stencil) and two vertex planes of the metric (the face metric, the mean of a
// face's four vertices).  Step t computes the x- and y-faces of cell plane t - 1 and the z-faces of vertex
// plane t, each face once over the tiles of a block, and writes them to the flux workspace exactly as
// k_faces does (faces_core.cuh, the same operations: bitwise the same fluxes); then it prefetches
// (cp.async) the planes of step t + 1 while the other CTAs on the SM compute.  For blocks with 3 ghosts and
// at most 16 cells along x, the ideal-gas EOS and the order-2 metric.
#include "faces_core.cuh"
#include "internal.h"
#include "physics.cuh"
#include "stage_common.cuh"

namespace grs {

constexpr int kTT = 256;                  // threads per CTA (three CTAs per SM)
constexpr int kTX = 16 + 6;               // stored cells per row (cells -3 .. n + 2, n <= 16)
constexpr int kTR = kTY + 6;              // stored cell rows (tile rows with a 3-cell halo)
constexpr int kTP = kTR * kTX;            // cells of a stored plane
constexpr int kTVX = 16 + 3;              // stored vertices per row (-1 .. n + 1)
constexpr int kTVR = kTY + 3;             // stored vertex rows
constexpr int kTVP = kTVR * kTVX;
constexpr int tW = 0;                     // [6][7][kTP]  rho, u~^x, u~^y, u~^z, p, calB^x, calB^y
constexpr int tBz = tW + 6 * 7 * kTP;     // [2][kTP]     calB^z
constexpr int tM = tBz + 2 * kTP;         // [2][10][kTVP]
constexpr size_t kTSmem = sizeof(float) * (tM + 2 * 10 * kTVP);
static_assert(3 * kTSmem <= 227 * 1024, "face tiles: three CTAs per SM must fit");

__device__ __forceinline__ int tring(int p, int r) {
  const int m = p % r;
  return m < 0 ? m + r : m;
}

__device__ __forceinline__ void tcopy4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void tcopy16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// the tile's rows y = j0 - 3 .. j1 + 2 of padded cell plane p + 3 of one pool, row stride kTX in shared memory
__device__ __forceinline__ void tile_cell_plane(float* dst, const float* pool, const DBlock& b, long long off, int p,
                                                int j0, int rows) {
  const int N0 = b.N[0];
  const float* src = pool + off + (long long)(p + 3) * N0 * b.N[1] + (long long)j0 * N0;   // padded row j0
  const int cnt = rows * N0;
  if (N0 == kTX && ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) && (cnt & 3) == 0) {
    for (int q = threadIdx.x; q < cnt / 4; q += kTT) tcopy16(dst + 4 * q, src + 4 * q);
  } else {
    for (int q = threadIdx.x; q < cnt; q += kTT) {
      const int y = q / N0, x = q - y * N0;
      tcopy4(dst + y * kTX + x, src + q);
    }
  }
}

// vertices x = -1 .. n + 1, y = j0 - 1 .. j1 + 1 of vertex plane v, the 10 components
__device__ __forceinline__ void tile_metric_plane(float* dst, const InView<float>& in, const DBlock& b, int v, int j0,
                                                  int vrows) {
  const int W0 = b.N[0] + 1, W1 = b.N[1] + 1;
  const int nx = b.n[0] + 3;
  const long long base = b.vert + (long long)(v + 3) * W0 * W1;
  for (int q = threadIdx.x; q < 10 * nx * vrows; q += kTT) {
    const int c = q / (nx * vrows), r = q - c * nx * vrows;
    const int y = r / nx, x = r - y * nx;   // vertex (x - 1, j0 - 1 + y)
    tcopy4(dst + c * kTVP + y * kTVX + x, in.M[c] + base + (long long)(j0 + 2 + y) * W0 + (x + 2));
  }
}

template <int METHOD, int D>
__device__ __forceinline__ void tile_face(const float* sm, const DBlock& b, const InView<float>& in, const Workspace& ws,
                                          const KParams& kp, uint8_t* bad, int j0, int i, int j, int p) {
  float st[7][6];
  const int r = j - j0 + 3;   // stored row of cell row j
  const float* bz = sm + tBz + tring(p, 2) * kTP;
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const float* wp;
    int c;
    if constexpr (D == 0) { wp = sm + tW + tring(p, 6) * 7 * kTP; c = r * kTX + (i + t); }
    else if constexpr (D == 1) { wp = sm + tW + tring(p, 6) * 7 * kTP; c = (r - 3 + t) * kTX + (i + 3); }
    else { wp = sm + tW + tring(p - 3 + t, 6) * 7 * kTP; c = r * kTX + (i + 3); }
#pragma unroll
    for (int v = 0; v < 5; ++v) st[v][t] = wp[v * kTP + c];
    if constexpr (D == 0) { st[5][t] = wp[6 * kTP + c]; st[6][t] = bz[c]; }
    else if constexpr (D == 1) { st[5][t] = bz[c]; st[6][t] = wp[5 * kTP + c]; }
    else { st[5][t] = wp[5 * kTP + c]; st[6][t] = wp[6 * kTP + c]; }
  }
  float L[7], Rr[7];
  face_recon<float, GR_EOS_IDEAL, METHOD>(st, kp, L, Rr);
  // face metric: the mean of the face's four vertices in face_metric's order (s1 along t1, s2 along t2)
  float met[10];
  {
    const int rv = j - j0 + 1, xv = i + 1;   // stored vertex row / column of vertex (i, j)
    const float* m0 = sm + tM + tring(p, 2) * 10 * kTVP;
    const float* m1 = sm + tM + tring(p + 1, 2) * 10 * kTVP;
#pragma unroll
    for (int c = 0; c < 10; ++c) {
      const float* a = m0 + c * kTVP;
      float f0, f1, f2, f3;
      if constexpr (D == 0) {   // t1 = y, t2 = z
        const float* a1 = m1 + c * kTVP;
        f0 = a[rv * kTVX + xv]; f1 = a[(rv + 1) * kTVX + xv]; f2 = a1[rv * kTVX + xv]; f3 = a1[(rv + 1) * kTVX + xv];
      } else if constexpr (D == 1) {   // t1 = z, t2 = x
        const float* a1 = m1 + c * kTVP;
        f0 = a[rv * kTVX + xv]; f1 = a1[rv * kTVX + xv]; f2 = a[rv * kTVX + xv + 1]; f3 = a1[rv * kTVX + xv + 1];
      } else {   // t1 = x, t2 = y (vertex plane p)
        f0 = a[rv * kTVX + xv]; f1 = a[rv * kTVX + xv + 1]; f2 = a[(rv + 1) * kTVX + xv]; f3 = a[(rv + 1) * kTVX + xv + 1];
      }
      met[c] = 0.25f * ((f0 + f1) + (f2 + f3));
    }
  }
  const long long fi = fix(b, D, i, j, p);
  const float Bn = in.B[D][b.face[D] + fi];
  float F[7], ye_up;
  face_flux<float, GR_EOS_IDEAL, D>(L, Rr, met, Bn, kp, F, &ye_up);
  float* out = reinterpret_cast<float*>(ws.flux[D]);
  const long long o = b.wface[D] + fi;
#pragma unroll
  for (int v = 0; v < 7; ++v) out[v * ws.fstride[D] + o] = F[v];
  // the block's flux flag (NaN and inf fail the test too)
  if (!(fabsf(F[1]) + fabsf(F[2]) + fabsf(F[3]) + fabsf(F[4]) < kFluxSafe)) *bad = 1;
}

template <int METHOD>
__global__ void __launch_bounds__(kTT, 3) k_faces_tile(const DBlock* __restrict__ blocks, const FaceTile* __restrict__ tiles,
                                                       const __grid_constant__ InView<float> in,
                                                       const __grid_constant__ Workspace ws,
                                                       const __grid_constant__ KParams kp) {
  extern __shared__ __align__(16) float sm[];
  const FaceTile tl = tiles[blockIdx.x];
  const DBlock b = blocks[tl.block];
  uint8_t* bad = ws.fbad + tl.block;
  const int n0 = b.n[0], n1 = b.n[1], n2 = b.n[2];
  const int j0 = tl.j0, j1 = tl.j1;
  const int rows = j1 - j0 + 6, vrows = j1 - j0 + 3;
  // face rows of this tile: x- and z-faces -1 .. n, y-faces 0 .. n, each row owned by one tile
  const int jlo = j0 == 0 ? -1 : j0, jhi = j1 == n1 ? n1 + 1 : j1;
  const int yhi = j1 == n1 ? n1 + 1 : j1;
  auto load_w = [&](int p) {
    float* d = sm + tW + tring(p, 6) * 7 * kTP;
#pragma unroll 1
    for (int v = 0; v < 5; ++v) tile_cell_plane(d + v * kTP, in.W[v], b, b.cell, p, j0, rows);
    tile_cell_plane(d + 5 * kTP, reinterpret_cast<const float*>(ws.bcc[0]), b, b.wcell, p, j0, rows);
    tile_cell_plane(d + 6 * kTP, reinterpret_cast<const float*>(ws.bcc[1]), b, b.wcell, p, j0, rows);
  };
  for (int p = -3; p <= 2; ++p) load_w(p);
  tile_cell_plane(sm + tBz + tring(-1, 2) * kTP, reinterpret_cast<const float*>(ws.bcc[2]), b, b.wcell, -1, j0, rows);
  tile_metric_plane(sm + tM + tring(-1, 2) * 10 * kTVP, in, b, -1, j0, vrows);
  tile_metric_plane(sm + tM + tring(0, 2) * 10 * kTVP, in, b, 0, j0, vrows);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  const int nx = (n0 + 1) * (jhi - jlo), ny = (n0 + 2) * (yhi - j0), nzr = (n0 + 2) * (jhi - jlo);
  for (int t = 0; t <= n2 + 1; ++t) {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    const int pf = t - 1;
    const int nz = t <= n2 ? nzr : 0;
    for (int q = threadIdx.x; q < nx + ny + nz; q += kTT) {
      if (q < nx) {
        const int i = q % (n0 + 1), j = jlo + q / (n0 + 1);
        tile_face<METHOD, 0>(sm, b, in, ws, kp, bad, j0, i, j, pf);
      } else if (q < nx + ny) {
        const int e = q - nx;
        const int i = e % (n0 + 2) - 1, j = j0 + e / (n0 + 2);
        tile_face<METHOD, 1>(sm, b, in, ws, kp, bad, j0, i, j, pf);
      } else {
        const int e = q - nx - ny;
        const int i = e % (n0 + 2) - 1, j = jlo + e / (n0 + 2);
        tile_face<METHOD, 2>(sm, b, in, ws, kp, bad, j0, i, j, t);
      }
    }
    __syncthreads();
    // the planes step t + 1 adds, into slots this step no longer reads
    if (t + 3 <= n2 + 2) load_w(t + 3);
    if (t <= n2)
      tile_cell_plane(sm + tBz + tring(t, 2) * kTP, reinterpret_cast<const float*>(ws.bcc[2]), b, b.wcell, t, j0, rows);
    if (t + 1 <= n2 + 1) tile_metric_plane(sm + tM + tring(t + 1, 2) * 10 * kTVP, in, b, t + 1, j0, vrows);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <int METHOD>
static cudaError_t launch_tile_m(const DBlock* blocks, const FaceTile* tiles, int ntiles, const InView<float>& in,
                                 const Workspace& ws, const KParams& kp, cudaStream_t st) {
  static unsigned long long attr = 0;   // the shared-memory opt-in, once per device
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev < 64 && !((attr >> dev) & 1ull)) {
    const cudaError_t e = cudaFuncSetAttribute(k_faces_tile<METHOD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kTSmem);
    if (e != cudaSuccess) return e;
    attr |= 1ull << dev;
  }
  k_faces_tile<METHOD><<<ntiles, kTT, kTSmem, st>>>(blocks, tiles, in, ws, kp);
  return cudaGetLastError();
}

cudaError_t launch_faces_tile(const DBlock* blocks, const FaceTile* tiles, int ntiles, const InView<float>& in,
                              const Workspace& ws, const KParams& kp, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  switch (kp.recon) {
    case GR_RECON_PLM: return launch_tile_m<GR_RECON_PLM>(blocks, tiles, ntiles, in, ws, kp, st);
    case GR_RECON_WENO5: return launch_tile_m<GR_RECON_WENO5>(blocks, tiles, ntiles, in, ws, kp, st);
    case GR_RECON_PPM: return launch_tile_m<GR_RECON_PPM>(blocks, tiles, ntiles, in, ws, kp, st);
    default: return launch_tile_m<GR_RECON_WENOZ>(blocks, tiles, ntiles, in, ws, kp, st);
  }
}

}  // namespace grs
