// driver.cu -- device side of the multi-block RK step: ghost exchange between same-level blocks and
// the time step on the device (the RK3 integration stated at the start of Sec. 4; the global CFL time
// step of Sec. 3.1, or a wave-speed rule).
//
//   k_ghost      every ghost cell and ghost face of every block is copied from the block that the
//                neighbour table names for its direction (or, at an outflow boundary, from the
//                nearest owned element of the same block); one CTA per block and element kind
//                striding over the ghost shell only.  Sources are always owned elements, so copies
//                never race with each other.
//   k_cfl_rate   max over interior cells and directions of max(|lambda-|, |lambda+|)/dx_d (the fast
//                speeds of Sec. 2.2 at the cell state), warp-reduced, one atomic max per warp
//   k_cfl_dt     dt = CFL / rate, left on the device for the stages to read
#include <algorithm>
#include <vector>

#include "internal.h"
#include "physics.cuh"
#include "stage_common.cuh"

namespace grs {

struct GhostArgs {
  double* W[7];
  int nw;
  double* B[3];
  const int* nbr;   // 27 entries per block
  GhostMap map;
  float* W32[6];    // optional FP32 copies of W[0..5] and B (the mixed path's reconstruction input): their
  float* B32[3];    // ghosts get the FP32 conversion of the copied FP64 value
};

__host__ __device__ __forceinline__ int nbr_slot(const int o[3]) { return (o[2] + 1) * 9 + (o[1] + 1) * 3 + (o[0] + 1); }

// Ghost shell of a box: the elements of the full array (extent F[a] from -g) outside the owned box
// (extent O[a] from 0), F[a] - O[a] = 2g.  Enumerated as the two z slabs (full x-y planes), then the
// two y slabs of each owned z (full x rows), then the two x runs of each owned (y, z) row, so that
// consecutive threads touch consecutive x wherever the rows are long.
__host__ __device__ __forceinline__ int shell_count(const int F[3], const int O[3]) {
  return F[0] * F[1] * F[2] - O[0] * O[1] * O[2];
}

static void shell_decode(int e, const int F[3], const int O[3], int g, int p[3]) {
  const int nz = (F[2] - O[2]) * F[1] * F[0];
  if (e < nz) {
    const int t = e / (F[1] * F[0]), r = e - t * F[1] * F[0];
    p[2] = t < g ? t - g : O[2] + t - g;
    p[1] = r / F[0] - g;
    p[0] = r % F[0] - g;
    return;
  }
  e -= nz;
  const int ny = O[2] * (F[1] - O[1]) * F[0];
  if (e < ny) {
    const int row = e / F[0];
    p[0] = e - row * F[0] - g;
    const int t = row % (F[1] - O[1]);
    p[1] = t < g ? t - g : O[1] + t - g;
    p[2] = row / (F[1] - O[1]);
    return;
  }
  e -= ny;
  const int w = F[0] - O[0];
  const int row = e / w, t = e - row * w;
  p[0] = t < g ? t - g : O[0] + t - g;
  p[1] = row % O[1];
  p[2] = row / O[1];
}

// side of coordinate x of an axis with owned extent own: -1 below, 0 inside, +1 above
static inline int side(int x, int own) { return x < 0 ? -1 : (x >= own ? 1 : 0); }

// full (F) and owned (O) extents of element kind D (-1 cells, 0..2 faces) of a block
__host__ __device__ __forceinline__ void shell_extents(const DBlock& b, int D, int F[3], int O[3]) {
  for (int d = 0; d < 3; ++d) {
    F[d] = b.N[d] + (d == D);
    O[d] = b.n[d] + (d == D);
  }
}

int build_ghost_map(const DBlock* hb, int nblocks, std::vector<int2>& ent, std::vector<int>& out,
                    std::vector<int4>& off) {
  ent.clear();
  out.clear();
  off.assign(nblocks, int4{0, 0, 0, 0});
  std::vector<int> rep;   // first block of each distinct shape
  for (int b = 0; b < nblocks; ++b) {
    const DBlock& x = hb[b];
    int found = -1;
    for (size_t r = 0; r < rep.size() && found < 0; ++r) {
      const DBlock& y = hb[rep[r]];
      if (x.g == y.g && x.n[0] == y.n[0] && x.n[1] == y.n[1] && x.n[2] == y.n[2]) found = (int)r;
    }
    if (found >= 0) {
      off[b] = off[rep[found]];
      continue;
    }
    rep.push_back(b);
    int o4[4];
    for (int D = -1; D < 3; ++D) {
      int F[3], O[3];
      shell_extents(x, D, F, O);
      if ((long long)F[0] * F[1] * F[2] >= kGhostMapMaxLocal) return -1;
      o4[D + 1] = (int)ent.size();
      const int cnt = shell_count(F, O);
      for (int e = 0; e < cnt; ++e) {
        int p[3], o[3], qn[3], qo[3];
        shell_decode(e, F, O, x.g, p);
        for (int d = 0; d < 3; ++d) {
          o[d] = side(p[d], O[d]);
          qn[d] = p[d] - o[d] * x.n[d];                // in the neighbour across o
          qo[d] = std::min(std::max(p[d], 0), O[d] - 1);   // outflow: nearest owned element
        }
        const long long dst = D < 0 ? cix(x, p[0], p[1], p[2]) : fix(x, D, p[0], p[1], p[2]);
        const long long srn = D < 0 ? cix(x, qn[0], qn[1], qn[2]) : fix(x, D, qn[0], qn[1], qn[2]);
        const long long sro = D < 0 ? cix(x, qo[0], qo[1], qo[2]) : fix(x, D, qo[0], qo[1], qo[2]);
        const unsigned packed = ((unsigned)nbr_slot(o) << 27) | (unsigned)srn;
        ent.push_back(int2{(int)dst, (int)packed});
        out.push_back((int)sro);
      }
    }
    off[b] = int4{o4[0], o4[1], o4[2], o4[3]};
  }
  return 0;
}

// One CTA per (block, array): the nw cell fields, then the x-, y- and z-face fields, so that every CTA
// copies one 8-byte array over its block's ghost shell (the same amount of work for all of them).  Each
// element's destination, neighbour slot and source offset come from the gather map of the block's shape
// (shared by all blocks of that shape, so it stays in L2).  Neighbours have the block's own sizes
// (checked when the driver is made), so a source element is the neighbour's base offset (the 27 bases
// staged in shared memory) plus the mapped offset.  Each thread copies kGhostU elements per pass, all
// loads before all stores: sources are owned elements and destinations ghosts, so they never alias, but
// the compiler cannot know that and would otherwise wait for each store before the next load.
constexpr int kGhostU = 8;

template <int D>
__device__ __forceinline__ void ghost_copy(const DBlock& b, const long long* sbase, const int2* __restrict__ ent,
                                           const int* __restrict__ outm, const double* src_arr, double* dst_arr,
                                           float* dst32) {
  int F[3], O[3];
  shell_extents(b, D, F, O);
  const int cnt = shell_count(F, O);
  const long long own = D < 0 ? b.cell : b.face[D < 0 ? 0 : D];
  constexpr int kStride = kGhostU * kGhostTile;
  // the map entries of the next pass are loaded while this pass's copies are in flight
  int2 t[kGhostU];
#pragma unroll
  for (int u = 0; u < kGhostU; ++u) {
    const int e = (int)threadIdx.x + u * kGhostTile;
    t[u] = e < cnt ? __ldg(ent + e) : int2{-1, 0};
  }
  for (int e0 = threadIdx.x; e0 < cnt; e0 += kStride) {
    long long dst[kGhostU];
    double v[kGhostU];
#pragma unroll
    for (int u = 0; u < kGhostU; ++u) {
      dst[u] = -1;
      if (t[u].x >= 0) {
        const long long base = sbase[(unsigned)t[u].y >> 27];
        const long long src = base >= 0 ? base + (t[u].y & (int)(kGhostMapMaxLocal - 1))
                                        : own + __ldg(outm + e0 + u * kGhostTile);
        dst[u] = own + t[u].x;
        v[u] = src_arr[src];
      }
    }
#pragma unroll
    for (int u = 0; u < kGhostU; ++u) {
      const int e = e0 + kStride + u * kGhostTile;
      t[u] = e < cnt ? __ldg(ent + e) : int2{-1, 0};
    }
#pragma unroll
    for (int u = 0; u < kGhostU; ++u)
      if (dst[u] >= 0) dst_arr[dst[u]] = v[u];
    if (dst32) {
#pragma unroll
      for (int u = 0; u < kGhostU; ++u)
        if (dst[u] >= 0) dst32[dst[u]] = d2f_rn(v[u]);
    }
  }
}

__global__ void __launch_bounds__(kGhostTile, 4) k_ghost(const DBlock* __restrict__ blocks,
                                                      const __grid_constant__ GhostArgs a) {
  __shared__ long long sbase[27];   // base offset of the source block per direction, -1: outflow
  const int na = a.nw + 3;
  const int blk = blockIdx.x / na, arr = (int)(blockIdx.x - blk * na);
  const int kind = arr < a.nw ? 0 : arr - a.nw + 1;   // 0 cells, 1 + D: D-faces
  const DBlock b = blocks[blk];
  if (threadIdx.x < 27) {
    const int src = __ldg(a.nbr + 27 * blk + threadIdx.x);
    sbase[threadIdx.x] = src < 0 ? -1 : (kind == 0 ? blocks[src].cell : blocks[src].face[kind - 1]);
  }
  __syncthreads();
  const int4 o = __ldg(a.map.off + blk);
  const int eo = kind == 0 ? o.x : (kind == 1 ? o.y : (kind == 2 ? o.z : o.w));
  const int2* ent = a.map.ent + eo;
  const int* outm = a.map.out + eo;
  if (kind == 0) {
    float* w32 = arr < 6 ? a.W32[arr] : nullptr;   // no FP32 copy of T (table)
    ghost_copy<-1>(b, sbase, ent, outm, a.W[arr], a.W[arr], w32);
  } else if (kind == 1) {
    ghost_copy<0>(b, sbase, ent, outm, a.B[0], a.B[0], a.B32[0]);
  } else if (kind == 2) {
    ghost_copy<1>(b, sbase, ent, outm, a.B[1], a.B[1], a.B32[1]);
  } else {
    ghost_copy<2>(b, sbase, ent, outm, a.B[2], a.B[2], a.B32[2]);
  }
}

__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

template <int EOS>
__global__ void __launch_bounds__(kTile) k_cfl_rate(const DBlock* __restrict__ blocks, const Work* __restrict__ work,
                                                    const __grid_constant__ InView<double> in,
                                                    const __grid_constant__ KParams kp, double* rate) {
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  int p[3];
  double r = 0.0;
  if (decode<R_INTERIOR, 0>(w, b, p)) {
    const int i = p[0], j = p[1], k = p[2];
    double val[16];
    cell_metric<double>(b, in, in.order, i, j, k, 0, 10, val, nullptr);
    CellMet<double> M;
    cellmet_from<double>(val, true, M);
    const long long c = b.cell + cix(b, i, j, k);
    double wv[6], Bd[3];
    for (int v = 0; v < 5; ++v) wv[v] = in.W[v][c];
    wv[5] = EOS ? in.W[5][c] : 0.0;
    const long long f0 = b.face[0] + fix(b, 0, i, j, k), f1 = b.face[1] + fix(b, 1, i, j, k);
    const long long f2 = b.face[2] + fix(b, 2, i, j, k);
    Bd[0] = 0.5 * (in.B[0][f0] + in.B[0][f0 + 1]);
    Bd[1] = 0.5 * (in.B[1][f1] + in.B[1][f1 + b.N[0]]);
    Bd[2] = 0.5 * (in.B[2][f2] + in.B[2][f2 + (long long)b.N[0] * b.N[1]]);
    CellFluid<double> fl;
    cell_fluid<double, EOS>(M, kp, wv, Bd, fl);
    double rhoh, cs2;
    eos_rhoh_cs2<double, EOS>(kp, fl.rho, fl.p, wv[5], &rhoh, &cs2);
    // fast speeds along each direction (the expression of the face states, at the cell centre)
    const double ca2 = fl.b2 / (rhoh + fl.b2);
    const double c2 = cs2 + ca2 - cs2 * ca2;
    const double v2 = fl.v[0] * fl.vl[0] + fl.v[1] * fl.vl[1] + fl.v[2] * fl.vl[2];
    const double iden = 1.0 / (1.0 - v2 * c2);
    const double cc = sqrt(c2);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double gdd = M.gi[d == 0 ? 0 : (d == 1 ? 3 : 5)];
      double disc = (1.0 - v2) * (gdd * (1.0 - v2 * c2) - fl.v[d] * fl.v[d] * (1.0 - c2));
      disc = disc > 0.0 ? disc : 0.0;
      const double cr = cc * sqrt(disc);
      const double vc = fl.v[d] * (1.0 - c2);
      const double lp = M.alpha * (vc + cr) * iden - M.beta[d];
      const double lm = M.alpha * (vc - cr) * iden - M.beta[d];
      r = fmax(r, fmax(fabs(lp), fabs(lm)) * b.idx[d]);
    }
    if (!(r == r)) r = __longlong_as_double(0x7FF0000000000000LL);   // NaN state: no finite dt
  }
  for (int off = 16; off > 0; off >>= 1) r = fmax(r, __shfl_down_sync(0xffffffffu, r, off));
  if ((threadIdx.x & 31) == 0) atomic_max_pos(rate, r);
}

__global__ void k_set_scalar(double* dst, double v) { *dst = v; }

cudaError_t launch_set_scalar(double* dst, double value, cudaStream_t st) {
  k_set_scalar<<<1, 1, 0, st>>>(dst, value);
  return cudaGetLastError();
}

__global__ void k_cfl_dt(const double* rate, double cfl, double* dt) {
  const double r = *rate;
  *dt = r > 0.0 ? cfl / r : 0.0;
}

cudaError_t launch_ghost_fill(const DBlock* blocks, int nblocks, const int* nbr, const GhostMap& gm,
                              double* const W[7], int nw, double* const B[3], cudaStream_t st,
                              float* const* W32, float* const* B32) {
  GhostArgs a{};
  a.map = gm;
  for (int v = 0; v < 7; ++v) a.W[v] = v < nw ? W[v] : nullptr;
  a.nw = nw;
  for (int d = 0; d < 3; ++d) a.B[d] = B[d];
  a.nbr = nbr;
  if (W32 && B32) {
    for (int v = 0; v < 6; ++v) a.W32[v] = v < nw ? W32[v] : nullptr;
    for (int d = 0; d < 3; ++d) a.B32[d] = B32[d];
  }
  if (nblocks) k_ghost<<<(nw + 3) * nblocks, kGhostTile, 0, st>>>(blocks, a);
  return cudaGetLastError();
}

cudaError_t launch_cfl_dt(const DBlock* blocks, const Work* wi, int nwi, const MetricView& m,
                          const double* const W[7], const double* const B[3], const KParams& kp, double cfl,
                          double* rate, double* dt, cudaStream_t st) {
  InView<double> in;
  for (int c = 0; c < 16; ++c) in.M[c] = m.v[c];
  for (int v = 0; v < 6; ++v) in.W[v] = W[v];
  for (int d = 0; d < 3; ++d) in.B[d] = B[d];
  in.order = m.order;
  in.k_zero = m.k_zero;
  cudaError_t e = cudaMemsetAsync(rate, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  if (nwi) {
    if (kp.eos == GR_EOS_TABLE) k_cfl_rate<GR_EOS_TABLE><<<nwi, kTile, 0, st>>>(blocks, wi, in, kp, rate);
    else k_cfl_rate<GR_EOS_IDEAL><<<nwi, kTile, 0, st>>>(blocks, wi, in, kp, rate);
  }
  k_cfl_dt<<<1, 1, 0, st>>>(rate, cfl, dt);
  return cudaGetLastError();
}

}  // namespace grs
