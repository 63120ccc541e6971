// stage_kernels.cu -- the GRMHD stage as a short sequence of kernels per call (sm_103a).
//
//   k_cast       (mixed path only) FP32 copies of the stage inputs W, B and the metric, made with
//                integer bit arithmetic so that no conversion runs on GB300's narrow FP64 pipe
//   k_cellprep   cell-centred field calB^i = mean of faces / sqrt(gamma) on all cells, and the
//                cell electric field E_m = alpha (v~^b B^a - v~^a B^b) on the ring -1..n  (Sec. 3.3);
//                with the order-2 metric k_cellprep_sweep: the same per tile of a block's x-y plane,
//                walked along z with the vertex planes in shared memory
//   k_faces<R>   reconstruction (Sec. 3.4) + face metric (Sec. 3.2) + HLLE flux (Eq. fluxB_def)
//                on every face with normal index 0..n and transverse index -1..n; with a tabulated
//                EOS (Sec. 2.2.1) also Y_e, and the D Y_e flux = D flux x upwind Y_e (faces_impl.cuh;
//                the mixed WENOZ evaluates both face states in packed FP32x2)
//   k_edges<R>   upwinded corner electric field from the four adjacent face fluxes (Sec. 3.3)
//   k_ct         constrained-transport face update B' = g0 B0 + g1 B - beta dt curl E  (FP64)
//   k_update     FP64 path: flux divergence + geometric sources (Eq. claw, Eq. hydsrc_def)
//                accumulated in FP64 and the atmosphere test (Sec. 3.5); mixed path: D' and the
//                atmosphere test only; atmosphere cells are reset, the others queued for k_c2p
//   k_c2p        on the compacted job list: (mixed path) the cell's U' as above, then FP64 con2prim
//                (Sec. 3.5, App. A)
//
// Kernels that evaluate the EOS are instantiated per EOS (ideal gas / table) as well as per R.
// Every kernel but the sweep and k_c2p takes one work item (block, direction, first element) per CTA;
// blocks of different sizes share one launch.  Within a work item the direction is a compile-time
// constant (one instantiation per direction), so no small array is indexed at run time.  Face fluxes
// and corner fields pass through the mesh's workspace in the arithmetic type R.
#include <cstdio>

#include "internal.h"
#include "physics.cuh"
#include "stage_common.cuh"
#include "update_common.cuh"

namespace grs {

// ------------------------------------------------------------------------------------------------
// k_cast: FP64 -> FP32 copies of up to 24 pools
// ------------------------------------------------------------------------------------------------
struct CastList {
  const double* src[24];
  float* dst[24];
  long long n[24];
  int count;
};

__global__ void __launch_bounds__(256) k_cast(const __grid_constant__ CastList L) {
  const int seg = blockIdx.y;
  if (seg >= L.count) return;
  const double* __restrict__ s = L.src[seg];
  float* __restrict__ d = L.dst[seg];
  const long long n = L.n[seg];
  const long long step = (long long)gridDim.x * blockDim.x;
  const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if ((((unsigned long long)s) & 15ull) || (((unsigned long long)d) & 7ull)) {   // unaligned pool: scalar
    for (long long i = i0; i < n; i += step) d[i] = d2f_rn(s[i]);
    return;
  }
  const long long n2 = n / 2;
  const double2* s2 = reinterpret_cast<const double2*>(s);
  float2* d2 = reinterpret_cast<float2*>(d);
  for (long long i = i0; i < n2; i += step) {
    const double2 v = s2[i];
    d2[i] = make_float2(d2f_rn(v.x), d2f_rn(v.y));
  }
  if (i0 == 0 && (n & 1)) d[n - 1] = d2f_rn(s[n - 1]);
}

// ------------------------------------------------------------------------------------------------
// k_cellprep<R>: undensitised cell field calB^i = mean of the face values / sqrt(gamma) on every cell,
// and the cell-centred electric field E_m = alpha (vt x calB)_m on cells -1..n (the EMF input)
// ------------------------------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void cellprep_cell(const DBlock& b, const InView<R>& in, const Workspace& ws, int i,
                                              int j, int k, const R val[10]) {
  const R* g6 = val + 4;
  const R sg = sqrt_r(det3(g6));
  R Bd[3];
  const long long f0 = b.face[0] + fix(b, 0, i, j, k), f1 = b.face[1] + fix(b, 1, i, j, k);
  const long long f2 = b.face[2] + fix(b, 2, i, j, k);
  Bd[0] = R(0.5) * (in.B[0][f0] + in.B[0][f0 + 1]);
  Bd[1] = R(0.5) * (in.B[1][f1] + in.B[1][f1 + b.N[0]]);
  Bd[2] = R(0.5) * (in.B[2][f2] + in.B[2][f2 + (long long)b.N[0] * b.N[1]]);
  const long long wc = b.wcell + cix(b, i, j, k);
  const R isg = rdiv(R(1), sg);
#pragma unroll
  for (int a = 0; a < 3; ++a) reinterpret_cast<R*>(ws.bcc[a])[wc] = Bd[a] * isg;
  const bool ring = i >= -1 && i <= b.n[0] && j >= -1 && j <= b.n[1] && k >= -1 && k <= b.n[2];
  if (!ring) return;
  const long long c = b.cell + cix(b, i, j, k);
  const R ut[3] = {in.W[1][c], in.W[2][c], in.W[3][c]};
  R utl[3];
  lower3(g6, ut, utl);
  const R iW = rdiv(R(1), sqrt_w(R(1) + ut[0] * utl[0] + ut[1] * utl[1] + ut[2] * utl[2]));
  const R ia = rdiv(R(1), val[0]);
  R vt[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) vt[a] = ut[a] * iW - val[1 + a] * ia;
#pragma unroll
  for (int mm = 0; mm < 3; ++mm) {
    const int a = (mm + 1) % 3, bb = (mm + 2) % 3;
    reinterpret_cast<R*>(ws.ecc[mm])[wc] = val[0] * (vt[bb] * Bd[a] - vt[a] * Bd[bb]);
  }
}

template <class R>
__device__ __forceinline__ void cellprep_body(const Work& w, const DBlock& b, const InView<R>& in,
                                              const Workspace& ws) {
  int p[3];
  if (!decode<R_CELLS_ALL, 0>(w, b, p)) return;
  if (in.order == 4) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (p[a] < -b.g + 1 || p[a] > b.n[a] + b.g - 2) return;
  }
  R val[10];
  cell_metric<R>(b, in, in.order, p[0], p[1], p[2], 0, 10, val, nullptr);
  cellprep_cell<R>(b, in, ws, p[0], p[1], p[2], val);
}

// Every stage kernel strides over its work list (one work item per CTA and pass): launched with one CTA
// per item, or persistent with as many CTAs as fit on the GPU.  The CTA size equals the work-item size.
template <class R>
__global__ void __launch_bounds__(kMaxTile) k_cellprep(const DBlock* __restrict__ blocks, const Work* __restrict__ work,
                                                       int nwork, const __grid_constant__ InView<R> in,
                                                       const __grid_constant__ Workspace ws) {
  for (int it = blockIdx.x; it < nwork; it += gridDim.x) {
    const Work w = work[it];
    cellprep_body<R>(w, blocks[w.block], in, ws);
  }
}

// k_cellprep_sweep<R> (order-2 metric): the same outputs, bitwise, with each vertex of the metric read
// from memory once per tile instead of by each of its eight cells.  One CTA per SweepWork tile walks the
// block along z; the vertex planes z and z + 1 of the tile (with its +1 halo in x and y) sit in shared
// memory (cp.async, two buffers), and each thread carries the 2 x 2 plane sums of its cell column from one
// cell to the next: the cell value is 1/8 ((f0 + f1) + (f2 + f3)) + ((f4 + f5) + (f6 + f7)) in the
// order cell_metric sums it, the first bracket being the previous cell's second.
template <class R>
__device__ __forceinline__ void sweep_copy(R* dst, const R* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(sizeof(R)) : "memory");
}
__device__ __forceinline__ void sweep_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void sweep_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <class R>
__global__ void __launch_bounds__(kSweepThreads) k_cellprep_sweep(const DBlock* __restrict__ blocks,
                                                                  const SweepWork* __restrict__ work,
                                                                  const __grid_constant__ InView<R> in,
                                                                  const __grid_constant__ Workspace ws) {
  extern __shared__ __align__(16) unsigned char sweep_smem[];
  R* sm = reinterpret_cast<R*>(sweep_smem);   // [buffer 2][component 10][kSweepVerts]
  const SweepWork w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  const int TX = w.txy & 0xFFFF, TY = w.txy >> 16;
  const int VX = TX + 1, NV = VX * (TY + 1);
  const int tx = (int)threadIdx.x % TX, ty = (int)threadIdx.x / TX;
  const bool act = ty < TY && w.x0 + tx < b.N[0] && w.y0 + ty < b.N[1];
  const int i = w.x0 + tx - b.g, j = w.y0 + ty - b.g;
  // the (at most two) tile vertices this thread copies: offsets within a vertex plane, or -1
  const long long VP = (long long)(b.N[0] + 1) * (b.N[1] + 1);
  long long voff[2];
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const int t = (int)threadIdx.x + m * kSweepThreads;
    const int X = w.x0 + t % VX, Y = w.y0 + t / VX;
    voff[m] = (t < NV && X <= b.N[0] && Y <= b.N[1]) ? (long long)Y * (b.N[0] + 1) + X : -1;
  }
  auto load_plane = [&](int kv, int buf) {   // vertex plane kv (0..N2) into buffer buf, one commit group
#pragma unroll
    for (int m = 0; m < 2; ++m)
      if (voff[m] >= 0) {
        const long long vi = b.vert + kv * VP + voff[m];
        const int t = (int)threadIdx.x + m * kSweepThreads;
#pragma unroll
        for (int c = 0; c < 10; ++c) sweep_copy<R>(sm + (buf * 10 + c) * kSweepVerts + t, in.M[c] + vi);
      }
    sweep_commit();
  };
  auto plane_sum = [&](int buf, R S[10]) {   // (f(i,j) + f(i+1,j)) + (f(i,j+1) + f(i+1,j+1))
    const int o = ty * VX + tx;
#pragma unroll
    for (int c = 0; c < 10; ++c) {
      const R* a = sm + (buf * 10 + c) * kSweepVerts + o;
      S[c] = (a[0] + a[1]) + (a[VX] + a[VX + 1]);
    }
  };
  const int N2 = b.N[2];
  load_plane(0, 0);
  load_plane(1, 1);
  sweep_wait1();
  __syncthreads();
  R S0[10], S1[10];
  if (act) plane_sum(0, S0);
  for (int kc = 0; kc < N2; ++kc) {
    __syncthreads();   // every thread is done with buffer kc & 1 (plane kc)
    if (kc + 2 <= N2) load_plane(kc + 2, kc & 1);
    else sweep_commit();   // an empty group keeps wait_group 1 meaning "plane kc + 1 has landed"
    sweep_wait1();
    __syncthreads();
    if (act) {
      plane_sum((kc + 1) & 1, S1);
      R val[10];
#pragma unroll
      for (int c = 0; c < 10; ++c) {
        val[c] = R(0.125) * (S0[c] + S1[c]);
        S0[c] = S1[c];
      }
      cellprep_cell<R>(b, in, ws, i, j, kc - b.g, val);
    }
  }
}

template <class R>
static cudaError_t launch_cellprep_sweep(const DBlock* blocks, const InView<R>& in, const Workspace& ws,
                                         cudaStream_t st) {
  constexpr size_t smem = sizeof(R) * 2 * 10 * kSweepVerts;
  // above the default 48 KB: the opt-in is per device (set once on each, one bit per device)
  static unsigned long long attr = 0;
  int dev = 0;
  if (smem > 48 * 1024 && cudaGetDevice(&dev) == cudaSuccess && dev < 64 && !((attr >> dev) & 1ull)) {
    const cudaError_t e = cudaFuncSetAttribute(k_cellprep_sweep<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr |= 1ull << dev;
  }
  k_cellprep_sweep<R><<<ws.nsweep, kSweepThreads, smem, st>>>(blocks, ws.sweep, in, ws);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// k_edges<R>: corner electric field E_m at (a-face ia, b-face ib, m-cell im), (a, b, m) cyclic
// ------------------------------------------------------------------------------------------------
template <class R, int M>
__device__ __forceinline__ void edge_body(const Work& w, const DBlock& b, const Workspace& ws,
                                          const KParams& kp) {
  int e[3];
  if (!decode<R_EDGES, M>(w, b, e)) return;
  constexpr int A = (M + 1) % 3, BB = (M + 2) % 3;
  const R* Fa = reinterpret_cast<const R*>(ws.flux[A]);
  const R* Fb = reinterpret_cast<const R*>(ws.flux[BB]);
  const long long sa = ws.fstride[A], sb = ws.fstride[BB];
  // a-face values at b-cells ib and ib-1; b-face values at a-cells ia and ia-1
  const long long fa1 = b.wface[A] + fix(b, A, e[0], e[1], e[2]);
  const long long fa0 = fa1 - face_stride<A>(b, BB);
  const long long fb1 = b.wface[BB] + fix(b, BB, e[0], e[1], e[2]);
  const long long fb0 = fb1 - face_stride<BB>(b, A);
  const R Ea1 = -Fa[5 * sa + fa1], Ea0 = -Fa[5 * sa + fa0];   // E_m = -F^a_{B^b}
  const R Eb1 = Fb[6 * sb + fb1], Eb0 = Fb[6 * sb + fb0];     // E_m = +F^b_{B^a}
  R E = R(0.25) * (Ea1 + Ea0 + Eb1 + Eb0);
  if (kp.emf == GR_EMF_UPWIND) {
    const R* ecc = reinterpret_cast<const R*>(ws.ecc[M]);
    const long long c11 = b.wcell + cix(b, e[0], e[1], e[2]);
    const long long sA = cell_stride(b, A), sB = cell_stride(b, BB);
    const R C11 = ecc[c11], C01 = ecc[c11 - sA], C10 = ecc[c11 - sB], C00 = ecc[c11 - sA - sB];
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
  reinterpret_cast<R*>(ws.edge[M])[b.wvert + vix(b, e[0], e[1], e[2])] = E;
}

template <class R>
__global__ void __launch_bounds__(kMaxTile) k_edges(const DBlock* __restrict__ blocks, const Work* __restrict__ work,
                                                    int nwork, const __grid_constant__ Workspace ws,
                                                    const __grid_constant__ KParams kp) {
  for (int it = blockIdx.x; it < nwork; it += gridDim.x) {
    const Work w = work[it];
    const DBlock b = blocks[w.block];
    if (w.dir == 0) edge_body<R, 0>(w, b, ws, kp);
    else if (w.dir == 1) edge_body<R, 1>(w, b, ws, kp);
    else edge_body<R, 2>(w, b, ws, kp);
  }
}

// ------------------------------------------------------------------------------------------------
// k_ct: B'^d on faces of interior cells (FP64)
// ------------------------------------------------------------------------------------------------
template <class R, int D, int RKF>
__device__ __forceinline__ void ct_body(const Work& w, const DBlock& b, const StateView& s,
                                        const Workspace& ws, const KParams& kp) {
  int p[3];
  if (!decode<R_CTFACES, D>(w, b, p)) return;
  constexpr int t1 = (D + 1) % 3, t2 = (D + 2) % 3;
  const R* E2 = reinterpret_cast<const R*>(ws.edge[t2]);
  const R* E1 = reinterpret_cast<const R*>(ws.edge[t1]);
  const long long v0 = b.wvert + vix(b, p[0], p[1], p[2]);
  const long long vs1 = t1 == 0 ? 1 : (t1 == 1 ? (long long)(b.N[0] + 1) : (long long)(b.N[0] + 1) * (b.N[1] + 1));
  const long long vs2 = t2 == 0 ? 1 : (t2 == 1 ? (long long)(b.N[0] + 1) : (long long)(b.N[0] + 1) * (b.N[1] + 1));
  // FP64 (the B' differences must stay exact enough for div B at round-off); GB300's FP64 rate is
  // ~1/64 of FP32, so the operation count is kept minimal: curl = idx1 dE2 - idx2 dE1 by one
  // multiply and one FMA, then B' = g1 B - beta dt curl by one FMA, with the RK form (RKF) fixed at
  // compile time so that g1 = 1 and g0 = 0 cost no FP64 instruction
  const double dE2 = diff64(E2[v0 + vs1], E2[v0]);
  const double dE1 = diff64(E1[v0 + vs2], E1[v0]);
  const double curl = fma(b.idx[t1], dE2, -(b.idx[t2] * dE1));
  const long long f = b.face[D] + fix(b, D, p[0], p[1], p[2]);
  const double B = s.B[D][f];
  double Bn = fma(-stage_bdt(kp), curl, (RKF & RK_G1) ? kp.rk_g1 * B : B);
  if constexpr ((RKF & RK_G0) != 0) Bn = fma(kp.rk_g0, s.B0[D][f], Bn);
  s.Bo[D][f] = Bn;
  if (s.Bo32[D]) s.Bo32[D][f] = d2f_rn(Bn);
}

template <class R, int RKF>
__device__ __forceinline__ void ct_loop(const DBlock* __restrict__ blocks, const Work* __restrict__ work, int nwork,
                                        const StateView& s, const Workspace& ws, const KParams& kp) {
  for (int it = blockIdx.x; it < nwork; it += gridDim.x) {
    const Work w = work[it];
    const DBlock b = blocks[w.block];
    if (w.dir == 0) ct_body<R, 0, RKF>(w, b, s, ws, kp);
    else if (w.dir == 1) ct_body<R, 1, RKF>(w, b, s, ws, kp);
    else ct_body<R, 2, RKF>(w, b, s, ws, kp);
  }
}

template <class R>
__global__ void __launch_bounds__(kMaxTile) k_ct(const DBlock* __restrict__ blocks, const Work* __restrict__ work,
                                                 int nwork, const __grid_constant__ StateView s,
                                                 const __grid_constant__ Workspace ws,
                                                 const __grid_constant__ KParams kp) {
  switch (kp.rk_form) {   // uniform over the grid: one branch, taken once
    case 0: ct_loop<R, 0>(blocks, work, nwork, s, ws, kp); break;
    case RK_G0: ct_loop<R, RK_G0>(blocks, work, nwork, s, ws, kp); break;
    case RK_G1: ct_loop<R, RK_G1>(blocks, work, nwork, s, ws, kp); break;
    default: ct_loop<R, RK_G0 | RK_G1>(blocks, work, nwork, s, ws, kp); break;
  }
}

// ------------------------------------------------------------------------------------------------
// k_update<R>: U' (sources in R, FP64 accumulation) and FP64 con2prim on interior cells
// ------------------------------------------------------------------------------------------------
// FP64 gamma_ij at a cell centre (con2prim's metric; FAST: c2pmet_from's form for the mixed stage)
template <bool FAST = false>
__device__ __forceinline__ void cell_gamma64(const DBlock& b, const InView<double>& m, int i, int j, int k,
                                             C2PMet& M) {
  double val[10];
  cell_metric<double>(b, m, m.order, i, j, k, 4, 10, val, nullptr);
  c2pmet_from<FAST>(val + 4, M);
}

// Conserved variable v of interior cell (i, j, k) after the stage from the workspace's face fluxes
// (component of v: D, S_j, tau at 0..4; D Y_e at 7 -- 5, 6 are the induction fluxes)
template <class R>
__device__ __forceinline__ double accumulate_cell(const DBlock& b, const StateView& s, const Workspace& ws,
                                                  const KParams& kp, int i, int j, int k, long long c, int v,
                                                  R src) {
  const int cv = v < 5 ? v : 7;
  const R* a0 = reinterpret_cast<const R*>(ws.flux[0]) + cv * ws.fstride[0] + b.wface[0] + fix(b, 0, i, j, k);
  const R* a1 = reinterpret_cast<const R*>(ws.flux[1]) + cv * ws.fstride[1] + b.wface[1] + fix(b, 1, i, j, k);
  const R* a2 = reinterpret_cast<const R*>(ws.flux[2]) + cv * ws.fstride[2] + b.wface[2] + fix(b, 2, i, j, k);
  const long long oy = b.N[0], oz = (long long)b.N[0] * b.N[1];
  return accumulate_vals<R>(b, s, kp, c, v, src, a0[0], a0[1], a1[0], a1[oy], a2[0], a2[oz]);
}

// U' of every conserved variable of interior cell (i, j, k): the geometric sources (cell_sources_at), then
// accumulate_cell.  M: the cell metric, for the caller.
template <class R, int EOS>
__device__ __forceinline__ void update_all(const DBlock& b, const InView<R>& in, const StateView& s,
                                           const Workspace& ws, const KParams& kp, int i, int j, int k,
                                           long long c, double q[6], CellMet<R>& M) {
  R src[6];
  cell_sources_at<R, EOS>(b, in, kp, i, j, k, c, src, M);
  constexpr int NQ = EOS ? 6 : 5;
#pragma unroll
  for (int v = 0; v < NQ; ++v) q[v] = accumulate_cell<R>(b, s, ws, kp, i, j, k, c, v, src[v]);
}

// k_update, per interior cell: the stage update and the atmosphere test (Sec. 3.5, App. A).
// Atmosphere cells are reset here (closed form); every other cell is returned as a con2prim job (the
// root find runs in k_c2p on the compacted job list).
// FP64 path: U' of all variables here, left in Uo for k_c2p.
// Mixed path: D has no source, so D' and the atmosphere test need only the fluxes and sqrt(gamma) of
// the FP32 metric (the same band atm_band as the FP64 test); gamma_ij and sqrt(gamma) are the values
// cellmet_from forms, so the test is the one the full metric would give.  The other variables of a
// matter cell are formed in k_c2p (update_all), densely packed, so that this kernel carries neither the
// metric derivatives nor the sources.
template <class R, int EOS>
__device__ __forceinline__ bool update_cell(const Work& w, const DBlock& b, const InView<R>& in,
                                            const StateView& s, const Workspace& ws, const KParams& kp) {
  int p[3];
  if (!decode<R_INTERIOR, 0>(w, b, p)) return false;
  const int i = p[0], j = p[1], k = p[2];
  const long long c = b.cell + cix(b, i, j, k);
  constexpr int NQ = EOS ? 6 : 5;
  double q[6], wn[7];
  if constexpr (sizeof(R) == sizeof(float)) {
    R gv[10];
    cell_metric<R>(b, in, in.order, i, j, k, 4, 10, gv, nullptr);
    const R* gam = gv + 4;
    const R sg = sqrt_r(det3(gam));
    q[0] = accumulate_cell<R>(b, s, ws, kp, i, j, k, c, 0, R(0));
    const double sg32 = to64(sg);
    if (!(finite64(q[0]) && q[0] < kp.rho_thr * sg32)) return true;
    // atmosphere: failed instead if any other variable's update is not finite.  The flux divergence of
    // those variables is finite for certain when the face kernel left the block's flag clear, so their
    // fluxes are read only in a flagged block
    bool finite = true;
    const bool fchk = ws.fbad[w.block] != 0;
#pragma unroll
    for (int v = 1; v < NQ; ++v) {
      if (fchk) {
        const int cv = v < 5 ? v : 7;
        const R* a0 = reinterpret_cast<const R*>(ws.flux[0]) + cv * ws.fstride[0] + b.wface[0] + fix(b, 0, i, j, k);
        const R* a1 = reinterpret_cast<const R*>(ws.flux[1]) + cv * ws.fstride[1] + b.wface[1] + fix(b, 1, i, j, k);
        const R* a2 = reinterpret_cast<const R*>(ws.flux[2]) + cv * ws.fstride[2] + b.wface[2] + fix(b, 2, i, j, k);
        const R t = a0[1] - a0[0] + a1[b.N[0]] - a1[0] + a2[(long long)b.N[0] * b.N[1]] - a2[0];
        finite = finite && isfinite(t);
      }
      finite = finite && finite64(s.U[v][c]);
    }
    mixed_atm_reset<R, EOS>(b, s, kp, i, j, k, c, gam, sg, finite);
    return false;
  } else {
    CellMet<R> M;
    update_all<R, EOS>(b, in, s, ws, kp, i, j, k, c, q, M);
    double Bn[3];
    cell_field(b, s.Bo, i, j, k, Bn);
    // FP64 path: the atmosphere test of con2prim (the same operations, on the same FP64 metric that
    // k_c2p interpolates), decided here for finite cells
    C2PMet Mc;
#pragma unroll
    for (int t = 0; t < 6; ++t) Mc.g[t] = to64(M.g[t]);
    Mc.sg = to64(M.sg);
    Mc.det = to64(M.det);
    bool finite = isfinite(Bn[0]) && isfinite(Bn[1]) && isfinite(Bn[2]);
#pragma unroll
    for (int v = 0; v < NQ; ++v) finite = finite && isfinite(q[v]);
    if (finite && q[0] < kp.rho_thr * Mc.sg) {
      atm_cell<EOS>(Mc, kp, Bn, q, wn);
      write_cell<EOS>(s, c, q, wn, GR_ST_ATM_THRESHOLD);
      return false;
    }
#pragma unroll
    for (int v = 0; v < NQ; ++v) s.Uo[v][c] = q[v];
    return true;
  }
}

// FP32: at most 64 registers (four 256-thread CTAs per SM): the mixed update is bound by load latency
template <class R, int EOS>
__global__ void __launch_bounds__(kMaxTile, sizeof(R) == sizeof(float) ? 4 : 0) k_update(const DBlock* __restrict__ blocks, const Work* __restrict__ work,
                                                     int nwork, const __grid_constant__ InView<R> in,
                                                     const __grid_constant__ StateView s,
                                                     const __grid_constant__ Workspace ws,
                                                     const __grid_constant__ KParams kp) {
  const unsigned lane = threadIdx.x & 31u;
  for (int it = blockIdx.x; it < nwork; it += gridDim.x) {
    const Work w = work[it];
    const bool queued = update_cell<R, EOS>(w, blocks[w.block], in, s, ws, kp);
    // warp-aggregated append to the job list: one atomic per warp, slots by rank among queued lanes
    const unsigned mask = __ballot_sync(0xffffffffu, queued);
    int base = 0;
    if (lane == 0 && mask) base = atomicAdd(ws.njobs, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (queued) ws.jobs[base + __popc(mask & ((1u << lane) - 1u))] = make_int2(w.block, w.start + (int)threadIdx.x);
  }
}

// k_c2p: FP64 con2prim (Sec. 3.5, App. A) of the queued cells, packed densely into warps whatever the
// pattern of atmosphere and matter cells: thread t of the grid takes jobs t, t + grid size, ...
// R = float (the mixed stage): the cell's U' is formed here first (update_all on the FP32 inputs);
// R = double: U' is read from Uo (left there by k_update or by the caller of gr_con2prim).
// FAST: con2prim_cell's mixed-stage form (FP32 bracket search, two-division master function); every
// mixed stage uses it, the fused sweep's k_c2p (R = double) included, so that both paths agree bitwise.
template <int EOS, class R = double, bool FAST = (sizeof(R) == sizeof(float))>
__global__ void __maxnreg__(168) k_c2p(const DBlock* __restrict__ blocks,
                                                  const __grid_constant__ InView<R> in,
                                                  const __grid_constant__ InView<double> in64,
                                                  const __grid_constant__ StateView s,
                                                  const __grid_constant__ Workspace ws,
                                                  const __grid_constant__ KParams kp) {
  const int n = *ws.njobs;
  for (int jdx = blockIdx.x * blockDim.x + threadIdx.x; jdx < n; jdx += gridDim.x * blockDim.x) {
    const int2 job = ws.jobs[jdx];
    const DBlock b = blocks[job.x];
    const int e = job.y;
    const unsigned q0 = udiv_m((unsigned)e, b.mdiv[0][0]), q1 = udiv_m(q0, b.mdiv[1][0]);
    const int i = e - (int)q0 * b.n[0], j = (int)q0 - (int)q1 * b.n[1], k = (int)q1;
    const long long c = b.cell + cix(b, i, j, k);
    constexpr int NQ = EOS ? 6 : 5;
    double q[6], Bn[3], wn[7];
    q[5] = 0.0;
    if constexpr (sizeof(R) == sizeof(float)) {
      CellMet<R> M32;
      update_all<R, EOS>(b, in, s, ws, kp, i, j, k, c, q, M32);
    } else {
#pragma unroll
      for (int v = 0; v < NQ; ++v) q[v] = s.Uo[v][c];
    }
    cell_field(b, s.Bo, i, j, k, Bn);
    C2PMet M;
    cell_gamma64<FAST>(b, in64, i, j, k, M);
    int iters;
    const int st = con2prim_cell<EOS, FAST>(M, kp, q, Bn, wn, &iters);
    write_cell<EOS>(s, c, q, wn, st);
    if (s.evals) s.evals[c] = iters;
  }
}

// ------------------------------------------------------------------------------------------------
// stand-alone prim2con / con2prim / diagnostics (FP64)
// ------------------------------------------------------------------------------------------------
struct P2CArgs {
  const double* W[7];
  const double* B[3];
  double* U[6];
  uint8_t* status;
  int32_t* evals;
};

template <int EOS>
__global__ void __launch_bounds__(kTile) k_prim2con(const DBlock* __restrict__ blocks, const Work* __restrict__ work,
                                                    const __grid_constant__ InView<double> m,
                                                    const __grid_constant__ P2CArgs a,
                                                    const __grid_constant__ KParams kp) {
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  int p[3];
  if (!decode<R_INTERIOR, 0>(w, b, p)) return;
  double val[16];
  cell_metric<double>(b, m, m.order, p[0], p[1], p[2], 0, 10, val, nullptr);
  CellMet<double> M;
  cellmet_from<double>(val, true, M);
  const long long c = b.cell + cix(b, p[0], p[1], p[2]);
  double wv[6], Bd[3], q[6];
  for (int v = 0; v < 5; ++v) wv[v] = a.W[v][c];
  wv[5] = EOS ? a.W[5][c] : 0.0;
  cell_field(b, a.B, p[0], p[1], p[2], Bd);
  CellFluid<double> f;
  cell_fluid<double, EOS>(M, kp, wv, Bd, f);
  cell_cons<double>(M, f, q);
  for (int v = 0; v < 5; ++v) a.U[v][c] = q[v];
  if (EOS) a.U[5][c] = q[0] * wv[5];
}

// gr_con2prim, first pass: atmosphere cells (the threshold test of con2prim on the same FP64 metric)
// are reset in place; every other cell goes to the job list that k_c2p solves densely.
template <int EOS>
__global__ void __launch_bounds__(kTile) k_con2prim_prep(const DBlock* __restrict__ blocks,
                                                         const Work* __restrict__ work,
                                                         const __grid_constant__ InView<double> m,
                                                         const __grid_constant__ StateView s,
                                                         const __grid_constant__ Workspace ws,
                                                         const __grid_constant__ KParams kp) {
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  int p[3];
  bool queued = false;
  if (decode<R_INTERIOR, 0>(w, b, p)) {
    C2PMet M;
    cell_gamma64(b, m, p[0], p[1], p[2], M);
    const long long c = b.cell + cix(b, p[0], p[1], p[2]);
    constexpr int NQ = EOS ? 6 : 5;
    double q[6], Bd[3], wn[7];
    q[5] = 0.0;
    for (int v = 0; v < NQ; ++v) q[v] = s.Uo[v][c];
    cell_field(b, s.Bo, p[0], p[1], p[2], Bd);
    bool finite = isfinite(Bd[0]) && isfinite(Bd[1]) && isfinite(Bd[2]);
    for (int v = 0; v < NQ; ++v) finite = finite && isfinite(q[v]);
    const double rho_thr = kp.rho_thr;
    if (finite && q[0] < rho_thr * M.sg) {
      atm_cell<EOS>(M, kp, Bd, q, wn);
      write_cell<EOS>(s, c, q, wn, GR_ST_ATM_THRESHOLD);
      if (s.evals) s.evals[c] = 0;
    } else {
      queued = true;
    }
  }
  const unsigned lane = threadIdx.x & 31u;
  const unsigned mask = __ballot_sync(0xffffffffu, queued);
  int base = 0;
  if (lane == 0 && mask) base = atomicAdd(ws.njobs, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (queued) ws.jobs[base + __popc(mask & ((1u << lane) - 1u))] = make_int2(w.block, w.start + (int)threadIdx.x);
}

// Training samples of the learned bracket: features and log(mu) of the plain bracketed solve of each
// interior cell (valid = 0 where the cell is not solved: atmosphere, limits, failure)
struct SampleArgs {
  const double* U[6];
  const double* B[3];
  float* feats[kMlpIn];
  float* target;
  uint8_t* valid;
};

template <int EOS>
__global__ void __launch_bounds__(kTile) k_c2p_samples(const DBlock* __restrict__ blocks, const Work* __restrict__ work,
                                                       const __grid_constant__ InView<double> m,
                                                       const __grid_constant__ SampleArgs a,
                                                       const __grid_constant__ KParams kp) {
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  int p[3];
  if (!decode<R_INTERIOR, 0>(w, b, p)) return;
  C2PMet M;
  cell_gamma64(b, m, p[0], p[1], p[2], M);
  const long long c = b.cell + cix(b, p[0], p[1], p[2]);
  constexpr int NQ = EOS ? 6 : 5;
  double q[6], Bd[3], wn[7];
  for (int v = 0; v < NQ; ++v) q[v] = a.U[v][c];
  cell_field(b, a.B, p[0], p[1], p[2], Bd);
  KParams k = kp;
  k.c2p_guess = GR_GUESS_NONE;
  int iters;
  C2PRecord rec;
  const int st = con2prim_cell<EOS>(M, k, q, Bd, wn, &iters, &rec);
  const bool ok = rec.solved && (st & (GR_ST_BD_LIMIT | GR_ST_TAU_FLOOR)) == 0;
  a.valid[c] = ok ? 1 : 0;
  float f[kMlpIn];
  for (int j = 0; j < kMlpIn; ++j) f[j] = 0.f;
  if (ok) {
    c2p_features(rec.q, rec.r2, rec.b2, rec.rb, f);
    f[4] = EOS ? (float)log(rec.D) : 0.f;
    f[5] = EOS ? (float)rec.ye : 0.f;
  }
  for (int j = 0; j < kMlpIn; ++j) a.feats[j][c] = f[j];
  a.target[c] = ok ? (float)log(rec.mu) : 0.f;
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// maximum that keeps a NaN (fmax would drop it and hide a field that has gone NaN)
__device__ __forceinline__ double max_nan(double a, double b) { return (b > a || b != b) ? b : a; }

// out: [0] sum D dV, [1] max |divB|, [2] sum |divB| dV, [3] max |B|, [4] sum dV; a NaN anywhere in B
// reaches [1] - [3] (the bit-pattern atomicMax orders a positive NaN above every finite value)
__global__ void __launch_bounds__(kTile) k_diag(const DBlock* __restrict__ blocks, const Work* __restrict__ work,
                                                const __grid_constant__ P2CArgs a, double* out) {
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  int p[3];
  double md = 0, dv = 0, mdiv = 0, sdiv = 0, mB = 0;
  if (decode<R_INTERIOR, 0>(w, b, p)) {
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
    mB = max_nan(max_nan(max_nan(fabs(bx0), fabs(bx1)), max_nan(fabs(by0), fabs(by1))),
                 max_nan(fabs(bz0), fabs(bz1)));
  }
  for (int o = 16; o > 0; o >>= 1) {
    md += __shfl_down_sync(0xffffffffu, md, o);
    dv += __shfl_down_sync(0xffffffffu, dv, o);
    sdiv += __shfl_down_sync(0xffffffffu, sdiv, o);
    mdiv = max_nan(mdiv, __shfl_down_sync(0xffffffffu, mdiv, o));
    mB = max_nan(mB, __shfl_down_sync(0xffffffffu, mB, o));
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
static InView<double> view64(const MetricView& m, const StateView* s) {
  InView<double> v;
  for (int c = 0; c < 16; ++c) v.M[c] = m.v[c];
  for (int q = 0; q < 6; ++q) v.W[q] = s ? s->W[q] : nullptr;
  for (int d = 0; d < 3; ++d) v.B[d] = s ? s->B[d] : nullptr;
  v.order = m.order;
  v.k_zero = m.k_zero;
  return v;
}

// FP32 inputs of the mixed path: the caller's copies where given (metric->v32, state W32/B32), else the
// mesh's own, which launch_cast fills
static InView<float> view32(const MetricView& m, const StateView& s, const Shadow& sh) {
  InView<float> v;
  for (int c = 0; c < 16; ++c) v.M[c] = m.v32[0] ? m.v32[c] : sh.M[c];
  for (int q = 0; q < 6; ++q) v.W[q] = s.W32[0] ? s.W32[q] : sh.W[q];
  for (int d = 0; d < 3; ++d) v.B[d] = s.W32[0] ? s.B32[d] : sh.B[d];
  v.order = m.order;
  v.k_zero = m.k_zero;
  return v;
}

// the conversions a mixed stage needs: W and B unless the caller gave copies, the metric unless the
// caller gave one or (cast_metric = false) the previous stage on this mesh made it
static cudaError_t launch_cast(const MetricView& m, const StateView& s, const Shadow& sh, int eos,
                               cudaStream_t st, bool cast_metric) {
  CastList L;
  int k = 0;
  const int nw = eos == GR_EOS_TABLE ? 6 : 5;   // rho, u~^i, p[, Y_e]
  if (!s.W32[0]) {
    for (int q = 0; q < nw; ++q) { L.src[k] = s.W[q]; L.dst[k] = sh.W[q]; L.n[k] = sh.ncell; ++k; }
    for (int d = 0; d < 3; ++d) { L.src[k] = s.B[d]; L.dst[k] = sh.B[d]; L.n[k] = sh.nface[d]; ++k; }
  }
  const int ncomp = (cast_metric && !m.v32[0]) ? (m.k_zero ? 10 : 16) : 0;
  for (int c = 0; c < ncomp; ++c) { L.src[k] = m.v[c]; L.dst[k] = sh.M[c]; L.n[k] = sh.nvert; ++k; }
  L.count = k;
  if (k == 0) return cudaSuccess;
  // two 256-thread CTAs per SM and pool, striding over it
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 1;
  dim3 grid(2 * nsm, k);
  k_cast<<<grid, 256, 0, st>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_cast_pool(const double* src, float* dst, long long n, cudaStream_t st) {
  CastList L{};
  L.src[0] = src;
  L.dst[0] = dst;
  L.n[0] = n;
  L.count = 1;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 1;
  k_cast<<<dim3(2 * nsm, 1), 256, 0, st>>>(L);
  return cudaGetLastError();
}

// The mixed stage through the fused sweep: cell prep, k_fused (faces, EMFs, CT, update), con2prim of the
// queued cells from their U' in Uo
static cudaError_t stage_fused(const DBlock* blocks, int nblocks, const KLaunch kl[SK_N], const InView<float>& in,
                               const InView<double>& in64, const StateView& s, const Workspace& ws, const KParams& kp,
                               cudaStream_t st, cudaEvent_t* ev) {
  cudaError_t e = launch_cellprep_sweep<float>(blocks, in, ws, st);
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[2], st);
  e = cudaMemsetAsync(ws.njobs, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  e = launch_fused(blocks, nblocks, in, s, ws, kp, st);
  if (e != cudaSuccess) return e;
  if (ev) {
    for (int k = 3; k <= 6; ++k) cudaEventRecord(ev[k], st);
  }
  const KLaunch& q = kl[SK_C2P];
  if (q.nwork) {
    KLaunch qq = q;
    qq.nwork = (q.nwork + q.threads - 1) / q.threads;
    k_c2p<GR_EOS_IDEAL, double, true><<<stage_grid(k_c2p<GR_EOS_IDEAL, double, true>, qq, 0), q.threads, 0, st>>>(
        blocks, in64, in64, s, ws, kp);
  }
  if (ev) cudaEventRecord(ev[7], st);
  return cudaGetLastError();
}

template <class R, int EOS>
static cudaError_t stage_impl(const DBlock* blocks, const KLaunch kl[SK_N], const InView<R>& in,
                              const InView<double>& in64, const StateView& s, const Workspace& ws, const KParams& kp,
                              cudaStream_t st, cudaEvent_t* ev) {
  const KLaunch& a = kl[SK_CELLPREP];
  if (in.order == 2 && ws.nsweep) {   // the order-2 metric: the z sweep (same results, any launch shape)
    const cudaError_t es = launch_cellprep_sweep<R>(blocks, in, ws, st);
    if (es != cudaSuccess) return es;
  } else if (a.nwork) {
    k_cellprep<R><<<stage_grid(k_cellprep<R>, a, 0), a.threads, 0, st>>>(blocks, a.work, a.nwork, in, ws);
  }
  if (ev) cudaEventRecord(ev[2], st);
  const KLaunch& f = kl[SK_FACES];
  if constexpr (sizeof(R) == sizeof(float)) {   // the per-block flux flags: set for all on a refined mesh
    const cudaError_t eb = cudaMemsetAsync(ws.fbad, ws.nlvl ? 1 : 0, ws.nfbad, st);
    if (eb != cudaSuccess) return eb;
  }
  if constexpr (sizeof(R) == sizeof(float) && EOS == GR_EOS_IDEAL) {
    if (ws.nftiles > 0 && in.order == 2) {   // the tiled face sweep (the host checked that every block qualifies)
      const cudaError_t e = launch_faces_tile(blocks, ws.ftiles, ws.nftiles, in, ws, kp, st);
      if (e != cudaSuccess) return e;
    } else if (f.nwork) {
      const cudaError_t e = launch_faces(f, blocks, in, ws, kp, st);
      if (e != cudaSuccess) return e;
    }
  } else if (f.nwork) {
    const cudaError_t e = launch_faces(f, blocks, in, ws, kp, st);
    if (e != cudaSuccess) return e;
  }
  if (ev) cudaEventRecord(ev[3], st);
  const KLaunch& e = kl[SK_EDGES];
  if (e.nwork) k_edges<R><<<stage_grid(k_edges<R>, e, 0), e.threads, 0, st>>>(blocks, e.work, e.nwork, ws, kp);
  if (ws.nlvl) {   // refined mesh: coarse fluxes and EMFs on level boundaries from the fine ones
    const cudaError_t el = launch_level_fix(sizeof(R) == sizeof(float) ? GR_PREC_MIXED : GR_PREC_FP64, blocks, ws.lvl,
                                            ws.nlvl, ws, EOS == GR_EOS_TABLE, st);
    if (el != cudaSuccess) return el;
  }
  if (ev) cudaEventRecord(ev[4], st);
  const KLaunch& c = kl[SK_CT];
  if (c.nwork) k_ct<R><<<stage_grid(k_ct<R>, c, 0), c.threads, 0, st>>>(blocks, c.work, c.nwork, s, ws, kp);
  if (ev) cudaEventRecord(ev[5], st);
  const KLaunch& u = kl[SK_UPDATE];
  cudaError_t e0 = cudaMemsetAsync(ws.njobs, 0, sizeof(int), st);
  if (e0 != cudaSuccess) return e0;
  if (u.nwork)
    k_update<R, EOS><<<stage_grid(k_update<R, EOS>, u, 0), u.threads, 0, st>>>(blocks, u.work, u.nwork, in, s, ws, kp);
  if (ev) cudaEventRecord(ev[6], st);
  // the job count is known only on the device: one CTA per possible job (the rest exit at once), or
  // a persistent grid that strides over the list
  const KLaunch& q = kl[SK_C2P];
  if (q.nwork) {
    KLaunch qq = q;
    qq.nwork = (q.nwork + q.threads - 1) / q.threads;   // q.nwork = the number of interior cells
    k_c2p<EOS, R><<<stage_grid(k_c2p<EOS, R>, qq, 0), q.threads, 0, st>>>(blocks, in, in64, s, ws, kp);
  }
  if (ev) cudaEventRecord(ev[7], st);
  return cudaGetLastError();
}

cudaError_t launch_stage(int precision, const DBlock* blocks, const KLaunch kl[SK_N], const MetricView& m,
                         const StateView& s, const Workspace& ws, const Shadow& sh, const KParams& kp,
                         cudaStream_t st, cudaEvent_t* ev, bool cast_metric, int nfused) {
  if (ev) cudaEventRecord(ev[0], st);
  const InView<double> in64 = view64(m, &s);
  const bool tab = kp.eos == GR_EOS_TABLE;
  if (precision == GR_PREC_MIXED) {
    cudaError_t e = launch_cast(m, s, sh, kp.eos, st, cast_metric);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], st);
    const InView<float> in32 = view32(m, s, sh);
    if (nfused > 0 && !tab) return stage_fused(blocks, nfused, kl, in32, in64, s, ws, kp, st, ev);
    return tab ? stage_impl<float, GR_EOS_TABLE>(blocks, kl, in32, in64, s, ws, kp, st, ev)
               : stage_impl<float, GR_EOS_IDEAL>(blocks, kl, in32, in64, s, ws, kp, st, ev);
  }
  if (ev) cudaEventRecord(ev[1], st);
  return tab ? stage_impl<double, GR_EOS_TABLE>(blocks, kl, in64, in64, s, ws, kp, st, ev)
             : stage_impl<double, GR_EOS_IDEAL>(blocks, kl, in64, in64, s, ws, kp, st, ev);
}

cudaError_t launch_prim2con(const DBlock* blocks, const Work* work, int nwork, const MetricView& m,
                            const double* const W[7], const double* const B[3], double* const U[6],
                            const KParams& kp, cudaStream_t st) {
  P2CArgs a;
  for (int v = 0; v < 7; ++v) a.W[v] = W[v];
  for (int v = 0; v < 6; ++v) a.U[v] = U[v];
  for (int d = 0; d < 3; ++d) a.B[d] = B[d];
  a.status = nullptr;
  a.evals = nullptr;
  if (!nwork) return cudaSuccess;
  if (kp.eos == GR_EOS_TABLE) k_prim2con<GR_EOS_TABLE><<<nwork, kTile, 0, st>>>(blocks, work, view64(m, nullptr), a, kp);
  else k_prim2con<GR_EOS_IDEAL><<<nwork, kTile, 0, st>>>(blocks, work, view64(m, nullptr), a, kp);
  return cudaGetLastError();
}

cudaError_t launch_con2prim(const DBlock* blocks, const Work* work, int nwork, int ninterior, const MetricView& m,
                            double* const U[6], const double* const B[3], double* const W[7],
                            uint8_t* status, int32_t* evals, const Workspace& ws, const KParams& kp,
                            cudaStream_t st) {
  if (!nwork) return cudaSuccess;
  // in place: the state's outputs are the caller's U, W, status
  StateView s{};
  for (int v = 0; v < 6; ++v) s.Uo[v] = U[v];
  for (int v = 0; v < 7; ++v) s.Wo[v] = W[v];
  for (int d = 0; d < 3; ++d) s.Bo[d] = const_cast<double*>(B[d]);
  s.status = status;
  s.evals = evals;
  cudaError_t e = cudaMemsetAsync(ws.njobs, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const InView<double> in64 = view64(m, nullptr);
  const int grid2 = (ninterior + kTile - 1) / kTile;
  if (kp.eos == GR_EOS_TABLE) {
    k_con2prim_prep<GR_EOS_TABLE><<<nwork, kTile, 0, st>>>(blocks, work, in64, s, ws, kp);
    k_c2p<GR_EOS_TABLE><<<grid2, kTile, 0, st>>>(blocks, in64, in64, s, ws, kp);
  } else {
    k_con2prim_prep<GR_EOS_IDEAL><<<nwork, kTile, 0, st>>>(blocks, work, in64, s, ws, kp);
    k_c2p<GR_EOS_IDEAL><<<grid2, kTile, 0, st>>>(blocks, in64, in64, s, ws, kp);
  }
  return cudaGetLastError();
}

cudaError_t launch_c2p_samples(const DBlock* blocks, const Work* work, int nwork, const MetricView& m,
                               const double* const U[6], const double* const B[3], float* const feats[6],
                               float* target, uint8_t* valid, const KParams& kp, cudaStream_t st) {
  SampleArgs a;
  for (int v = 0; v < 6; ++v) a.U[v] = U[v];
  for (int d = 0; d < 3; ++d) a.B[d] = B[d];
  for (int j = 0; j < kMlpIn; ++j) a.feats[j] = feats[j];
  a.target = target;
  a.valid = valid;
  if (!nwork) return cudaSuccess;
  if (kp.eos == GR_EOS_TABLE)
    k_c2p_samples<GR_EOS_TABLE><<<nwork, kTile, 0, st>>>(blocks, work, view64(m, nullptr), a, kp);
  else k_c2p_samples<GR_EOS_IDEAL><<<nwork, kTile, 0, st>>>(blocks, work, view64(m, nullptr), a, kp);
  return cudaGetLastError();
}

cudaError_t launch_diag(const DBlock* blocks, const Work* work, int nwork, const double* const U[5],
                        const double* const B[3], double* dev_out, cudaStream_t st) {
  P2CArgs a{};
  for (int v = 0; v < 5; ++v) a.U[v] = const_cast<double*>(U[v]);
  for (int d = 0; d < 3; ++d) a.B[d] = B[d];
  a.status = nullptr;
  a.evals = nullptr;
  cudaError_t e = cudaMemsetAsync(dev_out, 0, 8 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  if (nwork) k_diag<<<nwork, kTile, 0, st>>>(blocks, work, a, dev_out);
  return cudaGetLastError();
}

}  // namespace grs
