// internal.h -- declarations shared by the host side (capi.cu) and the kernels (stage_kernels.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <vector>

#include "grstage.h"

namespace grs {

constexpr int kTile = 128;   // elements per work item (threads per CTA) of the stand-alone kernels
// Stage kernels: work items of 64, 128 or 256 elements (one thread each), chosen per kernel
constexpr int kMaxTile = 256;
constexpr int kNumTiles = 3;
constexpr int tile_size(int t) { return 64 << t; }
enum StageKernel { SK_CELLPREP = 0, SK_FACES = 1, SK_EDGES = 2, SK_CT = 3, SK_UPDATE = 4, SK_C2P = 5, SK_N = 6 };
// work region of each stage kernel (Region below); k_c2p works on the job list of k_update
constexpr int kRegionOf[SK_N] = {0, 1, 2, 3, 4, 4};

// Device copy of one block: geometry, caller pool offsets and workspace offsets (in elements).
struct DBlock {
  int n[3];
  int g;
  int N[3];            // n + 2g
  double dx[3];
  double idx[3];       // 1/dx
  long long cell, face[3], vert;         // caller pools
  long long wcell, wface[3], wvert;      // workspace pools
  // quotients by the per-axis element counts n, n + 1, n + 2 and N without integer division (which the
  // compiler turns into conversions on the FP64 pipe): q = floor(e / d) = umulhi(2 e, mdiv) for 32-bit e,
  // mdiv = ceil(2^63 / d)
  unsigned long long mdiv[3][4];
};

__host__ __device__ __forceinline__ unsigned long long mdiv_of(unsigned d) {
  return (0x7FFFFFFFFFFFFFFFull) / d + 1ull;   // ceil(2^63 / d) for d >= 1
}

// One CTA's slice of work: elements [start, start + tile) of region `kind` of block `block`
// in direction `dir` (faces, edges) or 0, tile = the CTA size it was built for.
struct Work {
  int block;
  int dir;
  int start;
  int pad;
};

enum Region { R_CELLS_ALL = 0, R_FACES = 1, R_EDGES = 2, R_CTFACES = 3, R_INTERIOR = 4, R_NREGION = 5 };

// Device views of the caller's pools for one call
struct MetricView {
  const double* v[16];
  int order;
  int k_zero;
  const float* v32[16];   // caller's FP32 copies (mixed path) or nullptr
};
struct StateView {
  const double* U[6];     // [5] = D Y_e (table)
  const double* U0[6];
  const double* B[3];
  const double* B0[3];
  const double* W[7];     // [5] = Y_e, [6] = T (table; T unread)
  double* Uo[6];
  double* Bo[3];
  double* Wo[7];
  uint8_t* status;
  int32_t* evals;         // FP64 master-function evaluations per cell (gr_con2prim), or nullptr
  const float* W32[6];    // caller's FP32 copies of W, B (mixed path) or nullptr
  const float* B32[3];
  float* Wo32[6];         // FP32 copies of Wo, Bo to write (mixed path) or nullptr
  float* Bo32[3];
};
// Stage inputs seen in the arithmetic type R of a kernel: the caller's FP64 pools (R = double) or
// the FP32 copies made by the cast pass (R = float).  Same element indexing as the caller pools.
template <class R>
struct InView {
  const R* W[6];          // rho, u~^i, p[, Y_e]
  const R* B[3];
  const R* M[16];
  int order;
  int k_zero;
};

// FP32 copies of the stage inputs (owned by the mesh), sized to the extent of the caller pools
struct Shadow {
  float* W[6];
  float* B[3];
  float* M[16];
  long long ncell, nface[3], nvert;   // pool extents in elements
};

// k_cellprep sweep (order-2 metric): a TX x TY tile of the x-y cell plane of one block, swept along z;
// txy = TX | TY << 16 with TX <= 32, TX * TY <= kSweepThreads, (TX + 1)(TY + 1) <= kSweepVerts
constexpr int kSweepThreads = 256;
constexpr int kSweepVerts = 344;
struct SweepWork {
  int block, x0, y0, txy;
};

// k_faces_tile: a tile of at most kTY interior rows [j0, j1) of one block, walked along z
constexpr int kTY = 8;
struct FaceTile {
  int block, j0, j1, pad;
};

#ifdef __CUDACC__
// floor(e / d) for 32-bit e from mdiv = mdiv_of(d): exact (e (2^63 / d + eps) / 2^63 exceeds e / d by less
// than 2^33 / 2^63, far below 1 / d)
__device__ __forceinline__ unsigned udiv_m(unsigned e, unsigned long long mdiv) {
  return (unsigned)__umul64hi((unsigned long long)e << 1, mdiv);
}
#endif

// Level-boundary records (same layouts as gr_level_face / gr_level_map)
struct LevelFace {
  int coarse, fine, dir, side, o1, o2;
};
struct LevelMap {
  int coarse, fine, off[3], lo[3], hi[3];
};

// Workspace pools (owned by the mesh)
struct Workspace {
  void* bcc[3];        // undensitised cell-centred field calB^i (cells), FP64 or FP32
  void* ecc[3];        // cell-centred electric field E_m (cells, rings -1..n), FP64 or FP32
  void* flux[3];       // per direction: 8 arrays of face values (FP64 or FP32), stride fstride[d]:
                       // D, S_j, tau, the two induction fluxes, D Y_e
  void* edge[3];       // corner electric field E_m (vertex-indexed), FP64 or FP32
  long long fstride[3];
  long long estride;
  const LevelFace* lvl;   // level-boundary faces whose coarse fluxes / EMFs the stage corrects
  int nlvl;
  const SweepWork* sweep;  // k_cellprep sweep tiles of all blocks (order-2 metric)
  int nsweep;
  int* njobs;          // con2prim job list: cells (block, interior index) that need the root find
  int2* jobs;
  const FaceTile* ftiles;  // tiles of k_faces_tile when the stage computes its fluxes with it, else nftiles 0
  int nftiles;
  // mixed path, one byte per block: cleared before the face fluxes, set to 1 by the face kernels when a
  // flux of S_j, tau or D Y_e of the block is not finite or has |F| summed over them >= kFluxSafe (and set
  // for every block on a refined mesh, whose coarse fluxes the level fix rewrites).  A clear byte lets the
  // atmosphere test skip those fluxes: any six of them then sum to a finite FP32 value.
  uint8_t* fbad;
  int nfbad;
};
// Bound on |F_S1| + |F_S2| + |F_S3| + |F_tau| (+ |F_DYe|) of one face below which six such fluxes of
// one variable, each smaller, add and subtract to a finite FP32 value (6 x 4e37 < 3.4e38)
constexpr float kFluxSafe = 4e37f;

// Device view of an EOS table (Sec. 2.2.1) in precision R: node arrays of log p, log e, c_s^2, node
// (ir, iT, iy) at (iy * n[1] + iT) * n[0] + ir; uniform axes log rho, log T, Y_e.
template <class R>
struct TabView {
  const R* f[3];      // log p, log e, c_s^2
  int n[3];
  R x0[3], dx[3], idx[3], hi[3];   // first node, spacing, 1/spacing, last node of each axis
};

enum { RK_G0 = 1, RK_G1 = 2 };   // bits of KParams::rk_form

struct KParams {   // gr_params flattened for the device
  int recon, emf, ceiling, max_iter, c2p_guess, eos;
  double gamma_ad, rho_atm, p_atm, f_thr, W_max, M_max, tol, weno_eps;
  float gamma_f;      // gamma_ad rounded to FP32 once on the host (an FP64 -> FP32 conversion on the device
                      // would run on the narrow FP64 pipe in every FP32 face evaluation)
  // con2prim constants formed once on the host: the velocity cap v_max^2 = 1 - 1/W_max^2, the bracket top
  // 1/h0 and h0^2, in FP64 and (for the FP32 pre-solve) FP32
  double vmax2, top, h0sq;
  float vmax2_f, top_f, h0sq_f;
  double rk_g0, rk_g1, rk_beta;
  int rk_form;        // RK_G0 | RK_G1: which of rk_g0 != 0, rk_g1 != 1 hold (set on the host)
  double rho_thr;     // atmosphere threshold f_thr rho_atm (1 + atm_band): within the band counts as reached
  double dt;
  double bdt;         // rk_beta dt
  const double* dt_dev;   // dt on the device (the RK driver's CFL reduction), or nullptr: use dt
  const float* mlp;   // learned-bracket parameters (GR_GUESS_MLP) or nullptr
  // tabulated EOS: atmosphere (rho_atm, T_atm, Ye_atm) with p_atm and eint_atm precomputed from the
  // table, and the FP64 / FP32 node arrays
  double T_atm, Ye_atm;
  double eint_atm;    // internal energy density rho eps of the atmosphere (ideal: p_atm/(Gamma - 1))
  double h0;          // minimum enthalpy of the EOS (1 for the ideal gas)
  TabView<double> t64;
  TabView<float> t32;
};

// Launch of one stage kernel: its work list (built for CTAs of `threads`), and whether the grid is
// persistent (as many CTAs as fit on the device, striding over the list) or one CTA per work item.
// For k_c2p, work is unused and nwork is the number of interior cells (the job list's capacity).
struct KLaunch {
  const Work* work;
  int nwork;
  int threads;
  int persistent;
};

// k_faces launchers (faces_f32.cu, faces_f64.cu): one instantiation per EOS and reconstruction method
cudaError_t launch_faces(const KLaunch& f, const DBlock* blocks, const InView<float>& in, const Workspace& ws,
                         const KParams& kp, cudaStream_t st);
cudaError_t launch_faces(const KLaunch& f, const DBlock* blocks, const InView<double>& in, const Workspace& ws,
                         const KParams& kp, cudaStream_t st);

// Fused sweep of the mixed path (fused.cu): faces, corner EMFs, CT and the update of every block in one
// launch (one CTA per block); the blocks must satisfy fused_block_ok (ghost width 3, at most 16 x 16 cells
// in x-y), the EOS be the ideal gas and the metric of order 2.
cudaError_t launch_fused(const DBlock* blocks, int nblocks, const InView<float>& in, const StateView& s,
                         const Workspace& ws, const KParams& kp, cudaStream_t st);
bool fused_block_ok(const DBlock& b);
// Face fluxes of the mixed path by k_faces_tile (faces_tile.cu): stencils and metric staged in shared
// memory per tile of a block; blocks with 3 ghosts and at most 16 cells along x, ideal gas, order-2 metric.
cudaError_t launch_faces_tile(const DBlock* blocks, const FaceTile* tiles, int ntiles, const InView<float>& in,
                              const Workspace& ws, const KParams& kp, cudaStream_t st);

// Launchers (stage_kernels.cu).  Each returns the cudaError_t of its launch.
// ev: nullptr, or GR_NKERNELS + 1 events recorded before the input cast (mixed path) and after
// the cast and each kernel.  cast_metric = false reuses the FP32 metric shadow of the previous mixed
// stage on this mesh (the RK driver, whose stages share one metric).
// nfused > 0: the mixed path through the fused sweep over nfused blocks (the caller checked that it applies).
cudaError_t launch_stage(int precision, const DBlock* blocks, const KLaunch kl[SK_N], const MetricView& m,
                         const StateView& s, const Workspace& ws, const Shadow& sh, const KParams& kp,
                         cudaStream_t st, cudaEvent_t* ev, bool cast_metric = true, int nfused = 0);
cudaError_t launch_prim2con(const DBlock* blocks, const Work* work, int nwork, const MetricView& m,
                            const double* const W[7], const double* const B[3], double* const U[6],
                            const KParams& kp, cudaStream_t st);
cudaError_t launch_con2prim(const DBlock* blocks, const Work* work, int nwork, int ninterior, const MetricView& m,
                            double* const U[6], const double* const B[3], double* const W[7],
                            uint8_t* status, int32_t* evals, const Workspace& ws, const KParams& kp,
                            cudaStream_t st);
cudaError_t launch_c2p_samples(const DBlock* blocks, const Work* work, int nwork, const MetricView& m,
                               const double* const U[6], const double* const B[3], float* const feats[6],
                               float* target, uint8_t* valid, const KParams& kp, cudaStream_t st);
// FP32 copy of one FP64 pool by the mixed path's input conversion (d2f_rn)
cudaError_t launch_cast_pool(const double* src, float* dst, long long n, cudaStream_t st);
// RK driver (driver.cu): ghost exchange between same-level blocks, CFL dt on the device
cudaError_t launch_level_fix(int precision, const DBlock* blocks, const LevelFace* lf, int nlf, const Workspace& ws,
                             int table, cudaStream_t st);
cudaError_t launch_amr(bool prolong, const DBlock* blocks, const LevelMap* maps, const Work* work, int nwork,
                       double* const cells[8], int nvar, double* const B[3], cudaStream_t st);
// gr_host_stage transfers of interior cells / faces of interior cells (pinned, device-mapped host memory)
cudaError_t launch_io_cells(const DBlock* blocks, const Work* work, int nwork, const void* const* src, void* const* dst,
                            int n, int elem, cudaStream_t st);
cudaError_t launch_io_faces(const DBlock* blocks, const Work* work, int nwork, const double* const src[3],
                            double* const dst[3], cudaStream_t st);
constexpr int kAdmThreads = 256;
constexpr size_t kAdmSmemTarget = 96 * 1024;    // shared memory a k_adm_verts slab aims for
constexpr size_t kAdmSmemMax = 200 * 1024;      // ... and may not exceed (one vertex plane)
size_t adm_smem_bytes(const int n[3], int Z, int np, size_t elem);
cudaError_t launch_adm(int precision, const DBlock* blocks, const Work* cw, int ncw, const Work* vw, int nvw,
                       size_t smem, const MetricView& m, const double* const W[7], const double* const B[3],
                       const KParams& kp, int vc_order, void* const cv[10], double* const out[10], cudaStream_t st);
constexpr int kGhostTile = 256;
// Gather map of the same-level ghost fill, made once per distinct block shape (n, g) when the driver is
// made: for element e of the ghost shell of a block of that shape and element kind (cells, x-, y-,
// z-faces; shell order of shell_decode), ent[e] = {destination offset within the block's pool segment,
// (neighbour slot << 27) | source offset within the neighbour's segment} and out[e] = the source offset
// within the block itself when that neighbour is an outflow boundary.  off[block] = the entry offsets of
// the block's shape for the four kinds.
struct GhostMap {
  const int2* ent;
  const int* out;
  const int4* off;
};
constexpr long long kGhostMapMaxLocal = 1ll << 27;   // local offsets must fit 27 bits
// host: the map of a mesh's blocks (entries of equal shapes shared); 0, or -1 when a block's padded arrays
// hold kGhostMapMaxLocal elements or more
int build_ghost_map(const DBlock* hb, int nblocks, std::vector<int2>& ent, std::vector<int>& out,
                    std::vector<int4>& off);
// W32/B32 (optional): FP32 copies of W (up to 6 pools) and B whose ghosts get the converted copied values
cudaError_t launch_ghost_fill(const DBlock* blocks, int nblocks, const int* nbr, const GhostMap& gm,
                              double* const W[7], int nw, double* const B[3], cudaStream_t st,
                              float* const* W32 = nullptr, float* const* B32 = nullptr);
cudaError_t launch_cfl_dt(const DBlock* blocks, const Work* wi, int nwi, const MetricView& m,
                          const double* const W[7], const double* const B[3], const KParams& kp, double cfl,
                          double* rate, double* dt, cudaStream_t st);
cudaError_t launch_set_scalar(double* dst, double value, cudaStream_t st);
cudaError_t launch_diag(const DBlock* blocks, const Work* work, int nwork, const double* const U[5],
                        const double* const B[3], double* dev_out /* 4 + scratch */, cudaStream_t st);

}  // namespace grs
