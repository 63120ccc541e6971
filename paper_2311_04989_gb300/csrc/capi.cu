// capi.cu -- host side of the C ABI declared in include/grstage.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

using namespace grs;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(GR_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// region element counts on the host (mirror of the device decoder)
long long region_count(int kind, int dir, const DBlock& b) {
  long long c = 1;
  for (int a = 0; a < 3; ++a) {
    long long n;
    switch (kind) {
      case R_CELLS_ALL: n = b.N[a]; break;
      case R_FACES: n = (a == dir) ? b.n[a] + 1 : b.n[a] + 2; break;
      case R_EDGES: n = (a == dir) ? b.n[a] : b.n[a] + 1; break;
      case R_CTFACES: n = (a == dir) ? b.n[a] + 1 : b.n[a]; break;
      default: n = b.n[a]; break;
    }
    c *= n;
  }
  return c;
}
bool region_has_dir(int kind) {
  return kind == R_FACES || kind == R_EDGES || kind == R_CTFACES;
}

}  // namespace

struct gr_ctx {
  int device;
};

// Device copy of an EOS table (node arrays of log(p/rho), log(e/rho) = log(1 + eps) and c_s^2 in FP64
// and FP32) and a host copy of the FP64 arrays for per-call constants (the atmosphere state)
struct gr_eos {
  int device;
  int n[3];
  double x0[3], dx[3], hi[3];
  double h0;
  double* d64[3] = {nullptr, nullptr, nullptr};
  float* d32[3] = {nullptr, nullptr, nullptr};
  std::vector<double> host[3];
  int64_t bytes = 0;
};

namespace {
// trilinear interpolant of a host node array at (log rho, log T, Y_e), each moved into the table
double host_tri(const gr_eos& t, int f, const double x[3]) {
  int i[3];
  double w[3];
  for (int a = 0; a < 3; ++a) {
    const double xc = std::min(std::max(x[a], t.x0[a]), t.hi[a]);
    const double sx = (xc - t.x0[a]) / t.dx[a];
    i[a] = std::min((int)sx, t.n[a] - 2);
    w[a] = sx - i[a];
  }
  double s = 0;
  for (int c = 0; c < 8; ++c) {
    const int a = c & 1, b = (c >> 1) & 1, e = (c >> 2) & 1;
    const double wt = (a ? w[0] : 1 - w[0]) * (b ? w[1] : 1 - w[1]) * (e ? w[2] : 1 - w[2]);
    s += wt * t.host[f][((size_t)(i[2] + e) * t.n[1] + (i[1] + b)) * t.n[0] + (i[0] + a)];
  }
  return s;
}
template <class R>
TabView<R> tab_view(const gr_eos& t, R* const* d) {
  TabView<R> v;
  for (int f = 0; f < 3; ++f) v.f[f] = d[f];
  for (int a = 0; a < 3; ++a) {
    v.n[a] = t.n[a];
    v.x0[a] = (R)t.x0[a];
    v.dx[a] = (R)t.dx[a];
    v.idx[a] = (R)(1.0 / t.dx[a]);
    v.hi[a] = (R)t.hi[a];
  }
  return v;
}
}  // namespace

struct HostStage;
static void host_stage_free(HostStage* h);

struct gr_mesh {
  gr_ctx* ctx = nullptr;
  int nblocks = 0;
  int max_ng = 0;
  std::vector<DBlock> h_blocks;
  DBlock* d_blocks = nullptr;
  Work* d_work[R_NREGION] = {};      // work lists of the stand-alone kernels (kTile, direction-major)
  int nwork[R_NREGION] = {};
  // work lists of the stage kernels per CTA size and order (0 direction-major, 1 block-major)
  Work* tw[kNumTiles][2][R_NREGION] = {};
  int tn[kNumTiles][2][R_NREGION] = {};
  // launch shape of each stage kernel per (precision, EOS), set by gr_autotune or gr_mesh_set_shapes
  gr_shape shapes[2][2][SK_N];
  // path of the mixed stage with the ideal gas and the order-2 metric (GR_PATH_*: set by gr_autotune where
  // faster, or by gr_mesh_set_path): the fused sweep where every block qualifies (fused_ok), the tiled face
  // sweep where every block qualifies (tiles_ok; its tile list d_ftiles)
  bool fused_ok = false;
  bool tiles_ok = false;
  int path = GR_PATH_SEPARATE;
  // what GR_GUESS_AUTO stands for per (precision, EOS): set by gr_autotune
  int guess[2][2] = {{GR_GUESS_NONE, GR_GUESS_NONE}, {GR_GUESS_NONE, GR_GUESS_NONE}};
  FaceTile* d_ftiles = nullptr;
  int nftiles = 0;
  int nint = 0;   // interior cells of all blocks
  Workspace ws{};
  Shadow sh{};
  double* d_diag = nullptr;
  std::vector<void*> allocs;
  int64_t ws_bytes = 0;
  int min_ng = 0;
  // gr_host_stage: staging pools, batch sub-meshes, streams (made on first use)
  struct HostStage* hs = nullptr;
  // level boundaries (gr_mesh_set_levels): level faces for the stage, restriction / prolongation maps
  // with their work lists (cell items first: ncw_* of them)
  LevelFace* d_lvl = nullptr;
  LevelMap* d_rmap = nullptr;
  LevelMap* d_pmap = nullptr;
  Work* d_rwork = nullptr;
  Work* d_pwork = nullptr;
  int nrwork = 0, npwork = 0, ncw_r = 0, ncw_p = 0;
  std::vector<void*> lvl_allocs;
  // matter-source outputs (gr_adm_sources): cell-layout workspace (FP64-sized) and work lists per
  // (precision, order 2 / 4), made on first use
  void* adm_cv[10] = {};
  Work* adm_cw[2][2] = {};
  int adm_ncw[2][2] = {};
  Work* adm_vw[2][2] = {};
  int adm_nvw[2][2] = {};
  size_t adm_smem[2][2] = {};
  bool adm_ready[2][2] = {};
  // profiling: (GR_NKERNELS + 1) events per armed stage
  std::vector<cudaEvent_t> prof_events;
  int prof_capacity = 0;
  int prof_used = 0;
};

extern "C" {

const char* gr_strerror(int code) {
  switch (code) {
    case GR_OK: return "ok";
    case GR_EINVAL: return "invalid argument";
    case GR_ECUDA: return "CUDA error";
    case GR_ENOMEM: return "out of device memory";
    case GR_ETIMEOUT: return "bounded device wait expired";
    case GR_EUNSUPPORTED: return "unsupported option";
    default: return "unknown error";
  }
}

const char* gr_last_error(void) { return g_last_error.c_str(); }

int gr_abi_version(void) { return GR_ABI_VERSION; }

void gr_params_default(gr_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->size = sizeof(gr_params);
  p->recon = GR_RECON_WENOZ;
  p->precision = GR_PREC_FP64;
  p->emf = GR_EMF_UPWIND;
  p->ceiling = GR_CEIL_CLAMP;
  p->max_iter = 100;
  p->c2p_guess = GR_GUESS_NONE;
  p->gamma_ad = 2.0;
  p->rho_atm = 1e-13;
  p->p_atm = 100.0 * 1e-26;
  p->f_thr = 1.0;
  p->W_max = std::sqrt(1.0 + 400.0);
  p->M_max = 1e4;
  p->tol = 1e-10;
  p->weno_eps = 1e-40;
  p->rk_g0 = 0.0;
  p->rk_g1 = 1.0;
  p->rk_beta = 1.0;
  p->atm_band = 1e-12;
}

int gr_context_create(gr_ctx** ctx, int device) {
  if (!ctx) return fail(GR_EINVAL, "gr_context_create: ctx is NULL");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(GR_EINVAL, "gr_context_create: bad device index");
  DeviceGuard g(device);
  e = cudaFree(nullptr);   // establish the primary context
  if (e != cudaSuccess) return cuda_fail(e, "cudaFree(0)");
  *ctx = new gr_ctx{device};
  return GR_OK;
}

int gr_context_destroy(gr_ctx* ctx) {
  delete ctx;
  return GR_OK;
}

static void prof_release(gr_mesh* m) {
  for (cudaEvent_t e : m->prof_events) cudaEventDestroy(e);
  m->prof_events.clear();
  m->prof_capacity = m->prof_used = 0;
}

static void levels_free(gr_mesh* m) {
  for (void* p : m->lvl_allocs) cudaFree(p);
  m->lvl_allocs.clear();
  m->d_lvl = nullptr;
  m->d_rmap = m->d_pmap = nullptr;
  m->d_rwork = m->d_pwork = nullptr;
  m->nrwork = m->npwork = m->ncw_r = m->ncw_p = 0;
  m->ws.lvl = nullptr;
  m->ws.nlvl = 0;
}

static void mesh_free(gr_mesh* m) {
  if (!m) return;
  DeviceGuard g(m->ctx ? m->ctx->device : 0);
  prof_release(m);
  levels_free(m);
  host_stage_free(m->hs);
  m->hs = nullptr;
  for (void* p : m->allocs) cudaFree(p);
  delete m;
}

int gr_profile_begin(gr_mesh* mesh, int32_t max_stages) {
  if (!mesh || max_stages < 1 || max_stages > 100000) return fail(GR_EINVAL, "gr_profile_begin: bad argument");
  DeviceGuard g(mesh->ctx->device);
  prof_release(mesh);
  const int ne = (GR_NKERNELS + 1) * max_stages;
  mesh->prof_events.resize(ne);
  for (int i = 0; i < ne; ++i) {
    cudaError_t e = cudaEventCreate(&mesh->prof_events[i]);
    if (e != cudaSuccess) {
      mesh->prof_events.resize(i);
      prof_release(mesh);
      return cuda_fail(e, "cudaEventCreate");
    }
  }
  mesh->prof_capacity = max_stages;
  mesh->prof_used = 0;
  return GR_OK;
}

int gr_profile_end(gr_mesh* mesh, double* ms, int32_t* nstages) {
  if (!mesh || !ms || !nstages) return fail(GR_EINVAL, "gr_profile_end: NULL argument");
  DeviceGuard g(mesh->ctx->device);
  for (int k = 0; k < GR_NKERNELS; ++k) ms[k] = 0.0;
  *nstages = mesh->prof_used;
  for (int s = 0; s < mesh->prof_used; ++s) {
    cudaEvent_t* ev = &mesh->prof_events[(GR_NKERNELS + 1) * s];
    cudaError_t e = cudaEventSynchronize(ev[GR_NKERNELS]);
    if (e != cudaSuccess) { prof_release(mesh); return cuda_fail(e, "cudaEventSynchronize"); }
    for (int k = 0; k < GR_NKERNELS; ++k) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      if (e != cudaSuccess) { prof_release(mesh); return cuda_fail(e, "cudaEventElapsedTime"); }
      ms[k] += t;
    }
  }
  prof_release(mesh);
  return GR_OK;
}

int gr_mesh_destroy(gr_mesh* mesh) {
  mesh_free(mesh);
  return GR_OK;
}

int64_t gr_mesh_workspace_bytes(const gr_mesh* mesh) { return mesh ? mesh->ws_bytes : -1; }

int gr_mesh_create(gr_ctx* ctx, const gr_block* blocks, int32_t nblocks, int32_t max_ng, gr_mesh** out) {
  (void)max_ng;
  if (!ctx || !out) return fail(GR_EINVAL, "gr_mesh_create: NULL argument");
  if (nblocks < 0 || (nblocks > 0 && !blocks)) return fail(GR_EINVAL, "gr_mesh_create: bad block list");
  DeviceGuard g(ctx->device);
  gr_mesh* m = new gr_mesh();
  m->ctx = ctx;
  m->nblocks = nblocks;
  m->h_blocks.resize(nblocks);
  long long wcell = 0, wface[3] = {0, 0, 0}, wvert = 0;
  m->min_ng = 1 << 30;
  for (int b = 0; b < nblocks; ++b) {
    const gr_block& s = blocks[b];
    DBlock& d = m->h_blocks[b];
    if (s.ng < 1 || s.ng > 8) { mesh_free(m); return fail(GR_EINVAL, "gr_mesh_create: ng must be in [1, 8]"); }
    for (int a = 0; a < 3; ++a) {
      if (s.n[a] < 1 || s.n[a] > 1024) { mesh_free(m); return fail(GR_EINVAL, "gr_mesh_create: n out of range"); }
      if (!(s.dx[a] > 0) || !std::isfinite(s.dx[a])) { mesh_free(m); return fail(GR_EINVAL, "gr_mesh_create: dx must be positive"); }
      d.n[a] = s.n[a];
      d.N[a] = s.n[a] + 2 * s.ng;
      d.dx[a] = s.dx[a];
      d.idx[a] = 1.0 / s.dx[a];
      for (int k = 0; k < 3; ++k) d.mdiv[a][k] = mdiv_of((unsigned)(s.n[a] + k));
      d.mdiv[a][3] = mdiv_of((unsigned)d.N[a]);
    }
    if (s.cell_off < 0 || s.vert_off < 0 || s.face_off[0] < 0 || s.face_off[1] < 0 || s.face_off[2] < 0) {
      mesh_free(m);
      return fail(GR_EINVAL, "gr_mesh_create: negative pool offset");
    }
    d.g = s.ng;
    m->min_ng = std::min(m->min_ng, (int)s.ng);
    m->max_ng = std::max(m->max_ng, (int)s.ng);
    d.cell = s.cell_off;
    d.vert = s.vert_off;
    for (int a = 0; a < 3; ++a) d.face[a] = s.face_off[a];
    const long long nc = (long long)d.N[0] * d.N[1] * d.N[2];
    d.wcell = wcell;
    wcell += nc;
    for (int a = 0; a < 3; ++a) {
      d.wface[a] = wface[a];
      wface[a] += (long long)(d.N[0] + (a == 0)) * (d.N[1] + (a == 1)) * (d.N[2] + (a == 2));
    }
    d.wvert = wvert;
    wvert += (long long)(d.N[0] + 1) * (d.N[1] + 1) * (d.N[2] + 1);
  }
  // work lists for every CTA size and order.  Direction-major lists keep the CTAs resident on an SM
  // at any time mostly in the same per-direction instantiation (the three bodies would otherwise
  // share the I-cache); block-major lists keep a block's data together in L2.
  std::vector<Work> wl[kNumTiles][2][R_NREGION];
  for (int t = 0; t < kNumTiles; ++t)
    for (int order = 0; order < 2; ++order)
      for (int kind = 0; kind < R_NREGION; ++kind) {
        if (order == 1 && !region_has_dir(kind)) continue;   // same list as order 0
        const int ndir = region_has_dir(kind) ? 3 : 1;
        const int tile = tile_size(t);
        std::vector<Work>& L = wl[t][order][kind];
        for (int o1 = 0; o1 < (order == 0 ? ndir : nblocks); ++o1)
          for (int o2 = 0; o2 < (order == 0 ? nblocks : ndir); ++o2) {
            const int dir = order == 0 ? o1 : o2, b = order == 0 ? o2 : o1;
            const long long cnt = region_count(kind, dir, m->h_blocks[b]);
            for (long long s0 = 0; s0 < cnt; s0 += tile) L.push_back(Work{b, dir, (int)s0, 0});
          }
      }
  const int t128 = 1;   // tile_size(1) == kTile
  static_assert(tile_size(1) == kTile, "stand-alone kernels use the 128-element lists");
  for (int kind = 0; kind < R_NREGION; ++kind) m->nwork[kind] = (int)wl[t128][0][kind].size();
  for (int pr = 0; pr < 2; ++pr)
    for (int eo = 0; eo < 2; ++eo)
      for (int k = 0; k < SK_N; ++k) m->shapes[pr][eo][k] = gr_shape{kTile, 0, 0};
  auto dalloc = [&](size_t bytes, void** p) -> cudaError_t {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e == cudaSuccess) { m->allocs.push_back(*p); m->ws_bytes += (int64_t)bytes; }
    return e;
  };
  cudaError_t e = cudaSuccess;
  e = dalloc(sizeof(DBlock) * std::max(1, nblocks), (void**)&m->d_blocks);
  if (e == cudaSuccess && nblocks)
    e = cudaMemcpy(m->d_blocks, m->h_blocks.data(), sizeof(DBlock) * nblocks, cudaMemcpyHostToDevice);
  for (int t = 0; t < kNumTiles; ++t)
    for (int order = 0; order < 2; ++order)
      for (int kind = 0; kind < R_NREGION && e == cudaSuccess; ++kind) {
        if (order == 1 && !region_has_dir(kind)) {
          m->tw[t][1][kind] = m->tw[t][0][kind];
          m->tn[t][1][kind] = m->tn[t][0][kind];
          continue;
        }
        const std::vector<Work>& L = wl[t][order][kind];
        e = dalloc(sizeof(Work) * std::max<size_t>(1, L.size()), (void**)&m->tw[t][order][kind]);
        if (e == cudaSuccess && !L.empty())
          e = cudaMemcpy(m->tw[t][order][kind], L.data(), sizeof(Work) * L.size(), cudaMemcpyHostToDevice);
        m->tn[t][order][kind] = (int)L.size();
      }
  for (int kind = 0; kind < R_NREGION; ++kind) m->d_work[kind] = m->tw[t128][0][kind];
  // k_cellprep sweep tiles: the x-y cell plane of each block in tiles of TX <= 32 columns (equal
  // shares of N0) by TY = kSweepThreads / TX rows
  std::vector<SweepWork> sw;
  for (int b = 0; b < nblocks; ++b) {
    const DBlock& d = m->h_blocks[b];
    const int nxt = (d.N[0] + 31) / 32;
    const int TX = (d.N[0] + nxt - 1) / nxt, TY = kSweepThreads / TX;
    if ((TX + 1) * (TY + 1) > kSweepVerts) { e = cudaErrorInvalidValue; break; }
    for (int y0 = 0; y0 < d.N[1]; y0 += TY)
      for (int x0 = 0; x0 < d.N[0]; x0 += TX) sw.push_back(SweepWork{b, x0, y0, TX | (TY << 16)});
  }
  if (e == cudaSuccess) e = dalloc(sizeof(SweepWork) * std::max<size_t>(1, sw.size()), (void**)&m->ws.sweep);
  if (e == cudaSuccess && !sw.empty())
    e = cudaMemcpy((void*)m->ws.sweep, sw.data(), sizeof(SweepWork) * sw.size(), cudaMemcpyHostToDevice);
  m->ws.nsweep = (int)sw.size();
  for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
    e = dalloc(sizeof(double) * wcell, &m->ws.bcc[a]);
    if (e == cudaSuccess) e = dalloc(sizeof(double) * wcell, &m->ws.ecc[a]);
    if (e == cudaSuccess) e = dalloc(sizeof(double) * 8 * wface[a], &m->ws.flux[a]);
    if (e == cudaSuccess) e = dalloc(sizeof(double) * wvert, &m->ws.edge[a]);
    m->ws.fstride[a] = wface[a];
  }
  m->ws.estride = wvert;
  // FP32 copies of the stage inputs for the mixed path, covering the extent of the caller pools
  long long ec = 0, ef[3] = {0, 0, 0}, ev = 0;
  for (const DBlock& d : m->h_blocks) {
    ec = std::max(ec, d.cell + (long long)d.N[0] * d.N[1] * d.N[2]);
    for (int a = 0; a < 3; ++a)
      ef[a] = std::max(ef[a], d.face[a] + (long long)(d.N[0] + (a == 0)) * (d.N[1] + (a == 1)) * (d.N[2] + (a == 2)));
    ev = std::max(ev, d.vert + (long long)(d.N[0] + 1) * (d.N[1] + 1) * (d.N[2] + 1));
  }
  m->sh.ncell = ec; m->sh.nvert = ev;
  for (int a = 0; a < 3; ++a) m->sh.nface[a] = ef[a];
  for (int v = 0; v < 6 && e == cudaSuccess; ++v) e = dalloc(sizeof(float) * ec, (void**)&m->sh.W[v]);
  for (int a = 0; a < 3 && e == cudaSuccess; ++a) e = dalloc(sizeof(float) * ef[a], (void**)&m->sh.B[a]);
  for (int c = 0; c < 16 && e == cudaSuccess; ++c) e = dalloc(sizeof(float) * ev, (void**)&m->sh.M[c]);
  if (e == cudaSuccess) e = dalloc(sizeof(double) * 8, (void**)&m->d_diag);
  long long nint = 0;
  for (const DBlock& d : m->h_blocks) nint += (long long)d.n[0] * d.n[1] * d.n[2];
  if (nint > (1LL << 31) - 1024) e = cudaErrorInvalidValue;
  m->nint = (int)nint;
  m->fused_ok = nblocks > 0;
  for (const DBlock& d : m->h_blocks) m->fused_ok = m->fused_ok && fused_block_ok(d);
  // tiles of the face sweep: rows of each block in equal tiles of at most kTY (3 ghosts, <= 16 cells along x)
  m->tiles_ok = nblocks > 0;
  for (const DBlock& d : m->h_blocks) m->tiles_ok = m->tiles_ok && d.g == 3 && d.n[0] <= 16;
  if (m->tiles_ok && e == cudaSuccess) {
    std::vector<FaceTile> ft;
    for (int b = 0; b < nblocks; ++b) {
      const int n1 = m->h_blocks[b].n[1];
      const int nt = (n1 + kTY - 1) / kTY;
      for (int t = 0; t < nt; ++t) ft.push_back(FaceTile{b, (int)((long long)n1 * t / nt), (int)((long long)n1 * (t + 1) / nt), 0});
    }
    e = dalloc(sizeof(FaceTile) * ft.size(), (void**)&m->d_ftiles);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_ftiles, ft.data(), sizeof(FaceTile) * ft.size(), cudaMemcpyHostToDevice);
    m->nftiles = (int)ft.size();
  }
  if (e == cudaSuccess) e = dalloc(sizeof(int2) * std::max<long long>(1, nint), (void**)&m->ws.jobs);
  if (e == cudaSuccess) e = dalloc(sizeof(int) * 4, (void**)&m->ws.njobs);
  if (e == cudaSuccess) e = dalloc(std::max(1, nblocks), (void**)&m->ws.fbad);
  if (e == cudaSuccess) e = cudaMemset(m->ws.fbad, 1, std::max(1, nblocks));
  m->ws.nfbad = nblocks;
  if (e != cudaSuccess) {
    const int code = (e == cudaErrorMemoryAllocation) ? GR_ENOMEM : GR_ECUDA;
    std::string msg = std::string("gr_mesh_create: ") + cudaGetErrorString(e);
    cudaGetLastError();
    mesh_free(m);
    return fail(code, msg);
  }
  *out = m;
  return GR_OK;
}

// the per-block flux flag of the mixed stage relies on this: six fluxes of one variable, each below the
// bound, add and subtract to a finite FP32 value
static_assert(6.0 * kFluxSafe < 3.4e38, "kFluxSafe too large for the flux flag");

static int check_params(const gr_params* p) {
  if (!p) return fail(GR_EINVAL, "params is NULL");
  if (p->size != sizeof(gr_params)) return fail(GR_EINVAL, "gr_params.size does not match this library");
  if (p->recon < GR_RECON_PLM || p->recon > GR_RECON_PPM) return fail(GR_EINVAL, "bad recon");
  if (p->precision != GR_PREC_FP64 && p->precision != GR_PREC_MIXED) return fail(GR_EINVAL, "bad precision");
  if (p->emf != GR_EMF_UPWIND && p->emf != GR_EMF_MEAN) return fail(GR_EINVAL, "bad emf");
  if (p->ceiling != GR_CEIL_CLAMP && p->ceiling != GR_CEIL_ATMOSPHERE) return fail(GR_EINVAL, "bad ceiling");
  if (p->max_iter < 1 || p->max_iter > 10000) return fail(GR_EINVAL, "max_iter out of range");
  if (p->c2p_guess != GR_GUESS_NONE && p->c2p_guess != GR_GUESS_FP32 && p->c2p_guess != GR_GUESS_MLP &&
      p->c2p_guess != GR_GUESS_AUTO)
    return fail(GR_EINVAL, "bad c2p_guess");
  if (p->c2p_guess == GR_GUESS_MLP && (!p->mlp || (((uintptr_t)p->mlp) & 15u)))
    return fail(GR_EINVAL, "GR_GUESS_MLP needs a 16-byte aligned device parameter vector in params.mlp");
  if (!(p->gamma_ad > 1.0) || !(p->W_max >= 1.0) || !(p->M_max > 0) || !(p->tol > 0) ||
      !(p->rho_atm >= 0) || !(p->p_atm >= 0) || !(p->f_thr >= 0) || !(p->weno_eps > 0) ||
      !(p->atm_band >= 0 && p->atm_band <= 1e-3))
    return fail(GR_EINVAL, "physical parameter out of range");
  if (p->eos != GR_EOS_IDEAL && p->eos != GR_EOS_TABLE) return fail(GR_EINVAL, "bad eos");
  if (p->eos == GR_EOS_TABLE) {
    if (!p->table) return fail(GR_EINVAL, "GR_EOS_TABLE needs params.table (gr_eos_create)");
    if (!(p->rho_atm > 0) || !(p->T_atm > 0) || !std::isfinite(p->Ye_atm))
      return fail(GR_EINVAL, "table: rho_atm, T_atm must be positive and Ye_atm finite");
  }
  return GR_OK;
}


static KParams kparams(const gr_params* p, double dt);

// kparams with GR_GUESS_AUTO replaced by the mesh's choice for the call's precision and EOS
static KParams kparams_m(const gr_mesh* m, const gr_params* p, double dt) {
  KParams k = kparams(p, dt);
  if (p->c2p_guess == GR_GUESS_AUTO) k.c2p_guess = m->guess[p->precision][p->eos];
  return k;
}

static KParams kparams(const gr_params* p, double dt) {
  KParams k{};
  k.recon = p->recon; k.emf = p->emf; k.ceiling = p->ceiling; k.max_iter = p->max_iter;
  k.c2p_guess = p->c2p_guess;
  k.eos = p->eos;
  k.gamma_ad = p->gamma_ad; k.rho_atm = p->rho_atm; k.p_atm = p->p_atm; k.f_thr = p->f_thr;
  k.gamma_f = (float)p->gamma_ad;
  k.vmax2 = 1.0 - 1.0 / (p->W_max * p->W_max);
  k.vmax2_f = (float)k.vmax2;
  k.W_max = p->W_max; k.M_max = p->M_max; k.tol = p->tol; k.weno_eps = p->weno_eps;
  k.rk_g0 = p->rk_g0; k.rk_g1 = p->rk_g1; k.rk_beta = p->rk_beta;
  k.rk_form = (p->rk_g0 != 0.0 ? RK_G0 : 0) | (p->rk_g1 != 1.0 ? RK_G1 : 0);
  k.rho_thr = p->f_thr * p->rho_atm * (1.0 + p->atm_band);
  k.dt = dt;
  k.bdt = p->rk_beta * dt;
  k.mlp = p->c2p_guess == GR_GUESS_MLP ? p->mlp : nullptr;
  k.eint_atm = p->p_atm / (p->gamma_ad - 1.0);
  k.h0 = 1.0;
  if (p->eos == GR_EOS_TABLE) {
    const gr_eos& t = *p->table;
    k.T_atm = p->T_atm;
    k.Ye_atm = p->Ye_atm;
    k.h0 = t.h0;
    // atmosphere state of the table (App. A): rho_atm, T_atm, Ye_atm, its p and rho eps
    const double x[3] = {std::log(p->rho_atm), std::log(p->T_atm), p->Ye_atm};
    k.p_atm = p->rho_atm * std::exp(host_tri(t, 0, x));
    k.eint_atm = p->rho_atm * std::expm1(host_tri(t, 1, x));
    k.t64 = tab_view<double>(t, t.d64);
    k.t32 = tab_view<float>(t, t.d32);
  }
  k.top = 1.0 / k.h0;
  k.h0sq = k.h0 * k.h0;
  k.top_f = (float)k.top;
  k.h0sq_f = (float)k.h0sq;
  return k;
}

static int metric_view(const gr_metric* metric, MetricView& mv, bool need_K) {
  if (!metric) return fail(GR_EINVAL, "metric is NULL");
  if (metric->order != 2 && metric->order != 4) return fail(GR_EINVAL, "metric order must be 2 or 4");
  const bool has32 = metric->v32[0] != nullptr;
  for (int c = 0; c < 16; ++c) {
    mv.v[c] = metric->v[c];
    mv.v32[c] = has32 ? metric->v32[c] : nullptr;
    const bool needed = c < 10 || (need_K && !metric->k_zero);
    if (needed && !mv.v[c]) return fail(GR_EINVAL, "metric component pointer is NULL");
    if (needed && has32 && !mv.v32[c]) return fail(GR_EINVAL, "metric: v32 given for some components only");
  }
  mv.order = metric->order;
  mv.k_zero = metric->k_zero;
  return GR_OK;
}

struct gr_graph {
  int device;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

static int stage_impl(gr_mesh* mesh, const gr_metric* metric, const gr_state* state, double dt,
                      const gr_params* params, void* stream, bool allow_profile);

// The stage variant of a call for path `path` (GR_PATH_*): where the call is the mixed path with the ideal
// gas, the order-2 metric and no level-boundary corrections, the fused sweep (*nfused = blocks) or the
// tiled face sweep (ws->nftiles) if the mesh qualifies; otherwise (and for GR_PATH_SEPARATE) the separate
// kernels.  Returns whether the requested variant applies.
static bool stage_variant(const gr_mesh* mesh, const gr_params* p, const MetricView& mv, int path, int* nfused,
                          Workspace* ws) {
  *ws = mesh->ws;
  ws->ftiles = nullptr;
  ws->nftiles = 0;
  *nfused = 0;
  const bool mixed_ideal = p->precision == GR_PREC_MIXED && p->eos == GR_EOS_IDEAL && mv.order == 2 &&
                           mesh->ws.nlvl == 0;
  if (path == GR_PATH_FUSED && mixed_ideal && mesh->fused_ok && mesh->ws.nsweep > 0) {
    *nfused = mesh->nblocks;
    return true;
  }
  if (path == GR_PATH_TILED_FACES && mixed_ideal && mesh->tiles_ok) {
    ws->ftiles = mesh->d_ftiles;
    ws->nftiles = mesh->nftiles;
    return true;
  }
  return path == GR_PATH_SEPARATE;
}
static int stage_prepare(gr_mesh* mesh, const gr_metric* metric, const gr_state* state, double dt,
                         const gr_params* params, MetricView& mv, StateView& s);

int gr_stage(gr_mesh* mesh, const gr_metric* metric, const gr_state* state, double dt,
             const gr_params* params, void* stream) {
  return stage_impl(mesh, metric, state, dt, params, stream, true);
}

int gr_graph_capture(gr_mesh* mesh, const gr_metric* metric, const gr_state* state, double dt,
                     const gr_params* params, gr_graph** graph) {
  if (!mesh || !graph) return fail(GR_EINVAL, "gr_graph_capture: NULL argument");
  DeviceGuard g(mesh->ctx->device);
  cudaStream_t st;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
  e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { cudaStreamDestroy(st); return cuda_fail(e, "cudaStreamBeginCapture"); }
  const int r = stage_impl(mesh, metric, state, dt, params, st, false);
  cudaGraph_t gr = nullptr;
  e = cudaStreamEndCapture(st, &gr);
  cudaStreamDestroy(st);
  if (r != GR_OK) { if (gr) cudaGraphDestroy(gr); return r; }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, gr, 0);
  if (e != cudaSuccess) { cudaGraphDestroy(gr); return cuda_fail(e, "cudaGraphInstantiate"); }
  *graph = new gr_graph{mesh->ctx->device, gr, ex};
  return GR_OK;
}

int gr_graph_launch(gr_graph* graph, void* stream) {
  if (!graph) return fail(GR_EINVAL, "gr_graph_launch: NULL graph");
  DeviceGuard g(graph->device);
  cudaError_t e = cudaGraphLaunch(graph->exec, (cudaStream_t)stream);
  return e == cudaSuccess ? GR_OK : cuda_fail(e, "cudaGraphLaunch");
}

int gr_graph_destroy(gr_graph* graph) {
  if (!graph) return GR_OK;
  DeviceGuard g(graph->device);
  cudaGraphExecDestroy(graph->exec);
  cudaGraphDestroy(graph->graph);
  delete graph;
  return GR_OK;
}

}  // extern "C"

// ---- one stage on host-resident pools ---------------------------------------------------------
// The mesh keeps device copies of the pools (its own layout) and one sub-mesh per batch of consecutive
// blocks; copies in, stages and copies out run on three streams so that one batch's copies overlap
// another batch's stage.
struct HostStage {
  int nbatch = 0;
  std::vector<gr_mesh*> sub;
  // per batch: element ranges [lo, hi) in the parent pools; kind 0 cells, 1..3 faces, 4 vertices
  std::vector<long long> lo[5], hi[5];
  cudaStream_t st[3] = {};                // copies in, stages, copies out
  std::vector<cudaEvent_t> ev_in, ev_out;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;
  double *U[6] = {}, *U0[6] = {}, *W[7] = {}, *Uo[6] = {}, *Wo[7] = {}, *B[3] = {}, *B0[3] = {}, *Bo[3] = {};
  double* M[16] = {};
  uint8_t* status = nullptr;
  std::vector<void*> allocs;
};

static void host_batches_free(HostStage* h) {
  for (gr_mesh* s : h->sub) mesh_free(s);
  h->sub.clear();
  for (cudaEvent_t e : h->ev_in) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_out) cudaEventDestroy(e);
  h->ev_in.clear();
  h->ev_out.clear();
  for (int t = 0; t < 5; ++t) { h->lo[t].clear(); h->hi[t].clear(); }
  h->nbatch = 0;
}

static void host_stage_free(HostStage* h) {
  if (!h) return;
  host_batches_free(h);
  for (int i = 0; i < 3; ++i)
    if (h->st[i]) cudaStreamDestroy(h->st[i]);
  if (h->ev_start) cudaEventDestroy(h->ev_start);
  if (h->ev_end) cudaEventDestroy(h->ev_end);
  for (void* p : h->allocs) cudaFree(p);
  delete h;
}

// Batches of consecutive blocks with about equal cell counts.  Each batch is a mesh of its own whose
// block offsets are rebased to the batch's first element, so that it runs on the parent-layout staging
// pools advanced by those first offsets (its workspace and FP32 shadows cover the batch only).
static int host_stage_setup(gr_mesh* m, int nbatch) {
  if (m->hs && m->hs->nbatch == nbatch) return GR_OK;
  // batches are ranges of the pools: blocks must be laid out in increasing order without overlap
  for (int b = 0; b + 1 < m->nblocks; ++b) {
    const DBlock& x = m->h_blocks[b];
    const DBlock& y = m->h_blocks[b + 1];
    bool ok = x.cell + (long long)x.N[0] * x.N[1] * x.N[2] <= y.cell &&
              x.vert + (long long)(x.N[0] + 1) * (x.N[1] + 1) * (x.N[2] + 1) <= y.vert;
    for (int a = 0; a < 3; ++a)
      ok = ok && x.face[a] + (long long)(x.N[0] + (a == 0)) * (x.N[1] + (a == 1)) * (x.N[2] + (a == 2)) <= y.face[a];
    if (!ok) return fail(GR_EUNSUPPORTED, "gr_host_stage: pools must hold the blocks in increasing order");
  }
  if (m->hs) {
    host_batches_free(m->hs);
  } else {
    m->hs = new HostStage();
    cudaError_t e = cudaSuccess;
    // the transfer streams (0: in, 2: out) at the highest priority the device offers, so that their
    // transfer kernels are scheduled ahead of the waiting CTAs of another batch's stage (stream 1)
    int lo = 0, hi = 0;
    e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
      e = cudaStreamCreateWithPriority(&m->hs->st[i], cudaStreamNonBlocking, i == 1 ? lo : hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->hs->ev_start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->hs->ev_end, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      host_stage_free(m->hs);
      m->hs = nullptr;
      return cuda_fail(e, "gr_host_stage setup");
    }
  }
  HostStage* h = m->hs;
  long long total = 0;
  for (const DBlock& b : m->h_blocks) total += (long long)b.N[0] * b.N[1] * b.N[2];
  std::vector<int> first(1, 0);
  long long acc = 0;
  for (int b = 0; b < m->nblocks; ++b) {
    acc += (long long)m->h_blocks[b].N[0] * m->h_blocks[b].N[1] * m->h_blocks[b].N[2];
    const int k = (int)first.size();
    if (k < nbatch && acc * nbatch >= total * k && b + 1 < m->nblocks) first.push_back(b + 1);
  }
  first.push_back(m->nblocks);
  const int nb = (int)first.size() - 1;
  const long long ext[5] = {m->sh.ncell, m->sh.nface[0], m->sh.nface[1], m->sh.nface[2], m->sh.nvert};
  for (int k = 0; k < nb; ++k) {
    const DBlock& a = m->h_blocks[first[k]];
    const bool last = first[k + 1] >= m->nblocks;
    const DBlock* z = last ? nullptr : &m->h_blocks[first[k + 1]];
    const long long l[5] = {a.cell, a.face[0], a.face[1], a.face[2], a.vert};
    const long long u[5] = {last ? ext[0] : z->cell, last ? ext[1] : z->face[0], last ? ext[2] : z->face[1],
                            last ? ext[3] : z->face[2], last ? ext[4] : z->vert};
    for (int t = 0; t < 5; ++t) { h->lo[t].push_back(l[t]); h->hi[t].push_back(u[t]); }
    std::vector<gr_block> blk;
    for (int b = first[k]; b < first[k + 1]; ++b) {
      const DBlock& d = m->h_blocks[b];
      gr_block g{};
      for (int ax = 0; ax < 3; ++ax) {
        g.n[ax] = d.n[ax];
        g.dx[ax] = d.dx[ax];
        g.face_off[ax] = d.face[ax] - l[1 + ax];
      }
      g.ng = d.g;
      g.cell_off = d.cell - l[0];
      g.vert_off = d.vert - l[4];
      blk.push_back(g);
    }
    gr_mesh* sm = nullptr;
    int r = gr_mesh_create(m->ctx, blk.data(), (int)blk.size(), 0, &sm);
    if (r) { host_batches_free(h); return r; }
    h->sub.push_back(sm);
    cudaEvent_t ea = nullptr, eb = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ea, cudaEventDisableTiming);
    if (e == cudaSuccess) h->ev_in.push_back(ea);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&eb, cudaEventDisableTiming);
    if (e == cudaSuccess) h->ev_out.push_back(eb);
    if (e != cudaSuccess) { host_batches_free(h); return cuda_fail(e, "gr_host_stage events"); }
  }
  h->nbatch = nbatch;
  return GR_OK;
}

static int host_pool(HostStage* h, double** slot, long long n) {
  if (*slot) return GR_OK;
  cudaError_t e = cudaMalloc((void**)slot, sizeof(double) * std::max<long long>(n, 1));
  if (e != cudaSuccess) {
    *slot = nullptr;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? GR_ENOMEM : GR_ECUDA, "gr_host_stage: staging pool");
  }
  h->allocs.push_back(*slot);
  return GR_OK;
}

extern "C" {

static bool host_mapped(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost && at.devicePointer == p;
}

int gr_host_stage(gr_mesh* mesh, const gr_metric* metric, const gr_state* state, double dt, const gr_params* params,
                  int32_t nbatch, void* stream) {
  if (!mesh || !metric || !state) return fail(GR_EINVAL, "gr_host_stage: NULL argument");
  if (nbatch < 1 || nbatch > 1024) return fail(GR_EINVAL, "gr_host_stage: nbatch must be 1..1024");
  if (mesh->ws.nlvl) return fail(GR_EUNSUPPORTED, "gr_host_stage: not with level faces (batches would split them)");
  if (metric->v32[0] || state->W32[0] || state->Wo32[0])
    return fail(GR_EUNSUPPORTED, "gr_host_stage: FP32 copies of the pools are not taken from host memory");
  // the host arrays pass the same checks as a device stage
  MetricView mv0;
  StateView sv0{};
  int r = stage_prepare(mesh, metric, state, dt, params, mv0, sv0);
  if (r) return r;
  if (mesh->nblocks == 0) return GR_OK;
  const bool tab = params->eos == GR_EOS_TABLE;
  const int nq = tab ? 6 : 5, nwr = tab ? 6 : 5, nwo = tab ? 7 : 5, nm = metric->k_zero ? 10 : 16;
  const bool g0 = params->rk_g0 != 0.0;
  bool u0_alias = true, b0_alias = true;
  for (int v = 0; v < nq; ++v) u0_alias = u0_alias && state->U0[v] == state->U[v];
  for (int a = 0; a < 3; ++a) b0_alias = b0_alias && state->B0[a] == state->B[a];
  // every host pool is read or written by the transfer kernels: pinned, device-mapped memory only
  {
    bool ok = host_mapped(state->status);
    for (int v = 0; v < nq; ++v) ok = ok && host_mapped(state->U[v]) && host_mapped(state->Uo[v]);
    for (int v = 0; v < nwr; ++v) ok = ok && host_mapped(state->W[v]);
    for (int v = 0; v < nwo; ++v) ok = ok && host_mapped(state->Wo[v]);
    for (int a = 0; a < 3; ++a) ok = ok && host_mapped(state->B[a]) && host_mapped(state->Bo[a]);
    for (int c = 0; c < nm; ++c) ok = ok && host_mapped(metric->v[c]);
    if (g0 && !u0_alias)
      for (int v = 0; v < nq; ++v) ok = ok && host_mapped(state->U0[v]);
    if (g0 && !b0_alias)
      for (int a = 0; a < 3; ++a) ok = ok && host_mapped(state->B0[a]);
    if (!ok) return fail(GR_EINVAL, "gr_host_stage: host pools must be pinned (page-locked, device-mapped) memory");
  }
  DeviceGuard g(mesh->ctx->device);
  if ((r = host_stage_setup(mesh, nbatch))) return r;
  HostStage* h = mesh->hs;
  const long long nc = mesh->sh.ncell, nv = mesh->sh.nvert;
  // staging pools (device copies in the parent layout)
  for (int v = 0; v < nq; ++v)
    if ((r = host_pool(h, &h->U[v], nc)) || (r = host_pool(h, &h->Uo[v], nc))) return r;
  for (int v = 0; v < nwo; ++v)
    if ((r = host_pool(h, &h->W[v], nc)) || (r = host_pool(h, &h->Wo[v], nc))) return r;
  for (int a = 0; a < 3; ++a)
    if ((r = host_pool(h, &h->B[a], mesh->sh.nface[a])) || (r = host_pool(h, &h->Bo[a], mesh->sh.nface[a]))) return r;
  for (int c = 0; c < nm; ++c)
    if ((r = host_pool(h, &h->M[c], nv))) return r;
  if (g0 && !u0_alias)
    for (int v = 0; v < nq; ++v)
      if ((r = host_pool(h, &h->U0[v], nc))) return r;
  if (g0 && !b0_alias)
    for (int a = 0; a < 3; ++a)
      if ((r = host_pool(h, &h->B0[a], mesh->sh.nface[a]))) return r;
  if (!h->status) {
    cudaError_t ea = cudaMalloc((void**)&h->status, std::max<long long>(nc, 1));
    if (ea != cudaSuccess) { cudaGetLastError(); return fail(GR_ENOMEM, "gr_host_stage: staging pool"); }
    h->allocs.push_back(h->status);
  }
  cudaStream_t user = (cudaStream_t)stream;
  cudaError_t e = cudaEventRecord(h->ev_start, user);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(h->st[i], h->ev_start, 0);
  if (e != cudaSuccess) return cuda_fail(e, "gr_host_stage");
  auto copy = [&](void* dst, const void* src, long long lo, long long hi, cudaStream_t s) {
    if (e != cudaSuccess || hi <= lo) return;
    e = cudaMemcpyAsync((double*)dst + lo, (const double*)src + lo, (hi - lo) * 8, cudaMemcpyHostToDevice, s);
  };
  const int nb = (int)h->sub.size();
  for (int k = 0; k < nb && e == cudaSuccess; ++k) {
    gr_mesh* sm = h->sub[k];
    const long long c0 = h->lo[0][k], c1 = h->hi[0][k], v0 = h->lo[4][k], v1 = h->hi[4][k];
    long long f0[3], f1[3];
    for (int a = 0; a < 3; ++a) { f0[a] = h->lo[1 + a][k]; f1[a] = h->hi[1 + a][k]; }
    // inputs of this batch: W, B, the metric (ghosts included) by the copy engines; U (and U0) on the
    // interior cells only, B0 on the faces of interior cells only, by the transfer kernels
    for (int v = 0; v < nwr; ++v) copy(h->W[v], state->W[v], c0, c1, h->st[0]);
    for (int a = 0; a < 3; ++a) copy(h->B[a], state->B[a], f0[a], f1[a], h->st[0]);
    for (int c = 0; c < nm; ++c) copy(h->M[c], metric->v[c], v0, v1, h->st[0]);
    const void* src[8];
    void* dst[8];
    for (int v = 0; v < nq; ++v) { src[v] = state->U[v] + c0; dst[v] = h->U[v] + c0; }
    if (e == cudaSuccess)
      e = launch_io_cells(sm->d_blocks, sm->d_work[R_INTERIOR], sm->nwork[R_INTERIOR], src, dst, nq, 8, h->st[0]);
    if (g0 && !u0_alias) {
      for (int v = 0; v < nq; ++v) { src[v] = state->U0[v] + c0; dst[v] = h->U0[v] + c0; }
      if (e == cudaSuccess)
        e = launch_io_cells(sm->d_blocks, sm->d_work[R_INTERIOR], sm->nwork[R_INTERIOR], src, dst, nq, 8, h->st[0]);
    }
    if (g0 && !b0_alias && e == cudaSuccess) {
      const double* fs[3] = {state->B0[0] + f0[0], state->B0[1] + f0[1], state->B0[2] + f0[2]};
      double* fd[3] = {h->B0[0] + f0[0], h->B0[1] + f0[1], h->B0[2] + f0[2]};
      e = launch_io_faces(sm->d_blocks, sm->d_work[R_CTFACES], sm->nwork[R_CTFACES], fs, fd, h->st[0]);
    }
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_in[k], h->st[0]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->st[1], h->ev_in[k], 0);
    if (e != cudaSuccess) break;
    // its stage, on the staging pools advanced to the batch's first elements
    gr_metric md = *metric;
    for (int c = 0; c < 16; ++c) md.v[c] = c < nm ? h->M[c] + v0 : nullptr;
    for (int c = 0; c < 16; ++c) md.v32[c] = nullptr;
    gr_state sd{};
    for (int v = 0; v < nq; ++v) {
      sd.U[v] = h->U[v] + c0;
      sd.U0[v] = (g0 && !u0_alias ? h->U0[v] : h->U[v]) + c0;
      sd.Uo[v] = h->Uo[v] + c0;
    }
    for (int v = 0; v < nwo; ++v) {
      sd.W[v] = h->W[v] + c0;
      sd.Wo[v] = h->Wo[v] + c0;
    }
    for (int a = 0; a < 3; ++a) {
      sd.B[a] = h->B[a] + f0[a];
      sd.B0[a] = (g0 && !b0_alias ? h->B0[a] : h->B[a]) + f0[a];
      sd.Bo[a] = h->Bo[a] + f0[a];
    }
    sd.status = h->status + c0;
    std::memcpy(sm->shapes, mesh->shapes, sizeof(mesh->shapes));
    std::memcpy(sm->guess, mesh->guess, sizeof(mesh->guess));
    sm->path = mesh->path;
    if ((r = stage_impl(sm, &md, &sd, dt, params, h->st[1], false))) return r;
    e = cudaEventRecord(h->ev_out[k], h->st[1]);
    // its outputs, the elements the stage writes: interior cells of U', W', status, faces of interior
    // cells of B'
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->st[2], h->ev_out[k], 0);
    for (int v = 0; v < nq; ++v) { src[v] = h->Uo[v] + c0; dst[v] = state->Uo[v] + c0; }
    if (e == cudaSuccess)
      e = launch_io_cells(sm->d_blocks, sm->d_work[R_INTERIOR], sm->nwork[R_INTERIOR], src, dst, nq, 8, h->st[2]);
    for (int v = 0; v < nwo; ++v) { src[v] = h->Wo[v] + c0; dst[v] = state->Wo[v] + c0; }
    if (e == cudaSuccess)
      e = launch_io_cells(sm->d_blocks, sm->d_work[R_INTERIOR], sm->nwork[R_INTERIOR], src, dst, nwo, 8, h->st[2]);
    src[0] = h->status + c0;
    dst[0] = state->status + c0;
    if (e == cudaSuccess)
      e = launch_io_cells(sm->d_blocks, sm->d_work[R_INTERIOR], sm->nwork[R_INTERIOR], src, dst, 1, 1, h->st[2]);
    if (e == cudaSuccess) {
      const double* fs[3] = {h->Bo[0] + f0[0], h->Bo[1] + f0[1], h->Bo[2] + f0[2]};
      double* fd[3] = {state->Bo[0] + f0[0], state->Bo[1] + f0[1], state->Bo[2] + f0[2]};
      e = launch_io_faces(sm->d_blocks, sm->d_work[R_CTFACES], sm->nwork[R_CTFACES], fs, fd, h->st[2]);
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_end, h->st[2]);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(user, h->ev_end, 0);
  return e == cudaSuccess ? GR_OK : cuda_fail(e, "gr_host_stage");
}

// launches of the five stage kernels for the given shapes
static void stage_launches(const gr_mesh* mesh, const gr_shape shp[SK_N], KLaunch kl[SK_N]) {
  for (int k = 0; k < SK_N; ++k) {
    const int t = shp[k].tile == 64 ? 0 : (shp[k].tile == 256 ? 2 : 1);
    const int order = shp[k].order ? 1 : 0;
    kl[k].work = mesh->tw[t][order][kRegionOf[k]];
    kl[k].nwork = k == SK_C2P ? mesh->nint : mesh->tn[t][order][kRegionOf[k]];
    kl[k].threads = tile_size(t);
    kl[k].persistent = shp[k].persistent ? 1 : 0;
  }
}

// validation of a stage call; fills the device views
static int stage_prepare(gr_mesh* mesh, const gr_metric* metric, const gr_state* state, double dt,
                         const gr_params* params, MetricView& mv, StateView& s) {
  if (!mesh || !state) return fail(GR_EINVAL, "gr_stage: NULL argument");
  int r = check_params(params);
  if (r) return r;
  if (!std::isfinite(dt) || dt < 0) return fail(GR_EINVAL, "gr_stage: dt must be finite and >= 0");
  if ((r = metric_view(metric, mv, true))) return r;
  const int need = (params->recon == GR_RECON_PLM ? 2 : 3) + (metric->order == 4 ? 1 : 0);
  if (mesh->nblocks > 0 && mesh->min_ng < need)
    return fail(GR_EINVAL, "gr_stage: ghost width too small for the reconstruction / interpolation stencil");
  const bool tab = params->eos == GR_EOS_TABLE;
  const int nq = tab ? 6 : 5, nwr = tab ? 6 : 5, nwo = tab ? 7 : 5;
  if (tab && params->table->device != mesh->ctx->device)
    return fail(GR_EINVAL, "gr_stage: the EOS table lives on another device");
  for (int v = 0; v < 6; ++v) {
    s.U[v] = state->U[v]; s.U0[v] = state->U0[v]; s.Uo[v] = state->Uo[v];
    if (v >= nq) continue;
    if (!s.U[v] || !s.Uo[v]) return fail(GR_EINVAL, "gr_stage: NULL state array");
    if (params->rk_g0 != 0.0 && !s.U0[v]) return fail(GR_EINVAL, "gr_stage: U0 needed when rk_g0 != 0");
  }
  for (int v = 0; v < 7; ++v) {
    s.W[v] = state->W[v]; s.Wo[v] = state->Wo[v];
    if ((v < nwr && !s.W[v]) || (v < nwo && !s.Wo[v])) return fail(GR_EINVAL, "gr_stage: NULL state array");
  }
  for (int d = 0; d < 3; ++d) {
    s.B[d] = state->B[d]; s.B0[d] = state->B0[d]; s.Bo[d] = state->Bo[d];
    if (!s.B[d] || !s.Bo[d]) return fail(GR_EINVAL, "gr_stage: NULL face array");
    if (params->rk_g0 != 0.0 && !s.B0[d]) return fail(GR_EINVAL, "gr_stage: B0 needed when rk_g0 != 0");
    if ((const double*)s.Bo[d] == s.B[d]) return fail(GR_EINVAL, "gr_stage: Bo must not alias B");
  }
  for (int v = 0; v < nq; ++v)
    if ((const double*)s.Uo[v] == s.U[v]) return fail(GR_EINVAL, "gr_stage: outputs must not alias inputs");
  for (int v = 0; v < nwr; ++v)
    if ((const double*)s.Wo[v] == s.W[v]) return fail(GR_EINVAL, "gr_stage: outputs must not alias inputs");
  s.status = state->status;
  if (!s.status) return fail(GR_EINVAL, "gr_stage: status is NULL");
  s.evals = nullptr;
  // optional FP32 copies of the inputs and outputs (mixed path; all of a group or none)
  const int n32 = tab ? 6 : 5;
  if (params->precision == GR_PREC_MIXED) {
    if (state->W32[0]) {
      for (int v = 0; v < n32; ++v)
        if (!state->W32[v]) return fail(GR_EINVAL, "gr_stage: W32 given for some primitives only");
      for (int d = 0; d < 3; ++d)
        if (!state->B32[d]) return fail(GR_EINVAL, "gr_stage: W32 needs B32");
      for (int v = 0; v < n32; ++v) s.W32[v] = state->W32[v];
      for (int d = 0; d < 3; ++d) s.B32[d] = state->B32[d];
    }
    if (state->Wo32[0]) {
      for (int v = 0; v < n32; ++v)
        if (!state->Wo32[v]) return fail(GR_EINVAL, "gr_stage: Wo32 given for some primitives only");
      for (int d = 0; d < 3; ++d)
        if (!state->Bo32[d]) return fail(GR_EINVAL, "gr_stage: Wo32 needs Bo32");
      for (int v = 0; v < n32; ++v) s.Wo32[v] = state->Wo32[v];
      for (int d = 0; d < 3; ++d) s.Bo32[d] = state->Bo32[d];
      for (int v = 0; v < n32; ++v)
        if ((const float*)s.Wo32[v] == s.W32[v]) return fail(GR_EINVAL, "gr_stage: Wo32 must not alias W32");
      for (int d = 0; d < 3; ++d)
        if ((const float*)s.Bo32[d] == s.B32[d]) return fail(GR_EINVAL, "gr_stage: Bo32 must not alias B32");
    }
  }
  return GR_OK;
}

static int stage_impl(gr_mesh* mesh, const gr_metric* metric, const gr_state* state, double dt,
                      const gr_params* params, void* stream, bool allow_profile) {
  MetricView mv;
  StateView s{};
  const int r = stage_prepare(mesh, metric, state, dt, params, mv, s);
  if (r) return r;
  if (mesh->nblocks == 0) return GR_OK;
  DeviceGuard g(mesh->ctx->device);
  KLaunch kl[SK_N];
  stage_launches(mesh, mesh->shapes[params->precision][params->eos], kl);
  cudaEvent_t* ev = nullptr;
  if (allow_profile && mesh->prof_used < mesh->prof_capacity)
    ev = &mesh->prof_events[(GR_NKERNELS + 1) * mesh->prof_used++];
  int nf = 0;
  Workspace ws;
  stage_variant(mesh, params, mv, mesh->path, &nf, &ws);
  cudaError_t e = launch_stage(params->precision, mesh->d_blocks, kl, mv, s, ws, mesh->sh, kparams_m(mesh, params, dt),
                               (cudaStream_t)stream, ev, true, nf);
  if (e != cudaSuccess) return cuda_fail(e, "gr_stage launch");
  return GR_OK;
}

int gr_mesh_set_path(gr_mesh* mesh, int32_t path) {
  if (!mesh || path < GR_PATH_SEPARATE || path > GR_PATH_TILED_FACES) return fail(GR_EINVAL, "gr_mesh_set_path: bad argument");
  if (path == GR_PATH_FUSED && !mesh->fused_ok)
    return fail(GR_EUNSUPPORTED, "gr_mesh_set_path: a block is wider than 16 cells in x or y or has ghosts != 3");
  if (path == GR_PATH_TILED_FACES && !mesh->tiles_ok)
    return fail(GR_EUNSUPPORTED, "gr_mesh_set_path: a block is wider than 16 cells in x or has ghosts != 3");
  mesh->path = path;
  return GR_OK;
}

int gr_mesh_get_path(const gr_mesh* mesh) { return mesh ? mesh->path : -1; }

int gr_mesh_get_shapes(const gr_mesh* mesh, int32_t precision, int32_t eos, gr_shape out[GR_NSTAGE_KERNELS]) {
  if (!mesh || !out || (precision != GR_PREC_FP64 && precision != GR_PREC_MIXED) ||
      (eos != GR_EOS_IDEAL && eos != GR_EOS_TABLE))
    return fail(GR_EINVAL, "gr_mesh_get_shapes: bad argument");
  for (int k = 0; k < SK_N; ++k) out[k] = mesh->shapes[precision][eos][k];
  return GR_OK;
}

int gr_mesh_set_shapes(gr_mesh* mesh, int32_t precision, int32_t eos, const gr_shape in[GR_NSTAGE_KERNELS]) {
  if (!mesh || !in || (precision != GR_PREC_FP64 && precision != GR_PREC_MIXED) ||
      (eos != GR_EOS_IDEAL && eos != GR_EOS_TABLE))
    return fail(GR_EINVAL, "gr_mesh_set_shapes: bad argument");
  for (int k = 0; k < SK_N; ++k)
    if ((in[k].tile != 64 && in[k].tile != 128 && in[k].tile != 256) || (in[k].order != 0 && in[k].order != 1) ||
        (in[k].persistent != 0 && in[k].persistent != 1))
      return fail(GR_EINVAL, "gr_mesh_set_shapes: tile must be 64, 128 or 256; order and persistent 0 or 1");
  for (int k = 0; k < SK_N; ++k) mesh->shapes[precision][eos][k] = in[k];
  return GR_OK;
}

int gr_autotune(gr_mesh* mesh, const gr_metric* metric, const gr_state* state, double dt, const gr_params* params,
                int32_t reps, void* stream, double best_ms[GR_NSTAGE_KERNELS]) {
  MetricView mv;
  StateView s{};
  int r = stage_prepare(mesh, metric, state, dt, params, mv, s);
  if (r) return r;
  if (reps < 1 || reps > 1000) return fail(GR_EINVAL, "gr_autotune: reps must be in [1, 1000]");
  if (mesh->nblocks == 0) return GR_OK;
  DeviceGuard g(mesh->ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  KParams kp = kparams_m(mesh, params, dt);
  // candidates: CTA size x work-list order x persistent grid, the same for all five kernels in one
  // run; each kernel's time is read from its own events
  std::vector<gr_shape> cand;
  for (int tile : {64, 128, 256})
    for (int order = 0; order < 2; ++order)
      for (int pers = 0; pers < 2; ++pers) cand.push_back(gr_shape{tile, order, pers});
  std::vector<cudaEvent_t> ev((size_t)(GR_NKERNELS + 1) * reps);
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < ev.size() && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
  std::vector<std::vector<double>> ms(cand.size(), std::vector<double>(SK_N, 0.0));
  for (size_t c = 0; c < cand.size() && e == cudaSuccess; ++c) {
    gr_shape shp[SK_N];
    for (int k = 0; k < SK_N; ++k) shp[k] = cand[c];
    KLaunch kl[SK_N];
    stage_launches(mesh, shp, kl);
    e = launch_stage(params->precision, mesh->d_blocks, kl, mv, s, mesh->ws, mesh->sh, kp, st, nullptr);  // warm-up
    for (int rp = 0; rp < reps && e == cudaSuccess; ++rp)
      e = launch_stage(params->precision, mesh->d_blocks, kl, mv, s, mesh->ws, mesh->sh, kp, st,
                       &ev[(size_t)(GR_NKERNELS + 1) * rp]);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (int rp = 0; rp < reps && e == cudaSuccess; ++rp)
      for (int k = 0; k < SK_N && e == cudaSuccess; ++k) {
        float t = 0.f;
        // event slots: 0 before the cast, 1 after it, 2 + k after stage kernel k
        e = cudaEventElapsedTime(&t, ev[(size_t)(GR_NKERNELS + 1) * rp + 1 + k], ev[(size_t)(GR_NKERNELS + 1) * rp + 2 + k]);
        ms[c][k] += t / reps;
      }
  }
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  if (e != cudaSuccess) return cuda_fail(e, "gr_autotune");
  gr_shape* best = mesh->shapes[params->precision][params->eos];
  for (int k = 0; k < SK_N; ++k) {
    const bool has_dir = region_has_dir(kRegionOf[k]);
    int bi = -1;
    for (size_t c = 0; c < cand.size(); ++c) {
      if (!has_dir && cand[c].order != 0) continue;   // the order of a direction-less list is moot
      if (bi < 0 || ms[c][k] < ms[bi][k]) bi = (int)c;
    }
    best[k] = cand[bi];
    if (best_ms) best_ms[k] = ms[bi][k];
  }
  // the whole stage through every path that applies (separate kernels in their chosen shapes, the fused
  // sweep, the tiled face sweep); the fastest is kept for later stages on this mesh
  {
    KLaunch kl[SK_N];
    stage_launches(mesh, best, kl);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    float best_t = -1.f;
    int best_path = GR_PATH_SEPARATE;
    for (int path = GR_PATH_SEPARATE; path <= GR_PATH_TILED_FACES && e == cudaSuccess; ++path) {
      int nf = 0;
      Workspace ws;
      if (!stage_variant(mesh, params, mv, path, &nf, &ws)) continue;
      e = launch_stage(params->precision, mesh->d_blocks, kl, mv, s, ws, mesh->sh, kp, st, nullptr, true, nf);
      if (e == cudaSuccess) e = cudaEventRecord(t0, st);
      for (int rp = 0; rp < reps && e == cudaSuccess; ++rp)
        e = launch_stage(params->precision, mesh->d_blocks, kl, mv, s, ws, mesh->sh, kp, st, nullptr, true, nf);
      if (e == cudaSuccess) e = cudaEventRecord(t1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      float tm = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&tm, t0, t1);
      if (e == cudaSuccess && (best_t < 0.f || tm < best_t)) { best_t = tm; best_path = path; }
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (e != cudaSuccess) return cuda_fail(e, "gr_autotune (stage paths)");
    mesh->path = best_path;
  }
  // GR_GUESS_AUTO: the whole stage (chosen shapes and path) with no bracket proposal and with the FP32
  // pre-solve; the faster stands for AUTO on this mesh
  if (params->c2p_guess == GR_GUESS_AUTO) {
    KLaunch kl[SK_N];
    stage_launches(mesh, best, kl);
    int nf = 0;
    Workspace ws;
    stage_variant(mesh, params, mv, mesh->path, &nf, &ws);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    float best_t = -1.f;
    int best_guess = GR_GUESS_NONE;
    for (int gs : {GR_GUESS_NONE, GR_GUESS_FP32}) {
      if (e != cudaSuccess) break;
      kp.c2p_guess = gs;
      e = launch_stage(params->precision, mesh->d_blocks, kl, mv, s, ws, mesh->sh, kp, st, nullptr, true, nf);
      if (e == cudaSuccess) e = cudaEventRecord(t0, st);
      for (int rp = 0; rp < reps && e == cudaSuccess; ++rp)
        e = launch_stage(params->precision, mesh->d_blocks, kl, mv, s, ws, mesh->sh, kp, st, nullptr, true, nf);
      if (e == cudaSuccess) e = cudaEventRecord(t1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      float tm = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&tm, t0, t1);
      if (e == cudaSuccess && (best_t < 0.f || tm < best_t)) { best_t = tm; best_guess = gs; }
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (e != cudaSuccess) return cuda_fail(e, "gr_autotune (bracket proposal)");
    mesh->guess[params->precision][params->eos] = best_guess;
  }
  return GR_OK;
}

int gr_mesh_get_guess(const gr_mesh* mesh, int32_t precision, int32_t eos) {
  if (!mesh || precision < 0 || precision > 1 || eos < 0 || eos > 1) return -1;
  return mesh->guess[precision][eos];
}

int gr_prim2con(gr_mesh* mesh, const gr_metric* metric, const double* const W[7], const double* const B[3],
                double* const U[6], const gr_params* params, void* stream) {
  if (!mesh || !W || !B || !U) return fail(GR_EINVAL, "gr_prim2con: NULL argument");
  int r = check_params(params);
  if (r) return r;
  MetricView mv;
  if ((r = metric_view(metric, mv, false))) return r;
  const int n = params->eos == GR_EOS_TABLE ? 6 : 5;
  if (params->eos == GR_EOS_TABLE && params->table->device != mesh->ctx->device)
    return fail(GR_EINVAL, "gr_prim2con: the EOS table lives on another device");
  for (int v = 0; v < n; ++v)
    if (!W[v] || !U[v]) return fail(GR_EINVAL, "gr_prim2con: NULL array");
  for (int d = 0; d < 3; ++d)
    if (!B[d]) return fail(GR_EINVAL, "gr_prim2con: NULL face array");
  if (metric->order == 4 && mesh->min_ng < 1) return fail(GR_EINVAL, "gr_prim2con: order 4 needs a ghost");
  if (mesh->nblocks == 0) return GR_OK;
  DeviceGuard g(mesh->ctx->device);
  cudaError_t e = launch_prim2con(mesh->d_blocks, mesh->d_work[R_INTERIOR], mesh->nwork[R_INTERIOR], mv, W,
                                  B, U, kparams(params, 0.0), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gr_prim2con launch");
  return GR_OK;
}

// work lists of the matter-source kernels for one interpolation order (see adm.cu)
static int adm_prepare(gr_mesh* m, int precision, int vc_order) {
  const int o = vc_order == 4 ? 1 : 0, pr = precision == GR_PREC_MIXED ? 1 : 0;
  const size_t elem = pr ? sizeof(float) : sizeof(double);
  if (m->adm_ready[pr][o]) return GR_OK;
  const int np = vc_order, r = np / 2;
  std::vector<Work> cw, vw;
  size_t smem = 0;
  for (int bi = 0; bi < m->nblocks; ++bi) {
    const DBlock& b = m->h_blocks[bi];
    for (int k = -r; k < b.n[2] + r; ++k) cw.push_back(Work{bi, 0, k, 0});   // one CTA per cell plane
    if (adm_smem_bytes(b.n, 1, np, elem) > kAdmSmemMax)
      return fail(GR_EUNSUPPORTED, "gr_adm_sources: block too wide for the interpolation's shared-memory slab");
    const int planes = b.n[2] + 1;
    int zfit = 1;
    while (zfit < planes && adm_smem_bytes(b.n, zfit + 1, np, elem) <= kAdmSmemTarget) ++zfit;
    const int nslab = (planes + zfit - 1) / zfit, Z = (planes + nslab - 1) / nslab;
    for (int z0 = 0; z0 < planes; z0 += Z) {
      const int zc = std::min(Z, planes - z0);
      vw.push_back(Work{bi, zc, z0, 0});
      smem = std::max(smem, adm_smem_bytes(b.n, zc, np, elem));
    }
  }
  DeviceGuard g(m->ctx->device);
  auto upload = [&](const std::vector<Work>& v, Work** dst) -> cudaError_t {
    cudaError_t e = cudaMalloc((void**)dst, sizeof(Work) * std::max<size_t>(v.size(), 1));
    if (e != cudaSuccess) return e;
    m->allocs.push_back(*dst);
    return v.empty() ? cudaSuccess : cudaMemcpy(*dst, v.data(), sizeof(Work) * v.size(), cudaMemcpyHostToDevice);
  };
  cudaError_t e = upload(cw, &m->adm_cw[pr][o]);
  if (e == cudaSuccess) e = upload(vw, &m->adm_vw[pr][o]);
  for (int c = 0; c < 10 && e == cudaSuccess && !m->adm_cv[c]; ++c) {
    e = cudaMalloc(&m->adm_cv[c], sizeof(double) * std::max<long long>(m->sh.ncell, 1));
    if (e == cudaSuccess) m->allocs.push_back(m->adm_cv[c]);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? GR_ENOMEM : GR_ECUDA,
                std::string("gr_adm_sources: ") + cudaGetErrorString(e));
  }
  m->adm_ncw[pr][o] = (int)cw.size();
  m->adm_nvw[pr][o] = (int)vw.size();
  m->adm_smem[pr][o] = smem;
  m->adm_ready[pr][o] = true;
  return GR_OK;
}

int gr_adm_sources(gr_mesh* mesh, const gr_metric* metric, const double* const W[7], const double* const B[3],
                   const gr_params* params, int32_t vc_order, double* const out[10], void* stream) {
  if (!mesh || !W || !B || !out) return fail(GR_EINVAL, "gr_adm_sources: NULL argument");
  int r = check_params(params);
  if (r) return r;
  MetricView mv;
  if ((r = metric_view(metric, mv, false))) return r;
  if (vc_order != 2 && vc_order != 4) return fail(GR_EINVAL, "gr_adm_sources: vc_order must be 2 or 4");
  const bool tab = params->eos == GR_EOS_TABLE;
  if (tab && params->table->device != mesh->ctx->device)
    return fail(GR_EINVAL, "gr_adm_sources: the EOS table lives on another device");
  for (int v = 0; v < (tab ? 6 : 5); ++v)
    if (!W[v]) return fail(GR_EINVAL, "gr_adm_sources: NULL primitive array");
  for (int d = 0; d < 3; ++d)
    if (!B[d]) return fail(GR_EINVAL, "gr_adm_sources: NULL face array");
  for (int c = 0; c < 10; ++c)
    if (!out[c]) return fail(GR_EINVAL, "gr_adm_sources: NULL output array");
  if (mesh->nblocks == 0) return GR_OK;
  if (mesh->min_ng < vc_order / 2 + (metric->order == 4 ? 1 : 0))
    return fail(GR_EINVAL, "gr_adm_sources: ghost width too small for the interpolation orders");
  if ((r = adm_prepare(mesh, params->precision, vc_order))) return r;
  const int o = vc_order == 4 ? 1 : 0, pr = params->precision == GR_PREC_MIXED ? 1 : 0;
  DeviceGuard g(mesh->ctx->device);
  cudaError_t e = launch_adm(params->precision, mesh->d_blocks, mesh->adm_cw[pr][o], mesh->adm_ncw[pr][o],
                             mesh->adm_vw[pr][o], mesh->adm_nvw[pr][o], mesh->adm_smem[pr][o], mv, W, B,
                             kparams(params, 0.0), vc_order, mesh->adm_cv, out, (cudaStream_t)stream);
  return e == cudaSuccess ? GR_OK : cuda_fail(e, "gr_adm_sources launch");
}

// ---- level boundaries ---------------------------------------------------------------------------
static bool half_spacing(const DBlock& c, const DBlock& f) {
  for (int a = 0; a < 3; ++a)
    if (!(std::fabs(2.0 * f.dx[a] - c.dx[a]) <= 1e-12 * c.dx[a])) return false;
  return true;
}
static int floor2h(int i) { return i >= 0 ? i / 2 : -((-i + 1) / 2); }

static int check_map(const gr_mesh* m, const gr_level_map& mp, bool prolong) {
  if (mp.coarse < 0 || mp.coarse >= m->nblocks || mp.fine < 0 || mp.fine >= m->nblocks || mp.coarse == mp.fine)
    return fail(GR_EINVAL, "gr_mesh_set_levels: map block index out of range");
  const DBlock& c = m->h_blocks[mp.coarse];
  const DBlock& f = m->h_blocks[mp.fine];
  if (!half_spacing(c, f)) return fail(GR_EINVAL, "gr_mesh_set_levels: fine spacing must be half the coarse one");
  for (int a = 0; a < 3; ++a) {
    if (mp.hi[a] <= mp.lo[a]) return fail(GR_EINVAL, "gr_mesh_set_levels: empty map range");
    if (!prolong) {
      // coarse cells lo..hi-1 (faces to hi) and the fine cells 2(p - off) + {0, 1}
      if (mp.lo[a] < -c.g || mp.hi[a] > c.n[a] + c.g)
        return fail(GR_EINVAL, "gr_mesh_set_levels: restriction range outside the coarse block");
      if (2 * (mp.lo[a] - mp.off[a]) < -f.g || 2 * (mp.hi[a] - mp.off[a]) > f.n[a] + f.g)
        return fail(GR_EINVAL, "gr_mesh_set_levels: restriction reads outside the fine block");
    } else {
      if (mp.lo[a] < -f.g || mp.hi[a] > f.n[a] + f.g)
        return fail(GR_EINVAL, "gr_mesh_set_levels: prolongation range outside the fine block");
      const int c0 = floor2h(mp.lo[a]) + mp.off[a] - 1, c1 = floor2h(mp.hi[a] - 1) + mp.off[a] + 1;
      if (c0 < -c.g || c1 > c.n[a] + c.g - 1)
        return fail(GR_EINVAL, "gr_mesh_set_levels: prolongation reads outside the coarse block");
    }
  }
  return GR_OK;
}

int gr_mesh_set_levels(gr_mesh* m, const gr_level_face* faces, int32_t nfaces, const gr_level_map* rmaps,
                       int32_t nr, const gr_level_map* pmaps, int32_t np) {
  if (!m || nfaces < 0 || nr < 0 || np < 0 || (nfaces && !faces) || (nr && !rmaps) || (np && !pmaps))
    return fail(GR_EINVAL, "gr_mesh_set_levels: bad argument");
  for (int i = 0; i < nfaces; ++i) {
    const gr_level_face& r = faces[i];
    if (r.coarse < 0 || r.coarse >= m->nblocks || r.fine < 0 || r.fine >= m->nblocks || r.coarse == r.fine ||
        r.dir < 0 || r.dir > 2 || (r.side != 1 && r.side != -1))
      return fail(GR_EINVAL, "gr_mesh_set_levels: bad level face");
    const DBlock& c = m->h_blocks[r.coarse];
    const DBlock& f = m->h_blocks[r.fine];
    if (!half_spacing(c, f)) return fail(GR_EINVAL, "gr_mesh_set_levels: fine spacing must be half the coarse one");
    const int t1 = (r.dir + 1) % 3, t2 = (r.dir + 2) % 3;
    if (f.n[t1] % 2 || f.n[t2] % 2 || r.o1 < 0 || r.o2 < 0 || r.o1 + f.n[t1] / 2 > c.n[t1] ||
        r.o2 + f.n[t2] / 2 > c.n[t2])
      return fail(GR_EINVAL, "gr_mesh_set_levels: level face patch outside the coarse face");
  }
  for (int i = 0; i < nr; ++i)
    if (int e = check_map(m, rmaps[i], false)) return e;
  for (int i = 0; i < np; ++i)
    if (int e = check_map(m, pmaps[i], true)) return e;
  // work lists: cell items first, then the d-face items, per map
  auto build = [](const gr_level_map* maps, int n, std::vector<Work>& w) {
    int ncell = 0;
    for (int kind = 0; kind < 4; ++kind)
      for (int i = 0; i < n; ++i) {
        long long cnt = 1;
        for (int a = 0; a < 3; ++a) cnt *= maps[i].hi[a] - maps[i].lo[a] + (a == kind - 1);
        for (long long s0 = 0; s0 < cnt; s0 += kTile) w.push_back(Work{i, kind, (int)s0, 0});
        if (kind == 0) ncell = (int)w.size();
      }
    return ncell;
  };
  std::vector<Work> rw, pw;
  const int ncr = build(rmaps, nr, rw), ncp = build(pmaps, np, pw);
  DeviceGuard g(m->ctx->device);
  levels_free(m);
  cudaError_t e = cudaSuccess;
  auto up = [&](const void* src, size_t bytes, void** dst) {
    if (e != cudaSuccess || !bytes) return;
    e = cudaMalloc(dst, bytes);
    if (e != cudaSuccess) return;
    m->lvl_allocs.push_back(*dst);
    e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  };
  static_assert(sizeof(LevelFace) == sizeof(gr_level_face) && sizeof(LevelMap) == sizeof(gr_level_map),
                "level record layouts");
  up(faces, sizeof(LevelFace) * nfaces, (void**)&m->d_lvl);
  up(rmaps, sizeof(LevelMap) * nr, (void**)&m->d_rmap);
  up(pmaps, sizeof(LevelMap) * np, (void**)&m->d_pmap);
  up(rw.data(), sizeof(Work) * rw.size(), (void**)&m->d_rwork);
  up(pw.data(), sizeof(Work) * pw.size(), (void**)&m->d_pwork);
  if (e != cudaSuccess) {
    cudaGetLastError();
    levels_free(m);
    return fail(e == cudaErrorMemoryAllocation ? GR_ENOMEM : GR_ECUDA,
                std::string("gr_mesh_set_levels: ") + cudaGetErrorString(e));
  }
  m->ws.lvl = m->d_lvl;
  m->ws.nlvl = nfaces;
  m->nrwork = (int)rw.size();
  m->npwork = (int)pw.size();
  m->ncw_r = ncr;
  m->ncw_p = ncp;
  return GR_OK;
}

static int amr_apply(gr_mesh* m, bool prolong, double* const cells[8], int32_t nvar, double* const B[3],
                     void* stream) {
  const char* what = prolong ? "gr_prolong" : "gr_restrict";
  if (!m || nvar < 0 || nvar > 8 || (nvar && !cells)) return fail(GR_EINVAL, std::string(what) + ": bad argument");
  for (int v = 0; v < nvar; ++v)
    if (!cells[v]) return fail(GR_EINVAL, std::string(what) + ": NULL cell pool");
  if (B)
    for (int d = 0; d < 3; ++d)
      if (!B[d]) return fail(GR_EINVAL, std::string(what) + ": NULL face pool");
  DeviceGuard g(m->ctx->device);
  const Work* w = prolong ? m->d_pwork : m->d_rwork;
  const int nall = prolong ? m->npwork : m->nrwork, ncell = prolong ? m->ncw_p : m->ncw_r;
  double* cv[8] = {};
  for (int v = 0; v < nvar; ++v) cv[v] = cells[v];
  // without face pools only the cell items run (they come first); without cell pools only the faces
  const Work* w0 = nvar ? w : w + ncell;
  const int n = (nvar ? (B ? nall : ncell) : (B ? nall - ncell : 0));
  const cudaError_t e = launch_amr(prolong, m->d_blocks, prolong ? m->d_pmap : m->d_rmap, w0, n, cv, nvar, B,
                                   (cudaStream_t)stream);
  return e == cudaSuccess ? GR_OK : cuda_fail(e, what);
}

int gr_restrict(gr_mesh* m, double* const cells[8], int32_t nvar, double* const B[3], void* stream) {
  return amr_apply(m, false, cells, nvar, B, stream);
}

int gr_prolong(gr_mesh* m, double* const cells[8], int32_t nvar, double* const B[3], void* stream) {
  return amr_apply(m, true, cells, nvar, B, stream);
}

int gr_con2prim(gr_mesh* mesh, const gr_metric* metric, double* const U[6], const double* const B[3],
                double* const W[7], uint8_t* status, int32_t* evals, const gr_params* params, void* stream) {
  if (!mesh || !W || !B || !U) return fail(GR_EINVAL, "gr_con2prim: NULL argument");
  int r = check_params(params);
  if (r) return r;
  MetricView mv;
  if ((r = metric_view(metric, mv, false))) return r;
  const bool tab = params->eos == GR_EOS_TABLE;
  if (tab && params->table->device != mesh->ctx->device)
    return fail(GR_EINVAL, "gr_con2prim: the EOS table lives on another device");
  for (int v = 0; v < (tab ? 7 : 5); ++v)
    if (!W[v] || (v < (tab ? 6 : 5) && !U[v])) return fail(GR_EINVAL, "gr_con2prim: NULL array");
  for (int d = 0; d < 3; ++d)
    if (!B[d]) return fail(GR_EINVAL, "gr_con2prim: NULL face array");
  if (mesh->nblocks == 0) return GR_OK;
  DeviceGuard g(mesh->ctx->device);
  cudaError_t e = launch_con2prim(mesh->d_blocks, mesh->d_work[R_INTERIOR], mesh->nwork[R_INTERIOR], mesh->nint,
                                  mv, U, B, W, status, evals, mesh->ws, kparams_m(mesh, params, 0.0), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gr_con2prim launch");
  return GR_OK;
}

int gr_c2p_samples(gr_mesh* mesh, const gr_metric* metric, const double* const U[6], const double* const B[3],
                   const gr_params* params, float* const feats[6], float* target, uint8_t* valid, void* stream) {
  if (!mesh || !U || !B || !feats || !target || !valid) return fail(GR_EINVAL, "gr_c2p_samples: NULL argument");
  int r = check_params(params);
  if (r) return r;
  MetricView mv;
  if ((r = metric_view(metric, mv, false))) return r;
  if (params->eos == GR_EOS_TABLE && params->table->device != mesh->ctx->device)
    return fail(GR_EINVAL, "gr_c2p_samples: the EOS table lives on another device");
  for (int v = 0; v < (params->eos == GR_EOS_TABLE ? 6 : 5); ++v)
    if (!U[v]) return fail(GR_EINVAL, "gr_c2p_samples: NULL array");
  for (int j = 0; j < GR_MLP_NIN; ++j)
    if (!feats[j]) return fail(GR_EINVAL, "gr_c2p_samples: NULL feature array");
  for (int d = 0; d < 3; ++d)
    if (!B[d]) return fail(GR_EINVAL, "gr_c2p_samples: NULL face array");
  if (mesh->nblocks == 0) return GR_OK;
  DeviceGuard g(mesh->ctx->device);
  cudaError_t e = launch_c2p_samples(mesh->d_blocks, mesh->d_work[R_INTERIOR], mesh->nwork[R_INTERIOR], mv, U, B,
                                     feats, target, valid, kparams(params, 0.0), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gr_c2p_samples launch");
  return GR_OK;
}

// ------------------------------------------------------------------------------------------------
// RK driver: ghost exchange, CFL dt, SSP-RK2/RK3 steps
// ------------------------------------------------------------------------------------------------
struct gr_driver {
  gr_mesh* mesh = nullptr;
  int device = 0;
  int* d_nbr = nullptr;
  GhostMap gmap{};   // gather map of the same-level ghost fill (device arrays in allocs)
  double* d_rate = nullptr;
  double* d_dt = nullptr;
  double* U[2][6] = {};
  double* W[2][7] = {};
  double* B[2][3] = {};
  // mixed path: FP32 copies of the stage buffers' W and B, written by the stage that produces them and
  // ghost-filled with them, so that a later stage of the step converts nothing
  float* W32[2][6] = {};
  float* B32[2][3] = {};
  uint8_t* status = nullptr;
  std::vector<void*> allocs;
};

static void driver_free(gr_driver* d) {
  if (!d) return;
  DeviceGuard g(d->device);
  for (void* p : d->allocs) cudaFree(p);
  delete d;
}

int gr_driver_destroy(gr_driver* d) {
  driver_free(d);
  return GR_OK;
}

int gr_driver_create(gr_mesh* mesh, const int32_t* nbr, gr_driver** out) {
  if (!mesh || !nbr || !out) return fail(GR_EINVAL, "gr_driver_create: NULL argument");
  const int nb = mesh->nblocks;
  for (int b = 0; b < nb; ++b) {
    if (nbr[27 * b + 13] != b) return fail(GR_EINVAL, "gr_driver_create: entry 13 of a block must be the block itself");
    for (int k = 0; k < 27; ++k) {
      const int s = nbr[27 * b + k];
      if (s < -1 || s >= nb) return fail(GR_EINVAL, "gr_driver_create: neighbour index out of range");
      if (s >= 0) {
        const DBlock& x = mesh->h_blocks[b];
        const DBlock& y = mesh->h_blocks[s];
        if (x.g != y.g || x.n[0] != y.n[0] || x.n[1] != y.n[1] || x.n[2] != y.n[2])
          return fail(GR_EINVAL, "gr_driver_create: neighbours must have the same size and ghost width");
        // a ghost layer is copied from the neighbour's owned cells only when it is at least g cells deep
        const int o[3] = {k % 3 - 1, (k / 3) % 3 - 1, k / 9 - 1};
        for (int a = 0; a < 3; ++a)
          if (o[a] != 0 && x.n[a] < x.g)
            return fail(GR_EINVAL, "gr_driver_create: a block with a neighbour along an axis needs n >= ghost width");
      }
    }
  }
  std::vector<int2> gent;
  std::vector<int> gout;
  std::vector<int4> goff;
  if (build_ghost_map(mesh->h_blocks.data(), nb, gent, gout, goff) != 0)
    return fail(GR_EINVAL, "gr_driver_create: a block's ghost-padded arrays must hold fewer than 2^27 elements");
  DeviceGuard g(mesh->ctx->device);
  gr_driver* d = new gr_driver();
  d->mesh = mesh;
  d->device = mesh->ctx->device;
  auto dalloc = [&](size_t bytes, void** p) -> cudaError_t {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e == cudaSuccess) d->allocs.push_back(*p);
    return e;
  };
  cudaError_t e = dalloc(sizeof(int) * 27 * std::max(1, nb), (void**)&d->d_nbr);
  if (e == cudaSuccess && nb) e = cudaMemcpy(d->d_nbr, nbr, sizeof(int) * 27 * nb, cudaMemcpyHostToDevice);
  {
    int2* ge = nullptr;
    int* go = nullptr;
    int4* gf = nullptr;
    if (e == cudaSuccess) e = dalloc(sizeof(int2) * std::max<size_t>(gent.size(), 1), (void**)&ge);
    if (e == cudaSuccess) e = dalloc(sizeof(int) * std::max<size_t>(gout.size(), 1), (void**)&go);
    if (e == cudaSuccess) e = dalloc(sizeof(int4) * std::max<size_t>(goff.size(), 1), (void**)&gf);
    if (e == cudaSuccess && !gent.empty()) e = cudaMemcpy(ge, gent.data(), sizeof(int2) * gent.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !gout.empty()) e = cudaMemcpy(go, gout.data(), sizeof(int) * gout.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !goff.empty()) e = cudaMemcpy(gf, goff.data(), sizeof(int4) * goff.size(), cudaMemcpyHostToDevice);
    d->gmap = GhostMap{ge, go, gf};
  }
  if (e == cudaSuccess) e = dalloc(sizeof(double) * 2, (void**)&d->d_rate);
  if (e == cudaSuccess) e = dalloc(sizeof(double) * 2, (void**)&d->d_dt);
  const long long nc = mesh->sh.ncell;
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    for (int v = 0; v < 6 && e == cudaSuccess; ++v) e = dalloc(sizeof(double) * nc, (void**)&d->U[k][v]);
    for (int v = 0; v < 7 && e == cudaSuccess; ++v) e = dalloc(sizeof(double) * nc, (void**)&d->W[k][v]);
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) e = dalloc(sizeof(double) * mesh->sh.nface[a], (void**)&d->B[k][a]);
    // FP32 copies of the stage buffers' W and B for the mixed path (made here: a step may be captured)
    for (int v = 0; v < 6 && e == cudaSuccess; ++v) e = dalloc(sizeof(float) * nc, (void**)&d->W32[k][v]);
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) e = dalloc(sizeof(float) * mesh->sh.nface[a], (void**)&d->B32[k][a]);
  }
  if (e == cudaSuccess) e = dalloc(std::max<long long>(nc, 1), (void**)&d->status);
  if (e != cudaSuccess) {
    const int code = (e == cudaErrorMemoryAllocation) ? GR_ENOMEM : GR_ECUDA;
    std::string msg = std::string("gr_driver_create: ") + cudaGetErrorString(e);
    cudaGetLastError();
    driver_free(d);
    return fail(code, msg);
  }
  *out = d;
  return GR_OK;
}

int gr_ghost_fill(gr_driver* d, double* const W[7], int32_t nw, double* const B[3], void* stream) {
  if (!d || !W || !B || nw < 0 || nw > 7) return fail(GR_EINVAL, "gr_ghost_fill: bad argument");
  for (int v = 0; v < nw; ++v)
    if (!W[v]) return fail(GR_EINVAL, "gr_ghost_fill: NULL cell pool");
  for (int a = 0; a < 3; ++a)
    if (!B[a]) return fail(GR_EINVAL, "gr_ghost_fill: NULL face pool");
  gr_mesh* m = d->mesh;
  if (m->nblocks == 0) return GR_OK;
  DeviceGuard g(d->device);
  cudaError_t e = launch_ghost_fill(m->d_blocks, m->nblocks, d->d_nbr, d->gmap, W, nw, B, (cudaStream_t)stream);
  return e == cudaSuccess ? GR_OK : cuda_fail(e, "gr_ghost_fill");
}

int gr_cfl_dt(gr_driver* d, const gr_metric* metric, const double* const W[7], const double* const B[3],
              const gr_params* params, double cfl, double* dt_dev, void* stream) {
  if (!d || !W || !B) return fail(GR_EINVAL, "gr_cfl_dt: NULL argument");
  int r = check_params(params);
  if (r) return r;
  MetricView mv;
  if ((r = metric_view(metric, mv, false))) return r;
  if (!(cfl > 0) || !std::isfinite(cfl)) return fail(GR_EINVAL, "gr_cfl_dt: cfl must be positive");
  gr_mesh* m = d->mesh;
  DeviceGuard g(d->device);
  cudaError_t e = launch_cfl_dt(m->d_blocks, m->d_work[R_INTERIOR], m->nwork[R_INTERIOR], mv, W, B, kparams(params, 0.0),
                                cfl, d->d_rate, dt_dev ? dt_dev : d->d_dt, (cudaStream_t)stream);
  return e == cudaSuccess ? GR_OK : cuda_fail(e, "gr_cfl_dt");
}

// ghosts of the driver's state: same-level copies, then (on a refined mesh) restriction into coarse
// ghosts and prolongation into fine ghosts
static int driver_fill(gr_driver* d, double* const W[7], int nw, double* const B[3], void* stream) {
  int r = gr_ghost_fill(d, W, nw, B, stream);
  if (r) return r;
  gr_mesh* m = d->mesh;
  double* cells[8] = {};
  for (int v = 0; v < nw; ++v) cells[v] = W[v];
  if (m->nrwork && (r = amr_apply(m, false, cells, nw, B, stream))) return r;
  if (m->npwork && (r = amr_apply(m, true, cells, nw, B, stream))) return r;
  return GR_OK;
}

static int driver_step_impl(gr_driver* d, const gr_metric* metric, double* const U[6], double* const W[7],
                            double* const B[3], uint8_t* status, const gr_params* params, double cfl,
                            int32_t dt_mode, int32_t rk_order, void* stream) {
  if (!d || !U || !W || !B || !status) return fail(GR_EINVAL, "gr_driver_step: NULL argument");
  int r = check_params(params);
  if (r) return r;
  if (rk_order != 2 && rk_order != 3) return fail(GR_EINVAL, "gr_driver_step: rk_order must be 2 or 3");
  if (dt_mode != GR_DT_GRID && dt_mode != GR_DT_SIGNAL) return fail(GR_EINVAL, "gr_driver_step: bad dt_mode");
  if (!(cfl > 0) || !std::isfinite(cfl)) return fail(GR_EINVAL, "gr_driver_step: cfl must be positive");
  gr_mesh* m = d->mesh;
  const bool tab = params->eos == GR_EOS_TABLE;
  const int nq = tab ? 6 : 5, nw = tab ? 7 : 5;
  for (int v = 0; v < nq; ++v)
    if (!U[v]) return fail(GR_EINVAL, "gr_driver_step: NULL conserved pool");
  for (int v = 0; v < nw; ++v)
    if (!W[v]) return fail(GR_EINVAL, "gr_driver_step: NULL primitive pool");
  // (g0, g1, beta) per stage: SSP-RK2 / SSP-RK3 in Shu-Osher form
  static const double rk2[2][3] = {{0.0, 1.0, 1.0}, {0.5, 0.5, 0.5}};
  static const double rk3[3][3] = {{0.0, 1.0, 1.0}, {0.75, 0.25, 0.25}, {1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0}};
  const double (*co)[3] = rk_order == 2 ? rk2 : rk3;
  DeviceGuard g(d->device);
  cudaStream_t st = (cudaStream_t)stream;
  // ghosts of the step's input state, then dt from it
  if ((r = driver_fill(d, W, nw, B, stream))) return r;
  if (dt_mode == GR_DT_SIGNAL) {
    if ((r = gr_cfl_dt(d, metric, W, B, params, cfl, nullptr, stream))) return r;
  } else {
    double mindx = HUGE_VAL;
    for (const DBlock& b : m->h_blocks) mindx = std::min(mindx, std::min(b.dx[0], std::min(b.dx[1], b.dx[2])));
    const cudaError_t e = launch_set_scalar(d->d_dt, cfl * mindx, st);
    if (e != cudaSuccess) return cuda_fail(e, "gr_driver_step dt");
  }
  // mixed path on a mesh without level maps: FP32 copies chained between the stages
  const bool chain32 = params->precision == GR_PREC_MIXED && !m->nrwork && !m->npwork;
  double* inU[6];
  double* inW[7];
  double* inB[3];
  for (int v = 0; v < 6; ++v) inU[v] = v < nq ? U[v] : nullptr;
  for (int v = 0; v < 7; ++v) inW[v] = v < nw ? W[v] : nullptr;
  for (int a = 0; a < 3; ++a) inB[a] = B[a];
  for (int s = 0; s < rk_order; ++s) {
    const bool last = s == rk_order - 1;
    gr_params ps = *params;
    ps.rk_g0 = co[s][0];
    ps.rk_g1 = co[s][1];
    ps.rk_beta = co[s][2];
    gr_state state{};
    for (int v = 0; v < nq; ++v) {
      state.U[v] = inU[v];
      state.U0[v] = U[v];
      state.Uo[v] = last ? U[v] : d->U[s % 2][v];
    }
    for (int v = 0; v < nw; ++v) {
      state.W[v] = inW[v];
      state.Wo[v] = last ? W[v] : d->W[s % 2][v];
    }
    for (int a = 0; a < 3; ++a) {
      state.B[a] = inB[a];
      state.B0[a] = B[a];
      state.Bo[a] = last ? B[a] : d->B[s % 2][a];
    }
    state.status = last ? status : d->status;
    if (chain32) {
      if (s > 0) {   // the previous stage's outputs, FP32 copies included, ghosts filled below
        for (int v = 0; v < 6; ++v) state.W32[v] = d->W32[(s - 1) % 2][v];
        for (int a = 0; a < 3; ++a) state.B32[a] = d->B32[(s - 1) % 2][a];
      }
      if (!last) {
        for (int v = 0; v < 6; ++v) state.Wo32[v] = d->W32[s % 2][v];
        for (int a = 0; a < 3; ++a) state.Bo32[a] = d->B32[s % 2][a];
      }
    }
    MetricView mv;
    StateView sv{};
    // the last stage writes over the step's input (also its U0, B0): each thread reads U0, B0 of
    // its own element before writing it, and the stage's W and B inputs are the previous stage's
    if ((r = stage_prepare(m, metric, &state, 0.0, &ps, mv, sv))) return r;
    KLaunch kl[SK_N];
    stage_launches(m, m->shapes[params->precision][params->eos], kl);
    KParams kp = kparams_m(m, &ps, 0.0);
    kp.dt_dev = d->d_dt;
    // the stages of a step share the metric: its FP32 shadow (mixed path) is made by the first one
    int nf = 0;
    Workspace wsv;
    stage_variant(m, &ps, mv, m->path, &nf, &wsv);
    cudaError_t e = launch_stage(params->precision, m->d_blocks, kl, mv, sv, wsv, m->sh, kp, st, nullptr, s == 0, nf);
    if (e != cudaSuccess) return cuda_fail(e, "gr_driver_step stage");
    if (!last) {
      for (int v = 0; v < nq; ++v) inU[v] = d->U[s % 2][v];
      for (int v = 0; v < nw; ++v) inW[v] = d->W[s % 2][v];
      for (int a = 0; a < 3; ++a) inB[a] = d->B[s % 2][a];
      if (chain32) {   // same-level ghosts of the FP64 buffers and their FP32 copies in one pass
        e = launch_ghost_fill(m->d_blocks, m->nblocks, d->d_nbr, d->gmap, inW, nw, inB, st, d->W32[s % 2], d->B32[s % 2]);
        if (e != cudaSuccess) return cuda_fail(e, "gr_driver_step ghost fill");
      } else if ((r = driver_fill(d, inW, nw, inB, stream))) {
        return r;
      }
    }
  }
  return GR_OK;
}

int gr_driver_step(gr_driver* d, const gr_metric* metric, double* const U[6], double* const W[7], double* const B[3],
                   uint8_t* status, const gr_params* params, double cfl, int32_t dt_mode, int32_t rk_order,
                   void* stream) {
  return driver_step_impl(d, metric, U, W, B, status, params, cfl, dt_mode, rk_order, stream);
}

int gr_driver_dt(const gr_driver* d, double* dt) {
  if (!d || !dt) return fail(GR_EINVAL, "gr_driver_dt: NULL argument");
  DeviceGuard g(d->device);
  cudaError_t e = cudaMemcpy(dt, d->d_dt, sizeof(double), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? GR_OK : cuda_fail(e, "gr_driver_dt");
}

const double* gr_driver_dt_device(const gr_driver* d) { return d ? d->d_dt : nullptr; }

int gr_driver_capture(gr_driver* d, const gr_metric* metric, double* const U[6], double* const W[7],
                      double* const B[3], uint8_t* status, const gr_params* params, double cfl, int32_t dt_mode,
                      int32_t rk_order, gr_graph** graph) {
  if (!d || !graph) return fail(GR_EINVAL, "gr_driver_capture: NULL argument");
  DeviceGuard g(d->device);
  cudaStream_t st;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
  e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { cudaStreamDestroy(st); return cuda_fail(e, "cudaStreamBeginCapture"); }
  const int r = driver_step_impl(d, metric, U, W, B, status, params, cfl, dt_mode, rk_order, st);
  cudaGraph_t gr = nullptr;
  e = cudaStreamEndCapture(st, &gr);
  cudaStreamDestroy(st);
  if (r != GR_OK) { if (gr) cudaGraphDestroy(gr); return r; }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, gr, 0);
  if (e != cudaSuccess) { cudaGraphDestroy(gr); return cuda_fail(e, "cudaGraphInstantiate"); }
  *graph = new gr_graph{d->device, gr, ex};
  return GR_OK;
}

int gr_eos_destroy(gr_eos* t) {
  if (!t) return GR_OK;
  DeviceGuard g(t->device);
  for (int f = 0; f < 3; ++f) {
    if (t->d64[f]) cudaFree(t->d64[f]);
    if (t->d32[f]) cudaFree(t->d32[f]);
  }
  delete t;
  return GR_OK;
}

int64_t gr_eos_bytes(const gr_eos* t) { return t ? t->bytes : -1; }
double gr_eos_h0(const gr_eos* t) { return t ? t->h0 : -1.0; }

int gr_eos_create(gr_ctx* ctx, const gr_eos_table* in, gr_eos** out) {
  if (!ctx || !in || !out) return fail(GR_EINVAL, "gr_eos_create: NULL argument");
  if (!in->log_p || !in->log_e || !in->cs2) return fail(GR_EINVAL, "gr_eos_create: NULL node array");
  long long nn = 1;
  for (int a = 0; a < 3; ++a) {
    if (in->n[a] < 2 || in->n[a] > 100000) return fail(GR_EINVAL, "gr_eos_create: each axis needs 2..100000 nodes");
    if (!(in->dx[a] > 0) || !std::isfinite(in->dx[a]) || !std::isfinite(in->x0[a]))
      return fail(GR_EINVAL, "gr_eos_create: axis origin and spacing must be finite, spacing > 0");
    nn *= in->n[a];
  }
  if (nn > (1LL << 28)) return fail(GR_EINVAL, "gr_eos_create: more than 2^28 nodes");
  gr_eos* t = new gr_eos();
  t->device = ctx->device;
  for (int a = 0; a < 3; ++a) {
    t->n[a] = in->n[a];
    t->x0[a] = in->x0[a];
    t->dx[a] = in->dx[a];
    t->hi[a] = in->x0[a] + (in->n[a] - 1) * in->dx[a];
  }
  for (int f = 0; f < 3; ++f) t->host[f].resize(nn);
  t->h0 = HUGE_VAL;
  const int n0 = in->n[0], n1 = in->n[1], n2 = in->n[2];
  for (int iy = 0; iy < n2; ++iy)
    for (int iT = 0; iT < n1; ++iT)
      for (int ir = 0; ir < n0; ++ir) {
        const size_t k = ((size_t)iy * n1 + iT) * n0 + ir;
        const double lp = in->log_p[k], le = in->log_e[k], c2 = in->cs2[k];
        if (!std::isfinite(lp) || !std::isfinite(le) || !std::isfinite(c2)) {
          delete t;
          return fail(GR_EINVAL, "gr_eos_create: non-finite table value");
        }
        if (iT > 0 && !(lp > in->log_p[k - n0] && le > in->log_e[k - n0])) {
          delete t;
          return fail(GR_EINVAL, "gr_eos_create: log p and log e must increase strictly with T");
        }
        const double lr = in->x0[0] + ir * in->dx[0];
        t->host[0][k] = lp - lr;      // log(p/rho)
        t->host[1][k] = le - lr;      // log(e/rho) = log(1 + eps)
        t->host[2][k] = c2;
        const double h = std::exp(le - lr) + std::exp(lp - lr);   // (e + p)/rho
        if (h < t->h0) t->h0 = h;
      }
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaSuccess;
  std::vector<float> tmp(nn);
  for (int f = 0; f < 3 && e == cudaSuccess; ++f) {
    e = cudaMalloc(&t->d64[f], sizeof(double) * nn);
    if (e == cudaSuccess) e = cudaMemcpy(t->d64[f], t->host[f].data(), sizeof(double) * nn, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&t->d32[f], sizeof(float) * nn);
    for (long long k = 0; k < nn && e == cudaSuccess; ++k) tmp[k] = (float)t->host[f][k];
    if (e == cudaSuccess) e = cudaMemcpy(t->d32[f], tmp.data(), sizeof(float) * nn, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    const int code = (e == cudaErrorMemoryAllocation) ? GR_ENOMEM : GR_ECUDA;
    std::string msg = std::string("gr_eos_create: ") + cudaGetErrorString(e);
    cudaGetLastError();
    gr_eos_destroy(t);
    return fail(code, msg);
  }
  t->bytes = (int64_t)nn * 3 * (sizeof(double) + sizeof(float));
  *out = t;
  return GR_OK;
}

int gr_cast_f32(const double* src, float* dst, int64_t n, void* stream) {
  if (n < 0) return fail(GR_EINVAL, "gr_cast_f32: n < 0");
  if (n == 0) return GR_OK;
  if (!src || !dst) return fail(GR_EINVAL, "gr_cast_f32: NULL pointer");
  cudaError_t e = launch_cast_pool(src, dst, n, (cudaStream_t)stream);
  return e == cudaSuccess ? GR_OK : cuda_fail(e, "gr_cast_f32 launch");
}

int gr_diag(gr_mesh* mesh, const double* const U[5], const double* const B[3], double out[4], void* stream) {
  if (!mesh || !U || !B || !out) return fail(GR_EINVAL, "gr_diag: NULL argument");
  if (!U[0]) return fail(GR_EINVAL, "gr_diag: NULL D array");
  for (int d = 0; d < 3; ++d)
    if (!B[d]) return fail(GR_EINVAL, "gr_diag: NULL face array");
  DeviceGuard g(mesh->ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = launch_diag(mesh->d_blocks, mesh->d_work[R_INTERIOR], mesh->nwork[R_INTERIOR], U, B,
                              mesh->d_diag, st);
  if (e != cudaSuccess) return cuda_fail(e, "gr_diag launch");
  double h[8];
  e = cudaMemcpyAsync(h, mesh->d_diag, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "gr_diag copy");
  double mindx = 1e300;
  for (const DBlock& b : mesh->h_blocks) mindx = std::min(mindx, std::min(b.dx[0], std::min(b.dx[1], b.dx[2])));
  const double Bmax = (h[3] > 0 || std::isnan(h[3])) ? h[3] : 1.0;   // a NaN field stays NaN
  out[0] = h[0];
  out[1] = h[1] * mindx / Bmax;
  out[2] = (h[4] > 0) ? h[2] / (Bmax * h[4] / mindx) : 0.0;
  out[3] = h[3];
  return GR_OK;
}

}  // extern "C"
