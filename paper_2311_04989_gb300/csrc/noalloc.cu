// noalloc.cu -- gr_diag_noalloc: the mass / div B diagnostics without any device allocation.
//
// For callers that cannot call cudaMalloc: code running inside a host application that owns the
// device memory pool (a simulation framework with its own caching allocator or a fixed arena),
// code invoked while such an allocator forbids out-of-pool allocations, and in-situ analysis hooks
// that must not change the device's memory footprint between steps.  They still pass their own
// input arrays and receive the result on the host.
//
// The reduction's scratch lives in one file-scope static device array of fixed size (below); every
// GPU that loads the library holds it until the process exits.  All calls share it: a call
// overwrites every slot it reads, so nothing carries over from the previous call, but two calls
// whose kernels overlap on the GPU (different streams, or different host threads) race on it and
// must be serialised by the caller.
#include <cmath>
#include <string>

#include "internal.h"

namespace {

constexpr int kNaMaxBlocks = 256;   // blocks per call (the descriptors travel as a kernel parameter)
constexpr int kNaCtas = 512;        // CTAs of the partial-sum pass
constexpr int kNaThreads = 256;
constexpr int kNaStride = 8;        // doubles per partial-sum slot

// per-CTA partial sums (kNaCtas slots) followed by the final slot: 33 KB in total
static __device__ __align__(256) double g_na_scratch[(kNaCtas + 1) * kNaStride];

struct NaBlock {
  int n[3];
  int g;
  double dx[3];
  double idx[3];   // 1/dx, formed on the host as in gr_diag
  long long cell, face[3];
  long long first;   // prefix sum of interior cells of the preceding blocks
};

struct NaArgs {
  NaBlock b[kNaMaxBlocks];
  int nblocks;
  long long total;
  const double* D;
  const double* B[3];
  double* scratch;   // device address of g_na_scratch on the current device
};

// maximum that keeps a NaN, like gr_diag: a field that has gone NaN must not read as finite
__device__ __forceinline__ void na_max(double& a, double b) { a = (b > a || b != b) ? b : a; }

// slots: 0 sum D dV, 1 max |div B|, 2 sum |div B| dV, 3 max |B|, 4 sum dV
__global__ void __launch_bounds__(kNaThreads) k_na_partial(const __grid_constant__ NaArgs a) {
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0;
  for (long long e = blockIdx.x * (long long)kNaThreads + threadIdx.x; e < a.total;
       e += (long long)kNaCtas * kNaThreads) {
    int lo = 0, hi = a.nblocks - 1;   // last block with first <= e
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.b[mid].first <= e) lo = mid; else hi = mid - 1;
    }
    const NaBlock& bk = a.b[lo];
    const long long r = e - bk.first;
    const int i = (int)(r % bk.n[0]), j = (int)((r / bk.n[0]) % bk.n[1]), k = (int)(r / ((long long)bk.n[0] * bk.n[1]));
    const int N0 = bk.n[0] + 2 * bk.g, N1 = bk.n[1] + 2 * bk.g;
    const long long c = bk.cell + ((long long)(k + bk.g) * N1 + (j + bk.g)) * N0 + (i + bk.g);
    const long long fx = bk.face[0] + ((long long)(k + bk.g) * N1 + (j + bk.g)) * (N0 + 1) + (i + bk.g);
    const long long fy = bk.face[1] + ((long long)(k + bk.g) * (N1 + 1) + (j + bk.g)) * N0 + (i + bk.g);
    const long long fz = bk.face[2] + ((long long)(k + bk.g) * N1 + (j + bk.g)) * N0 + (i + bk.g);
    const double dv = bk.dx[0] * bk.dx[1] * bk.dx[2];
    const double bx0 = a.B[0][fx], bx1 = a.B[0][fx + 1];
    const double by0 = a.B[1][fy], by1 = a.B[1][fy + N0];
    const double bz0 = a.B[2][fz], bz1 = a.B[2][fz + (long long)N0 * N1];
    const double div = (bx1 - bx0) * bk.idx[0] + (by1 - by0) * bk.idx[1] + (bz1 - bz0) * bk.idx[2];
    s0 += a.D[c] * dv;
    na_max(s1, fabs(div));
    s2 += fabs(div) * dv;
    na_max(s3, fabs(bx0)); na_max(s3, fabs(bx1)); na_max(s3, fabs(by0));
    na_max(s3, fabs(by1)); na_max(s3, fabs(bz0)); na_max(s3, fabs(bz1));
    s4 += dv;
  }
  __shared__ double sh[kNaThreads / 32][5];
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    na_max(s1, __shfl_down_sync(0xffffffffu, s1, o));
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
    na_max(s3, __shfl_down_sync(0xffffffffu, s3, o));
    s4 += __shfl_down_sync(0xffffffffu, s4, o);
  }
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { sh[wid][0] = s0; sh[wid][1] = s1; sh[wid][2] = s2; sh[wid][3] = s3; sh[wid][4] = s4; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0;
    for (int w = 0; w < kNaThreads / 32; ++w) {
      t0 += sh[w][0]; na_max(t1, sh[w][1]); t2 += sh[w][2]; na_max(t3, sh[w][3]); t4 += sh[w][4];
    }
    double* slot = a.scratch + (long long)blockIdx.x * kNaStride;   // every slot is written each call
    slot[0] = t0; slot[1] = t1; slot[2] = t2; slot[3] = t3; slot[4] = t4;
  }
}

__global__ void __launch_bounds__(32) k_na_final(double* scratch) {
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0;
  for (int c = threadIdx.x; c < kNaCtas; c += 32) {
    const double* slot = scratch + (long long)c * kNaStride;
    s0 += slot[0]; na_max(s1, slot[1]); s2 += slot[2]; na_max(s3, slot[3]); s4 += slot[4];
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    na_max(s1, __shfl_down_sync(0xffffffffu, s1, o));
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
    na_max(s3, __shfl_down_sync(0xffffffffu, s3, o));
    s4 += __shfl_down_sync(0xffffffffu, s4, o);
  }
  if (threadIdx.x == 0) {
    double* fin = scratch + (long long)kNaCtas * kNaStride;
    fin[0] = s0; fin[1] = s1; fin[2] = s2; fin[3] = s3; fin[4] = s4;
  }
}

thread_local std::string g_na_error;

int na_fail(int code, const std::string& msg) {
  g_na_error = msg;
  return code;
}

}  // namespace

extern "C" const char* gr_noalloc_last_error(void) { return g_na_error.c_str(); }

extern "C" int gr_diag_noalloc(const gr_block* blocks, int32_t nblocks, const double* const U[5],
                               const double* const B[3], double out[4], void* stream) {
  if (!blocks || !U || !U[0] || !B || !out) return na_fail(GR_EINVAL, "gr_diag_noalloc: NULL argument");
  for (int d = 0; d < 3; ++d)
    if (!B[d]) return na_fail(GR_EINVAL, "gr_diag_noalloc: NULL face array");
  if (nblocks < 1 || nblocks > kNaMaxBlocks)
    return na_fail(GR_EINVAL, "gr_diag_noalloc: nblocks must be in [1, 256] (the block list travels as a "
                              "kernel parameter); split larger meshes or use gr_diag");
  NaArgs a;
  a.nblocks = nblocks;
  long long first = 0;
  double mindx = 1e300;
  for (int b = 0; b < nblocks; ++b) {
    const gr_block& s = blocks[b];
    NaBlock& d = a.b[b];
    if (s.ng < 0 || s.ng > 8) return na_fail(GR_EINVAL, "gr_diag_noalloc: ng out of range");
    for (int k = 0; k < 3; ++k) {
      if (s.n[k] < 1 || s.n[k] > 1024) return na_fail(GR_EINVAL, "gr_diag_noalloc: n out of range");
      if (!(s.dx[k] > 0) || !std::isfinite(s.dx[k])) return na_fail(GR_EINVAL, "gr_diag_noalloc: dx must be positive");
      d.n[k] = s.n[k];
      d.dx[k] = s.dx[k];
      d.idx[k] = 1.0 / s.dx[k];
      d.face[k] = s.face_off[k];
      mindx = std::fmin(mindx, s.dx[k]);
    }
    if (s.cell_off < 0 || s.face_off[0] < 0 || s.face_off[1] < 0 || s.face_off[2] < 0)
      return na_fail(GR_EINVAL, "gr_diag_noalloc: negative pool offset");
    d.g = s.ng;
    d.cell = s.cell_off;
    d.first = first;
    first += (long long)s.n[0] * s.n[1] * s.n[2];
  }
  a.total = first;
  a.D = U[0];
  for (int d = 0; d < 3; ++d) a.B[d] = B[d];
  // The scratch array's device address belongs to the CUDA context that is current now (the caller's
  // device, possibly a context of its own, or a fresh one after cudaDeviceReset), so it is looked up on
  // every call rather than cached; the lookup allocates nothing.
  void* sp = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&sp, g_na_scratch);
  if (e != cudaSuccess) return na_fail(GR_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  a.scratch = static_cast<double*>(sp);
  cudaStream_t st = (cudaStream_t)stream;
  k_na_partial<<<kNaCtas, kNaThreads, 0, st>>>(a);
  k_na_final<<<1, 32, 0, st>>>(a.scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(GR_ECUDA, std::string("gr_diag_noalloc launch: ") + cudaGetErrorString(e));
  double h[5];
  e = cudaMemcpyAsync(h, a.scratch + (long long)kNaCtas * kNaStride, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return na_fail(GR_ECUDA, std::string("gr_diag_noalloc copy: ") + cudaGetErrorString(e));
  const double Bmax = (h[3] > 0 || std::isnan(h[3])) ? h[3] : 1.0;   // a NaN field stays NaN
  out[0] = h[0];
  out[1] = h[1] * mindx / Bmax;
  out[2] = (h[4] > 0) ? h[2] / (Bmax * h[4] / mindx) : 0.0;
  out[3] = h[3];
  return GR_OK;
}
