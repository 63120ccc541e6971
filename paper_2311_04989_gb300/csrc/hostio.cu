// hostio.cu -- transfers of gr_host_stage that move only the elements a stage reads or writes: the
// interior cells of U (and U0) in, the interior cells of U', W', status and the faces of interior cells
// of B' (and B0 in) out.  The kernels read or write pinned, device-mapped host memory directly (the
// host pools are checked to be such before any launch); a warp covers two 16-cell rows of a 16^3 block,
// 128 contiguous bytes each.
#include "internal.h"
#include "physics.cuh"
#include "stage_common.cuh"

namespace grs {

struct IoCells {
  const void* src[8];
  void* dst[8];
  int n;
};

struct IoFaces {
  const double* src[3];
  double* dst[3];
};

template <class T>
__global__ void __launch_bounds__(kTile) k_io_cells(const DBlock* __restrict__ blocks, const Work* __restrict__ work,
                                                    const __grid_constant__ IoCells a) {
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  int p[3];
  if (!decode<R_INTERIOR, 0>(w, b, p)) return;
  const long long c = b.cell + cix(b, p[0], p[1], p[2]);
  for (int v = 0; v < a.n; ++v) static_cast<T*>(a.dst[v])[c] = static_cast<const T*>(a.src[v])[c];
}

template <int D>
__device__ __forceinline__ void io_face(const Work& w, const DBlock& b, const IoFaces& a) {
  int p[3];
  if (!decode<R_CTFACES, D>(w, b, p)) return;
  const long long f = b.face[D] + fix(b, D, p[0], p[1], p[2]);
  a.dst[D][f] = a.src[D][f];
}

__global__ void __launch_bounds__(kTile) k_io_faces(const DBlock* __restrict__ blocks, const Work* __restrict__ work,
                                                    const __grid_constant__ IoFaces a) {
  const Work w = work[blockIdx.x];
  const DBlock b = blocks[w.block];
  if (w.dir == 0) io_face<0>(w, b, a);
  else if (w.dir == 1) io_face<1>(w, b, a);
  else io_face<2>(w, b, a);
}

cudaError_t launch_io_cells(const DBlock* blocks, const Work* work, int nwork, const void* const* src, void* const* dst,
                            int n, int elem, cudaStream_t st) {
  if (!nwork || !n) return cudaSuccess;
  IoCells a{};
  for (int v = 0; v < n && v < 8; ++v) {
    a.src[v] = src[v];
    a.dst[v] = dst[v];
  }
  a.n = n;
  if (elem == 8) k_io_cells<double><<<nwork, kTile, 0, st>>>(blocks, work, a);
  else k_io_cells<uint8_t><<<nwork, kTile, 0, st>>>(blocks, work, a);
  return cudaGetLastError();
}

cudaError_t launch_io_faces(const DBlock* blocks, const Work* work, int nwork, const double* const src[3],
                            double* const dst[3], cudaStream_t st) {
  if (!nwork) return cudaSuccess;
  IoFaces a{};
  for (int d = 0; d < 3; ++d) {
    a.src[d] = src[d];
    a.dst[d] = dst[d];
  }
  k_io_faces<<<nwork, kTile, 0, st>>>(blocks, work, a);
  return cudaGetLastError();
}

}  // namespace grs
