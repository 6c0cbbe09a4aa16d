// mgr_classes.cu -- coefficient-class layout (arXiv 2105.12764, Sec. I: the
// refactored representation is a series of hierarchically organised
// coefficient classes; a prefix of them rebuilds an approximation).
//
// Class 0 is the coarsest grid N_0, class l the level-l coefficients on
// N_l \ N_{l-1}; the class-packed layout stores them coarsest first, each in
// row-major order of its level grid without the nodes of N_{l-1}.  The level
// kernels write and read that layout directly (mgr_decompose_packed,
// mgr_recompose_packed); this file holds the stand-alone conversions between
// it and the nodal layout and the host queries.
//
// Conversion kernel: one warp per full-grid row (z, y), lanes along x, so the
// nodal side is read / written coalesced.  A full-grid index g of an axis with
// N nodes first appears at level L - min(tz(g), L) (tz = trailing zero bits;
// 0 and N-1 belong to every level), its node at level l has index g >> (L-l)
// (N-1 has the last one), and a node belongs to the class of the finest level
// among its three axes.
#include <cuda_runtime.h>

#include <algorithm>

#include "mgr_internal.h"

namespace mgr {
namespace {

#include "mgr_device.cuh"

struct ClassMap {
  int L;
  int ncls;                 // unpack: classes kept
  int64_t full[kAxes];
  int n[kMaxLevels + 1][kAxes];  // level-l grid sizes, l = 0..L
  int64_t off[kMaxLevels + 2];   // class starts
};

__device__ __forceinline__ int first_level(int64_t g, int64_t N, int L) {
  if (g == 0 || g == N - 1) return 0;
  const int tz = __ffsll(static_cast<long long>(g)) - 1;
  return L - min(tz, L);
}

__device__ __forceinline__ int level_index(int64_t g, int64_t N, int shift, int nl) {
  return g == N - 1 ? nl - 1 : int(g >> shift);
}

// dir 0: pack (nodal -> packed), dir 1: unpack (packed -> nodal)
template <typename T, int DIR>
__global__ void k_classes(const ClassMap cm, const T* __restrict__ src, T* __restrict__ dst) {
  const int64_t rows = cm.full[0] * cm.full[1];
  const int64_t nx = cm.full[2];
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = w0; r < rows; r += nw) {
    const int64_t gz = r / cm.full[1], gy = r - gz * cm.full[1];
    const int lz = first_level(gz, cm.full[0], cm.L), ly = first_level(gy, cm.full[1], cm.L);
    for (int64_t gx = lane; gx < nx; gx += 32) {
      const int l = max(max(lz, ly), first_level(gx, nx, cm.L));
      const int sh = cm.L - l;
      const int n0 = cm.n[l][0], n1 = cm.n[l][1], n2 = cm.n[l][2];
      const int iz = level_index(gz, cm.full[0], sh, n0);
      const int iy = level_index(gy, cm.full[1], sh, n1);
      const int ix = level_index(gx, nx, sh, n2);
      int64_t pos;
      if (l == 0) {
        pos = (int64_t(iz) * n1 + iy) * n2 + ix;
      } else {
        const int m1 = cm.n[l - 1][1], m2 = cm.n[l - 1][2];
        pos = cm.off[l] + int64_t(iz) * n1 * n2 - int64_t(cidx(iz)) * m1 * m2;
        if (!is_coarse(iz, n0)) {
          pos += int64_t(iy) * n2 + ix;
        } else {
          pos += int64_t(iy) * n2 - int64_t(cidx(iy)) * m2 + (is_coarse(iy, n1) ? ix - cidx(ix) : ix);
        }
      }
      const int64_t e = r * nx + gx;
      if (DIR == 0) {
        dst[pos] = src[e];
      } else {
        dst[e] = l < cm.ncls ? src[pos] : T(0);
      }
    }
  }
}

ClassMap class_map(const mgr_plan* p, int ncls) {
  ClassMap cm{};
  cm.L = p->levels;
  cm.ncls = ncls;
  for (int a = 0; a < kAxes; ++a) {
    cm.full[a] = p->full[a];
    cm.n[0][a] = int(p->coarsest[a]);
    for (int l = 1; l <= p->levels; ++l) cm.n[l][a] = p->geom[l].ax[a].n;
  }
  for (int c = 0; c <= p->levels + 1; ++c) cm.off[c] = p->class_off[c];
  return cm;
}

template <int DIR>
cudaError_t launch(const mgr_plan* p, const void* src, void* dst, int ncls, cudaStream_t st) {
  const ClassMap cm = class_map(p, ncls);
  const int64_t rows = p->full[0] * p->full[1];
  const int threads = 256;
  const int64_t want = (rows + 7) / 8;
  const int blocks = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(p->ctx->num_sms) * 16)));
  if (p->elem == 8)
    k_classes<double, DIR><<<blocks, threads, 0, st>>>(cm, static_cast<const double*>(src), static_cast<double*>(dst));
  else
    k_classes<float, DIR><<<blocks, threads, 0, st>>>(cm, static_cast<const float*>(src), static_cast<float*>(dst));
  return cudaGetLastError();
}

bool overlap(const void* a, const void* b, size_t n) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + n && pb < pa + n;
}

int check(const mgr_plan* p, const void* a, const void* b) {
  if (!p || !a || !b || p->desc.ndim == 4) return MGR_EINVAL;
  if ((reinterpret_cast<uintptr_t>(a) % p->elem) || (reinterpret_cast<uintptr_t>(b) % p->elem)) return MGR_EINVAL;
  if (overlap(a, b, size_t(p->count) * p->elem)) return MGR_EINVAL;
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return MGR_ECUDA;
  }
  return MGR_OK;
}

}  // namespace

cudaError_t enqueue_pack_classes(const mgr_plan* p, const void* nodal, void* packed, cudaStream_t st) {
  return launch<0>(p, nodal, packed, p->levels + 1, st);
}

cudaError_t enqueue_unpack_classes(const mgr_plan* p, const void* packed, int ncls, void* nodal, cudaStream_t st) {
  return launch<1>(p, packed, nodal, ncls, st);
}

}  // namespace mgr

extern "C" {

int mgr_class_offsets(const mgr_plan* p, int64_t* offsets, int cap, int* nclasses) {
  if (!p || !nclasses || (cap > 0 && !offsets) || p->desc.ndim == 4) return MGR_EINVAL;
  const int n = p->levels + 2;
  for (int i = 0; i < std::min(cap, n); ++i) offsets[i] = p->class_off[i];
  *nclasses = p->levels + 1;
  return MGR_OK;
}

int mgr_pack_classes(const mgr_plan* p, const void* nodal, void* packed, mgr_stream_t stream) {
  const int rc = mgr::check(p, nodal, packed);
  if (rc != MGR_OK) return rc;
  return mgr::enqueue_pack_classes(p, nodal, packed, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? MGR_OK
             : MGR_ECUDA;
}

int mgr_unpack_classes(const mgr_plan* p, const void* packed, int nclasses, void* nodal, mgr_stream_t stream) {
  const int rc = mgr::check(p, packed, nodal);
  if (rc != MGR_OK) return rc;
  if (nclasses < 1 || nclasses > p->levels + 1) return MGR_EINVAL;
  return mgr::enqueue_unpack_classes(p, packed, nclasses, nodal, reinterpret_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? MGR_OK
             : MGR_ECUDA;
}

}  // extern "C"
