// mgr_core.cu -- sm_103a kernels and level loops of the multigrid
// decomposition / recomposition (arXiv 2105.12764, Sec. II.A, III.A).
//
// One decomposition level l (n nodes -> m coarse nodes) is three kinds of
// launches (the paper's GPK / LPK / IPK roles, redesigned):
//
//   k_level_load   coefficients (Sec. II.A.1) and the load vector
//                  f' = (x_k D_k^-1 P_k^T M_k) c (Sec. II.A.2, III.A.2) in one
//                  pass.  A CTA owns a (BY x BX) tile of coarse (y, x) nodes and
//                  a chunk of coarse z planes; it streams the fine z planes of
//                  its tile region (with a two-node halo for the 5-tap stencil)
//                  through shared memory with cp.async double buffering,
//                  computes the coefficients of each plane, writes them to the
//                  nodal output, applies the x and y stencils in shared memory
//                  and accumulates the z stencil in registers.  The coarse nodal
//                  values go to a compact coarse workspace.
//   k_solve_*      the Thomas recurrences along one axis of the compact coarse
//                  grid (Sec. III.A.3).  Strided axes: one thread per line,
//                  coalesced across the contiguous axis.  The contiguous axis:
//                  lines staged in shared memory.  The last solve of a level
//                  adds (decompose) or subtracts (recompose) the correction
//                  into the coarse workspace (Eq. (1)).
//   k_interp       recomposition only: v = c + interpolant of the coarse nodes.
//
// Arithmetic: TS is the stencil type (coefficients, interpolation, K), TW the
// solve / coarse-workspace type; (double, double) for FP64, (float, float) for
// FP32, (float, double) for the mixed precision form.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>

#include "mgr_internal.h"

namespace mgr {

thread_local Recorder* t_recorder = nullptr;

namespace {

// Optional per-launch CUDA-event instrumentation (mgr_profile).
inline void rec_begin(cudaStream_t st) {
  if (!t_recorder) return;
  LaunchRecord r{};
  cudaEventCreate(&r.start);
  cudaEventCreate(&r.stop);
  cudaEventRecord(r.start, st);
  t_recorder->launches.push_back(r);
}
inline void rec_end(cudaStream_t st, const char* name, int level, double bytes, double flops) {
  if (!t_recorder) return;
  LaunchRecord& r = t_recorder->launches.back();
  cudaEventRecord(r.stop, st);
  std::snprintf(r.name, sizeof(r.name), "%s", name);
  r.level = level;
  r.bytes = bytes;
  r.flops = flops;
}

constexpr int BX = 32;   // coarse x nodes per CTA tile (one warp across x)
constexpr int BY = 8;    // coarse y nodes per CTA tile
constexpr int NT = BX * BY;
constexpr int RXMAX = 2 * BX + 3;  // fine region width incl. halo (5-tap stencil)
constexpr int RYMAX = 2 * BY + 3;
constexpr int RXP = RXMAX + 1;     // shared-memory row pitch
constexpr int PLANE = RYMAX * RXP;

__device__ __forceinline__ int pidx(int q, int n) { return min(2 * q, n - 1); }
__device__ __forceinline__ bool is_coarse(int i, int n) { return ((i & 1) == 0) || (i == n - 1); }
__device__ __forceinline__ int cidx(int i) { return (i + 1) >> 1; }
// first fine node of the stencil region of coarse node q0, moved down to a coarse node
__device__ __forceinline__ int region_start(int q0, int n) {
  const int r = pidx(q0, n) - 2;
  return (r & 1) ? r - 1 : r;
}
__device__ __forceinline__ int64_t fmap(int i, int64_t s, int64_t N) {
  int64_t f = int64_t(i) * s;
  return f < N - 1 ? f : N - 1;
}

__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes) {
  unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------
// k_level_load
// ---------------------------------------------------------------------------

template <typename TS, typename TW>
struct LoadArgs {
  const void* in;      // DEC: level-l values; REC: nodal coefficients (full grid)
  int64_t in_sz, in_sy;
  int in_full;         // 1: index `in` through the full-grid map min(i*s, N-1)
  void* y;             // DEC: nodal output (full grid)
  int64_t y_sz, y_sy;
  TW* w;               // DEC: coarse nodal values (compact m grid)
  TW* f;               // load vector (compact m grid)
  int64_t c_sz, c_sy;
  int n[3], m[3];
  int64_t s[3], N[3];
  const TS* wa[3];
  const TS* wb[3];
  const TS* k[3];
  int qz_chunk;
  int write_y;
};

enum { MODE_DEC = 0, MODE_REC = 1 };

template <int MODE, typename TI, typename TD, typename TS, typename TW>
__global__ void __launch_bounds__(NT, 2) k_level_load(const LoadArgs<TS, TW> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TI* raw = reinterpret_cast<TI*>(smem_raw);                        // [2 stages][2 planes][PLANE]
  TS* Ibuf = reinterpret_cast<TS*>(smem_raw + sizeof(TI) * 4 * PLANE);  // [2][PLANE]
  TS* cb = Ibuf + 2 * PLANE;                                          // [PLANE]
  TS* gxb = cb + PLANE;                                               // [RYMAX][BX]

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int nz = a.n[0], ny = a.n[1], nx = a.n[2];
  const int mz = a.m[0], my = a.m[1], mx = a.m[2];
  const int qx0 = blockIdx.x * BX, qx1 = min(qx0 + BX, mx);
  const int qy0 = blockIdx.y * BY, qy1 = min(qy0 + BY, my);
  const int qz0 = blockIdx.z * a.qz_chunk, qz1 = min(qz0 + a.qz_chunk, mz);
  // the region starts on a coarse node so every fine node in it has both
  // interpolation neighbours inside; pidx(q0) - 2 is fine only in the
  // keep-last case (q0 = m-1, n even), where one more node is taken
  const int rx0 = max(region_start(qx0, nx), 0), rx1 = min(pidx(qx1 - 1, nx) + 2, nx - 1);
  const int ry0 = max(region_start(qy0, ny), 0), ry1 = min(pidx(qy1 - 1, ny) + 2, ny - 1);
  const int RX = rx1 - rx0 + 1, RY = ry1 - ry0 + 1, RE = RX * RY;
  // owned fine ranges (each fine node is written by exactly one CTA)
  const int ox0 = pidx(qx0, nx), ox1 = (qx1 == mx) ? nx : pidx(qx1, nx);
  const int oy0 = pidx(qy0, ny), oy1 = (qy1 == my) ? ny : pidx(qy1, ny);
  // first coarse plane streamed: the one before the chunk, or two before it
  // when the chunk starts at a keep-last coarse plane (then the fine plane
  // pidx(qz0) - 2 and its interpolation planes are needed)
  int t_start = qz0 > 0 ? qz0 - 1 : 0;
  if (qz0 >= 2 && pidx(qz0, nz) - pidx(qz0 - 1, nz) == 1) t_start = qz0 - 2;
  const int t_end = min(qz1, mz - 1);

  const TI* in = static_cast<const TI*>(a.in);
  const TS* wax = a.wa[2]; const TS* wbx = a.wb[2];
  const TS* way = a.wa[1]; const TS* wby = a.wb[1];
  const TS* waz = a.wa[0]; const TS* wbz = a.wb[0];
  const TS* kx = a.k[2]; const TS* ky = a.k[1]; const TS* kz = a.k[0];

  auto in_off = [&](int gz, int gy, int gx) -> int64_t {
    if (a.in_full)
      return fmap(gz, a.s[0], a.N[0]) * a.in_sz + fmap(gy, a.s[1], a.N[1]) * a.in_sy + fmap(gx, a.s[2], a.N[2]);
    return int64_t(gz) * a.in_sz + int64_t(gy) * a.in_sy + gx;
  };
  auto load_plane = [&](TI* dst, int gz) {
    for (int e = tid; e < RE; e += NT) {
      const int r = e / RX, c = e - r * RX;
      cp_async(dst + r * RXP + c, in + in_off(gz, ry0 + r, rx0 + c), int(sizeof(TI)));
    }
  };
  auto plane_has_fine = [&](int t) { return t > t_start && (pidx(t, nz) - pidx(t - 1, nz) == 2); };
  auto issue = [&](int t) {
    TI* st = raw + ((t - t_start) & 1) * 2 * PLANE;
    load_plane(st, pidx(t, nz));
    if (plane_has_fine(t)) load_plane(st + PLANE, pidx(t, nz) - 1);
    cp_commit();
  };

  // K_z accumulators for coarse planes t-1, t, t+1
  const int qy = qy0 + ty, qx = qx0 + tx;
  const bool own = (qy < qy1) && (qx < qx1);
  TS acc0 = TS(0), acc1 = TS(0), acc2 = TS(0);
  TS* Iprev = Ibuf;
  TS* Inext = Ibuf + PLANE;

  // x then y stencil of the plane in cb, result for (qy, qx) returned
  auto stencil_xy = [&]() -> TS {
    if (qx < qx1) {
      const int p = pidx(qx, nx);
      const TS* kr = kx + 5 * qx;
      for (int r = ty; r < RY; r += BY) {
        TS s = TS(0);
#pragma unroll
        for (int o = -2; o <= 2; ++o) {
          const int j = p + o;
          if (j >= 0 && j < nx) s += kr[o + 2] * cb[r * RXP + (j - rx0)];
        }
        gxb[r * BX + tx] = s;
      }
    }
    __syncthreads();
    TS g = TS(0);
    if (own) {
      const int p = pidx(qy, ny);
      const TS* kr = ky + 5 * qy;
#pragma unroll
      for (int o = -2; o <= 2; ++o) {
        const int j = p + o;
        if (j >= 0 && j < ny) g += kr[o + 2] * gxb[(j - ry0) * BX + tx];
      }
    }
    return g;
  };
  auto accumulate_z = [&](int t, int gz, TS g) {
    // contributions of fine plane gz to coarse planes t-1, t, t+1
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
      const int q = t + d;
      if (q < qz0 || q >= qz1) continue;
      const int off = gz - pidx(q, nz);
      if (off < -2 || off > 2) continue;
      const TS wgt = kz[5 * q + off + 2];
      if (d == -1) acc0 += wgt * g;
      else if (d == 0) acc1 += wgt * g;
      else acc2 += wgt * g;
    }
  };
  auto store_y = [&](int gz, const TI* vplane, bool zc) {
    if (MODE != MODE_DEC || !a.write_y) return;
    TD* y = static_cast<TD*>(a.y);
    const int64_t zoff = fmap(gz, a.s[0], a.N[0]) * a.y_sz;
    for (int e = tid; e < RE; e += NT) {
      const int r = e / RX, c = e - r * RX;
      const int gy = ry0 + r, gx = rx0 + c;
      if (gy < oy0 || gy >= oy1 || gx < ox0 || gx >= ox1) continue;
      const bool allc = zc && is_coarse(gy, ny) && is_coarse(gx, nx);
      // all-coarse nodes get their (uncorrected) value as a placeholder that a
      // coarser level overwrites; it keeps the row's sectors fully written.
      const TS v = allc ? TS(vplane[r * RXP + c]) : cb[r * RXP + c];
      y[zoff + fmap(gy, a.s[1], a.N[1]) * a.y_sy + fmap(gx, a.s[2], a.N[2])] = TD(v);
    }
  };

  issue(t_start);
  for (int t = t_start; t <= t_end; ++t) {
    if (t < t_end) {
      issue(t + 1);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    const TI* vc = raw + ((t - t_start) & 1) * 2 * PLANE;
    const TI* vf = vc + PLANE;
    const int Pc = pidx(t, nz);
    const bool has_f = plane_has_fine(t);
    const bool owned_c = (t >= qz0) && (t < qz1);
    // ---- coarse-in-z plane Pc: xy interpolant and coefficients
    for (int e = tid; e < RE; e += NT) {
      const int r = e / RX, c = e - r * RX;
      const int gy = ry0 + r, gx = rx0 + c;
      const bool yc = is_coarse(gy, ny), xc = is_coarse(gx, nx);
      if (MODE == MODE_DEC) {
        const TS v = TS(vc[r * RXP + c]);
        TS I;
        if (yc && xc) {
          I = v;
        } else if (yc) {
          I = wax[gx] * TS(vc[r * RXP + c - 1]) + wbx[gx] * TS(vc[r * RXP + c + 1]);
        } else if (xc) {
          I = way[gy] * TS(vc[(r - 1) * RXP + c]) + wby[gy] * TS(vc[(r + 1) * RXP + c]);
        } else {
          const TS lo = wax[gx] * TS(vc[(r - 1) * RXP + c - 1]) + wbx[gx] * TS(vc[(r - 1) * RXP + c + 1]);
          const TS hi = wax[gx] * TS(vc[(r + 1) * RXP + c - 1]) + wbx[gx] * TS(vc[(r + 1) * RXP + c + 1]);
          I = way[gy] * lo + wby[gy] * hi;
        }
        Inext[r * RXP + c] = I;
        cb[r * RXP + c] = v - I;
      } else {
        cb[r * RXP + c] = (yc && xc) ? TS(0) : TS(vc[r * RXP + c]);
      }
    }
    __syncthreads();
    if (owned_c) store_y(Pc, vc, true);
    {
      const TS g = stencil_xy();
      accumulate_z(t, Pc, g);
    }
    if (MODE == MODE_DEC && owned_c && own) {
      const int gy = pidx(qy, ny), gx = pidx(qx, nx);
      a.w[int64_t(t) * a.c_sz + int64_t(qy) * a.c_sy + qx] = TW(vc[(gy - ry0) * RXP + (gx - rx0)]);
    }
    __syncthreads();
    // ---- fine-in-z plane Pc-1
    if (has_f) {
      const int Pf = Pc - 1;
      const bool owned_f = (t > qz0) && (t <= qz1);
      if (MODE == MODE_DEC) {
        const TS za = waz[Pf], zb = wbz[Pf];
        for (int e = tid; e < RE; e += NT) {
          const int r = e / RX, c = e - r * RX;
          cb[r * RXP + c] = TS(vf[r * RXP + c]) - (za * Iprev[r * RXP + c] + zb * Inext[r * RXP + c]);
        }
      } else {
        for (int e = tid; e < RE; e += NT) {
          const int r = e / RX, c = e - r * RX;
          cb[r * RXP + c] = TS(vf[r * RXP + c]);
        }
      }
      __syncthreads();
      if (owned_f) store_y(Pf, vf, false);
      const TS g = stencil_xy();
      accumulate_z(t, Pf, g);
      __syncthreads();
    }
    // coarse plane t-1 is complete
    if (own && t - 1 >= qz0 && t - 1 < qz1) a.f[int64_t(t - 1) * a.c_sz + int64_t(qy) * a.c_sy + qx] = TW(acc0);
    acc0 = acc1;
    acc1 = acc2;
    acc2 = TS(0);
    TS* tmp = Iprev;
    Iprev = Inext;
    Inext = tmp;
  }
  if (own && t_end == mz - 1 && qz1 == mz) a.f[int64_t(mz - 1) * a.c_sz + int64_t(qy) * a.c_sy + qx] = TW(acc0);
}

template <typename TI, typename TS>
constexpr size_t load_smem_bytes() {
  return sizeof(TI) * 4 * PLANE + sizeof(TS) * (3 * PLANE + RYMAX * BX);
}

// ---------------------------------------------------------------------------
// In-place decomposition of the finest level: coefficients written pointwise
// (the load pass ran first with write_y = 0).  Only fine nodes are written and
// every value read is either the node itself or an all-coarse node, so the
// kernel can run on the array it reads.
// ---------------------------------------------------------------------------
template <typename TD, typename TS>
__global__ void k_coef_inplace(TD* y, int nz, int ny, int nx, const TS* waz, const TS* wbz, const TS* way,
                               const TS* wby, const TS* wax, const TS* wbx) {
  const int64_t total = int64_t(nz) * ny * nx;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int gx = int(e % nx);
    const int64_t rest = e / nx;
    const int gy = int(rest % ny), gz = int(rest / ny);
    const bool zc = is_coarse(gz, nz), yc = is_coarse(gy, ny), xc = is_coarse(gx, nx);
    if (zc && yc && xc) continue;
    const int64_t sz = int64_t(ny) * nx, sy = nx;
    auto ixy = [&](int z) -> TS {
      const TD* p = y + int64_t(z) * sz;
      if (yc && xc) return TS(p[int64_t(gy) * sy + gx]);
      if (yc) return wax[gx] * TS(p[int64_t(gy) * sy + gx - 1]) + wbx[gx] * TS(p[int64_t(gy) * sy + gx + 1]);
      if (xc) return way[gy] * TS(p[int64_t(gy - 1) * sy + gx]) + wby[gy] * TS(p[int64_t(gy + 1) * sy + gx]);
      const TS lo = wax[gx] * TS(p[int64_t(gy - 1) * sy + gx - 1]) + wbx[gx] * TS(p[int64_t(gy - 1) * sy + gx + 1]);
      const TS hi = wax[gx] * TS(p[int64_t(gy + 1) * sy + gx - 1]) + wbx[gx] * TS(p[int64_t(gy + 1) * sy + gx + 1]);
      return way[gy] * lo + wby[gy] * hi;
    };
    const TS v = TS(y[e]);
    TS c;
    if (zc) c = v - ixy(gz);
    else c = v - (waz[gz] * ixy(gz - 1) + wbz[gz] * ixy(gz + 1));
    y[e] = TD(c);
  }
}

// ---------------------------------------------------------------------------
// Thomas recurrences (scaled LU, one FMA per step and direction)
// ---------------------------------------------------------------------------
enum { SOLVE_INPLACE = 0, SOLVE_ADD = 1, SOLVE_SUB = 2 };

// Lines along a strided axis: element q of line (o, i) at o*ostride + i + q*lstride.
template <typename TW, int OP>
__global__ void __launch_bounds__(256) k_solve_strided(TW* __restrict__ f, TW* __restrict__ w, int mline,
                                                       int64_t lstride, int inner, int64_t outer, int64_t ostride,
                                                       const TW* __restrict__ ta, const TW* __restrict__ tb) {
  const int64_t id = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (id >= int64_t(inner) * outer) return;
  const int i = int(id % inner);
  const int64_t o = id / inner;
  TW* fl = f + o * ostride + i;
  constexpr int U = 8;
  TW prev = TW(0);
  for (int q0 = 0; q0 < mline; q0 += U) {
    TW buf[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (q0 + u < mline) buf[u] = fl[int64_t(q0 + u) * lstride];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (q0 + u < mline) {
        prev = buf[u] - ta[q0 + u] * prev;
        fl[int64_t(q0 + u) * lstride] = prev;
      }
  }
  TW* wl = w + o * ostride + i;
  TW next = TW(0);
  for (int q1 = mline - 1; q1 >= 0; q1 -= U) {
    TW buf[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (q1 - u >= 0) buf[u] = fl[int64_t(q1 - u) * lstride];
    TW wv[U];
    if (OP != SOLVE_INPLACE) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (q1 - u >= 0) wv[u] = wl[int64_t(q1 - u) * lstride];
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (q1 - u >= 0) {
        const int q = q1 - u;
        next = buf[u] - tb[q] * next;
        if (OP == SOLVE_INPLACE) fl[int64_t(q) * lstride] = next;
        else if (OP == SOLVE_ADD) wl[int64_t(q) * lstride] = wv[u] + next;
        else wl[int64_t(q) * lstride] = wv[u] - next;
      }
  }
}

// Lines along the contiguous axis: R rows of length mline staged in shared
// memory (coalesced load/store), one thread per row for the recurrences.
template <typename TW, int OP>
__global__ void k_solve_contig(TW* __restrict__ f, TW* __restrict__ w, int mline, int64_t rows, int64_t row_pitch,
                               int R, const TW* __restrict__ ta, const TW* __restrict__ tb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TW* s = reinterpret_cast<TW*>(smem_raw);
  const int pitch = mline | 1;  // odd pitch spreads rows over banks
  const int64_t r0 = blockIdx.x * int64_t(R);
  const int nr = int(rows - r0 < int64_t(R) ? rows - r0 : int64_t(R));
  for (int e = threadIdx.x; e < nr * mline; e += blockDim.x) {
    const int r = e / mline, c = e - r * mline;
    s[r * pitch + c] = f[(r0 + r) * row_pitch + c];
  }
  __syncthreads();
  if (threadIdx.x < nr) {
    TW* l = s + threadIdx.x * pitch;
    TW prev = TW(0);
    for (int q = 0; q < mline; ++q) {
      prev = l[q] - ta[q] * prev;
      l[q] = prev;
    }
    TW next = TW(0);
    for (int q = mline - 1; q >= 0; --q) {
      next = l[q] - tb[q] * next;
      l[q] = next;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nr * mline; e += blockDim.x) {
    const int r = e / mline, c = e - r * mline;
    const int64_t g = (r0 + r) * row_pitch + c;
    if (OP == SOLVE_INPLACE) f[g] = s[r * pitch + c];
    else if (OP == SOLVE_ADD) w[g] = w[g] + s[r * pitch + c];
    else w[g] = w[g] - s[r * pitch + c];
  }
}

// ---------------------------------------------------------------------------
// Recompose: v = c + (P_z x P_y x P_x) v_coarse at every level-l node
// ---------------------------------------------------------------------------
template <typename TD, typename TO, typename TS, typename TW>
__global__ void k_interp(const TD* __restrict__ y, int64_t y_sz, int64_t y_sy, int3 n, longlong3 s, longlong3 N,
                         const TW* __restrict__ w, int64_t c_sz, int64_t c_sy, TO* __restrict__ out, int64_t o_sz,
                         int64_t o_sy, const TS* waz, const TS* wbz, const TS* way, const TS* wby, const TS* wax,
                         const TS* wbx) {
  const int64_t total = int64_t(n.x) * n.y * n.z;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int gx = int(e % n.z);
    const int64_t rest = e / n.z;
    const int gy = int(rest % n.y), gz = int(rest / n.y);
    int qz[2], qy[2], qx[2];
    TS wz[2], wy[2], wx[2];
    int cz, cy, cx;
    auto axis = [&](int g, int nn, const TS* wa, const TS* wb, int* q, TS* wt, int& cnt) {
      if (is_coarse(g, nn)) {
        q[0] = cidx(g); wt[0] = TS(1); cnt = 1;
      } else {
        q[0] = cidx(g - 1); wt[0] = wa[g];
        q[1] = cidx(g + 1); wt[1] = wb[g];
        cnt = 2;
      }
    };
    axis(gz, n.x, waz, wbz, qz, wz, cz);
    axis(gy, n.y, way, wby, qy, wy, cy);
    axis(gx, n.z, wax, wbx, qx, wx, cx);
    TS I = TS(0);
    for (int a = 0; a < cz; ++a) {
      TS Iy = TS(0);
      for (int b = 0; b < cy; ++b) {
        const TW* row = w + int64_t(qz[a]) * c_sz + int64_t(qy[b]) * c_sy;
        TS Ix = (cx == 1) ? TS(row[qx[0]]) : wx[0] * TS(row[qx[0]]) + wx[1] * TS(row[qx[1]]);
        Iy = (cy == 1) ? Ix : (b == 0 ? wy[0] * Ix : Iy + wy[1] * Ix);
      }
      I = (cz == 1) ? Iy : (a == 0 ? wz[0] * Iy : I + wz[1] * Iy);
    }
    const bool allc = (cz == 1) && (cy == 1) && (cx == 1);
    TS c = TS(0);
    if (!allc) c = TS(y[fmap(gz, s.x, N.x) * y_sz + fmap(gy, s.y, N.y) * y_sy + fmap(gx, s.z, N.z)]);
    out[int64_t(gz) * o_sz + int64_t(gy) * o_sy + gx] = TO(c + I);
  }
}

// Coarsest grid <-> nodal positions (dir 0: gather nodal -> compact; 1: scatter)
template <typename TD, typename TW>
__global__ void k_coarsest(TD* y, int64_t y_sz, int64_t y_sy, TW* w, int3 n, longlong3 s, longlong3 N, int dir) {
  const int64_t total = int64_t(n.x) * n.y * n.z;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int gx = int(e % n.z);
    const int64_t rest = e / n.z;
    const int gy = int(rest % n.y), gz = int(rest / n.y);
    const int64_t yo = fmap(gz, s.x, N.x) * y_sz + fmap(gy, s.y, N.y) * y_sy + fmap(gx, s.z, N.z);
    if (dir == 0) w[e] = TW(y[yo]);
    else y[yo] = TD(w[e]);
  }
}

// ---------------------------------------------------------------------------
// Host-side level loops
// ---------------------------------------------------------------------------

template <typename T>
const T* table(const mgr_plan* p);
template <>
const double* table<double>(const mgr_plan* p) { return p->tables.d64; }
template <>
const float* table<float>(const mgr_plan* p) { return p->tables.d32; }

inline int grid_1d(int64_t total, int block, const mgr_plan* p) {
  int64_t g = (total + block - 1) / block;
  int64_t cap = int64_t(p->ctx->num_sms) * 32;
  return int(std::max<int64_t>(1, std::min(g, cap)));
}

struct Bufs {
  void* A;
  void* B;
  void* F;
};

inline Bufs split_ws(const mgr_plan* p, void* ws) {
  char* b = static_cast<char*>(ws);
  return Bufs{b, b + p->ws_a, b + p->ws_a + p->ws_b};
}

template <typename TS, typename TW>
LoadArgs<TS, TW> load_args(const mgr_plan* p, int l) {
  const LevelGeom& g = p->geom[l];
  LoadArgs<TS, TW> a{};
  const TS* T = table<TS>(p);
  for (int k = 0; k < 3; ++k) {
    a.n[k] = g.ax[k].n;
    a.m[k] = g.ax[k].m;
    a.s[k] = g.ax[k].s;
    a.N[k] = g.ax[k].N;
    a.wa[k] = T + g.ax[k].o_wa;
    a.wb[k] = T + g.ax[k].o_wb;
    a.k[k] = T + g.ax[k].o_k;
  }
  a.y_sz = p->full[1] * p->full[2];
  a.y_sy = p->full[2];
  a.c_sz = int64_t(g.ax[1].m) * g.ax[2].m;
  a.c_sy = g.ax[2].m;
  return a;
}

template <typename TS, typename TW>
dim3 load_grid(const mgr_plan* p, LoadArgs<TS, TW>& a) {
  const int gx = (a.m[2] + BX - 1) / BX, gy = (a.m[1] + BY - 1) / BY;
  // enough CTAs for ~2 waves at 2 CTAs/SM; each chunk streams >= 4 coarse planes
  const int64_t want = int64_t(p->ctx->num_sms) * 4;
  int chunks = int(std::max<int64_t>(1, want / std::max(1, gx * gy)));
  chunks = std::min(chunks, std::max(1, a.m[0] / 4));
  a.qz_chunk = (a.m[0] + chunks - 1) / chunks;
  const int gz = (a.m[0] + a.qz_chunk - 1) / a.qz_chunk;
  return dim3(gx, gy, gz);
}

template <typename TW>
cudaError_t solve_axis_launch(const mgr_plan* p, int l, int axis, TW* f, TW* w, int op, cudaStream_t st);

template <typename TW>
cudaError_t solve_axis(const mgr_plan* p, int l, int axis, TW* f, TW* w, int op, cudaStream_t st) {
  const Work wk = work_solve(p, l, axis, op != SOLVE_INPLACE);
  static const char* names[3] = {"solve_z", "solve_y", "solve_x"};
  rec_begin(st);
  cudaError_t err = solve_axis_launch<TW>(p, l, axis, f, w, op, st);
  rec_end(st, names[axis], l, wk.bytes, wk.flops);
  return err;
}

template <typename TW>
cudaError_t solve_axis_launch(const mgr_plan* p, int l, int axis, TW* f, TW* w, int op, cudaStream_t st) {
  const LevelGeom& g = p->geom[l];
  const int mz = g.ax[0].m, my = g.ax[1].m, mx = g.ax[2].m;
  const TW* T = table<TW>(p);
  const TW* ta = T + g.ax[axis].o_ta;
  const TW* tb = T + g.ax[axis].o_tb;
  if (axis == 2) {
    const int64_t rows = int64_t(mz) * my;
    const int pitch = mx | 1;
    int R = int(std::min<size_t>(32, (96 * 1024) / (sizeof(TW) * pitch)));
    R = std::max(R, 1);
    const size_t sm = sizeof(TW) * size_t(R) * pitch;
    const int blocks = int((rows + R - 1) / R);
    const int threads = 128;
    if (op == SOLVE_INPLACE) {
      cudaFuncSetAttribute(k_solve_contig<TW, SOLVE_INPLACE>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
      k_solve_contig<TW, SOLVE_INPLACE><<<blocks, threads, sm, st>>>(f, w, mx, rows, mx, R, ta, tb);
    } else if (op == SOLVE_ADD) {
      cudaFuncSetAttribute(k_solve_contig<TW, SOLVE_ADD>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
      k_solve_contig<TW, SOLVE_ADD><<<blocks, threads, sm, st>>>(f, w, mx, rows, mx, R, ta, tb);
    } else {
      cudaFuncSetAttribute(k_solve_contig<TW, SOLVE_SUB>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
      k_solve_contig<TW, SOLVE_SUB><<<blocks, threads, sm, st>>>(f, w, mx, rows, mx, R, ta, tb);
    }
    return cudaGetLastError();
  }
  int mline, inner;
  int64_t lstride, outer, ostride;
  if (axis == 1) {
    mline = my; lstride = mx; inner = mx; outer = mz; ostride = int64_t(my) * mx;
  } else {
    mline = mz; lstride = int64_t(my) * mx; inner = mx; outer = my; ostride = mx;
  }
  const int64_t lines = int64_t(inner) * outer;
  const int threads = 128;
  const int blocks = int((lines + threads - 1) / threads);
  if (op == SOLVE_INPLACE)
    k_solve_strided<TW, SOLVE_INPLACE><<<blocks, threads, 0, st>>>(f, w, mline, lstride, inner, outer, ostride, ta, tb);
  else if (op == SOLVE_ADD)
    k_solve_strided<TW, SOLVE_ADD><<<blocks, threads, 0, st>>>(f, w, mline, lstride, inner, outer, ostride, ta, tb);
  else
    k_solve_strided<TW, SOLVE_SUB><<<blocks, threads, 0, st>>>(f, w, mline, lstride, inner, outer, ostride, ta, tb);
  return cudaGetLastError();
}

// solve along every active axis, x first; the last one applies `final_op` into w
template <typename TW>
cudaError_t solve_level(const mgr_plan* p, int l, TW* f, TW* w, int final_op, cudaStream_t st) {
  const LevelGeom& g = p->geom[l];
  int last = -1;
  for (int axis = 2; axis >= 0; --axis)
    if (g.ax[axis].active) last = axis;
  for (int axis = 2; axis >= 0; --axis) {
    if (!g.ax[axis].active) continue;
    cudaError_t e = solve_axis<TW>(p, l, axis, f, w, axis == last ? final_op : SOLVE_INPLACE, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename TD, typename TS, typename TW>
cudaError_t decompose_t(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st) {
  const int L = p->levels;
  const size_t bytes = size_t(p->count) * sizeof(TD);
  if (L == 0) {
    if (in != out) return cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, st);
    return cudaSuccess;
  }
  const bool inplace = (in == out);
  Bufs b = split_ws(p, ws);
  TW* F = static_cast<TW*>(b.F);
  TW* cur = nullptr;  // compact level-l values for l < L
  for (int l = L; l >= 1; --l) {
    TW* nxt = static_cast<TW*>(((L - l) % 2 == 0) ? b.A : b.B);
    auto a = load_args<TS, TW>(p, l);
    a.y = out;
    a.w = nxt;
    a.f = F;
    a.write_y = (l == L && inplace) ? 0 : 1;
    dim3 grid = load_grid(p, a);
    dim3 block(BX, BY);
    if (l == L) {
      a.in = in;
      a.in_full = 1;
      a.in_sz = a.y_sz;
      a.in_sy = a.y_sy;
      constexpr size_t sm = load_smem_bytes<TD, TS>();
      cudaFuncSetAttribute(k_level_load<MODE_DEC, TD, TD, TS, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
      rec_begin(st);
      k_level_load<MODE_DEC, TD, TD, TS, TW><<<grid, block, sm, st>>>(a);
    } else {
      const LevelGeom& g = p->geom[l];
      a.in = cur;
      a.in_full = 0;
      a.in_sz = int64_t(g.ax[1].n) * g.ax[2].n;
      a.in_sy = g.ax[2].n;
      constexpr size_t sm = load_smem_bytes<TW, TS>();
      cudaFuncSetAttribute(k_level_load<MODE_DEC, TW, TD, TS, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
      rec_begin(st);
      k_level_load<MODE_DEC, TW, TD, TS, TW><<<grid, block, sm, st>>>(a);
    }
    cudaError_t e = cudaGetLastError();
    {
      const Work wk = work_level_load(p, l, true);
      rec_end(st, "level_load_dec", l, wk.bytes, wk.flops);
    }
    if (e != cudaSuccess) return e;
    if (l == L && inplace) {
      const LevelGeom& g = p->geom[l];
      const TS* T = table<TS>(p);
      const int64_t total = g.fine_count();
      rec_begin(st);
      k_coef_inplace<TD, TS><<<grid_1d(total, 256, p), 256, 0, st>>>(
          static_cast<TD*>(out), g.ax[0].n, g.ax[1].n, g.ax[2].n, T + g.ax[0].o_wa, T + g.ax[0].o_wb,
          T + g.ax[1].o_wa, T + g.ax[1].o_wb, T + g.ax[2].o_wa, T + g.ax[2].o_wb);
      e = cudaGetLastError();
      {
        const Work wi = work_interp(p, l);
        rec_end(st, "coef_inplace", l, 2.0 * double(total) * sizeof(TD), wi.flops);
      }
      if (e != cudaSuccess) return e;
    }
    if ((e = solve_level<TW>(p, l, F, nxt, SOLVE_ADD, st)) != cudaSuccess) return e;
    cur = nxt;
  }
  // coarsest values into their nodal positions
  const int3 n0 = make_int3(int(p->coarsest[0]), int(p->coarsest[1]), int(p->coarsest[2]));
  const int64_t s0 = int64_t(1) << L;
  const longlong3 s = make_longlong3(p->full[0] > 1 ? s0 : 1, p->full[1] > 1 ? s0 : 1, s0);
  const longlong3 N = make_longlong3(p->full[0], p->full[1], p->full[2]);
  const int64_t total = int64_t(n0.x) * n0.y * n0.z;
  rec_begin(st);
  k_coarsest<TD, TW><<<grid_1d(total, 256, p), 256, 0, st>>>(static_cast<TD*>(out), p->full[1] * p->full[2],
                                                               p->full[2], cur, n0, s, N, 1);
  cudaError_t e = cudaGetLastError();
  rec_end(st, "coarsest", 0, double(total) * (sizeof(TD) + sizeof(TW)), 0.0);
  return e;
}

template <typename TD, typename TS, typename TW>
cudaError_t recompose_t(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st) {
  const int L = p->levels;
  const size_t bytes = size_t(p->count) * sizeof(TD);
  if (L == 0) {
    if (in != out) return cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, st);
    return cudaSuccess;
  }
  Bufs b = split_ws(p, ws);
  TW* F = static_cast<TW*>(b.F);
  // coarsest grid from the nodal positions
  TW* cur = static_cast<TW*>((L % 2 == 1) ? b.A : b.B);  // level 0 lives where decompose left it
  {
    const int3 n0 = make_int3(int(p->coarsest[0]), int(p->coarsest[1]), int(p->coarsest[2]));
    const int64_t s0 = int64_t(1) << L;
    const longlong3 s = make_longlong3(p->full[0] > 1 ? s0 : 1, p->full[1] > 1 ? s0 : 1, s0);
    const longlong3 N = make_longlong3(p->full[0], p->full[1], p->full[2]);
    const int64_t total = int64_t(n0.x) * n0.y * n0.z;
    rec_begin(st);
    k_coarsest<TD, TW><<<grid_1d(total, 256, p), 256, 0, st>>>(const_cast<TD*>(static_cast<const TD*>(in)),
                                                                 p->full[1] * p->full[2], p->full[2], cur, n0, s, N, 0);
    cudaError_t e = cudaGetLastError();
    rec_end(st, "coarsest", 0, double(total) * (sizeof(TD) + sizeof(TW)), 0.0);
    if (e != cudaSuccess) return e;
  }
  for (int l = 1; l <= L; ++l) {
    auto a = load_args<TS, TW>(p, l);
    a.in = in;
    a.in_full = 1;
    a.in_sz = a.y_sz;
    a.in_sy = a.y_sy;
    a.f = F;
    a.w = nullptr;
    a.y = nullptr;
    a.write_y = 0;
    dim3 grid = load_grid(p, a);
    dim3 block(BX, BY);
    constexpr size_t sm = load_smem_bytes<TD, TS>();
    cudaFuncSetAttribute(k_level_load<MODE_REC, TD, TD, TS, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    rec_begin(st);
    k_level_load<MODE_REC, TD, TD, TS, TW><<<grid, block, sm, st>>>(a);
    cudaError_t e = cudaGetLastError();
    {
      const Work wk = work_level_load(p, l, false);
      rec_end(st, "level_load_rec", l, wk.bytes, wk.flops);
    }
    if (e != cudaSuccess) return e;
    if ((e = solve_level<TW>(p, l, F, cur, SOLVE_SUB, st)) != cudaSuccess) return e;
    const LevelGeom& g = p->geom[l];
    const TS* T = table<TS>(p);
    const int3 n = make_int3(g.ax[0].n, g.ax[1].n, g.ax[2].n);
    const longlong3 s = make_longlong3(g.ax[0].s, g.ax[1].s, g.ax[2].s);
    const longlong3 N = make_longlong3(g.ax[0].N, g.ax[1].N, g.ax[2].N);
    const int64_t total = g.fine_count();
    const int64_t c_sz = int64_t(g.ax[1].m) * g.ax[2].m, c_sy = g.ax[2].m;
    rec_begin(st);
    if (l == L) {
      k_interp<TD, TD, TS, TW><<<grid_1d(total, 256, p), 256, 0, st>>>(
          static_cast<const TD*>(in), a.y_sz, a.y_sy, n, s, N, cur, c_sz, c_sy, static_cast<TD*>(out), a.y_sz, a.y_sy,
          T + g.ax[0].o_wa, T + g.ax[0].o_wb, T + g.ax[1].o_wa, T + g.ax[1].o_wb, T + g.ax[2].o_wa, T + g.ax[2].o_wb);
    } else {
      TW* nxt = static_cast<TW*>(cur == b.A ? b.B : b.A);
      k_interp<TD, TW, TS, TW><<<grid_1d(total, 256, p), 256, 0, st>>>(
          static_cast<const TD*>(in), a.y_sz, a.y_sy, n, s, N, cur, c_sz, c_sy, nxt, int64_t(n.y) * n.z, n.z,
          T + g.ax[0].o_wa, T + g.ax[0].o_wb, T + g.ax[1].o_wa, T + g.ax[1].o_wb, T + g.ax[2].o_wa, T + g.ax[2].o_wb);
      cur = nxt;
    }
    e = cudaGetLastError();
    {
      const Work wk = work_interp(p, l);
      rec_end(st, "interp", l, wk.bytes, wk.flops);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t enqueue_decompose(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st) {
  switch (p->form) {
    case kFormF64: return decompose_t<double, double, double>(p, in, out, ws, st);
    case kFormF32: return decompose_t<float, float, float>(p, in, out, ws, st);
    default: return decompose_t<float, float, double>(p, in, out, ws, st);
  }
}

cudaError_t enqueue_recompose(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st) {
  switch (p->form) {
    case kFormF64: return recompose_t<double, double, double>(p, in, out, ws, st);
    case kFormF32: return recompose_t<float, float, float>(p, in, out, ws, st);
    default: return recompose_t<float, float, double>(p, in, out, ws, st);
  }
}

}  // namespace mgr
