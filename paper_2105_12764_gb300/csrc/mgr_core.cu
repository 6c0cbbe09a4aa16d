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
#include <type_traits>

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

#include "mgr_device.cuh"
#include "mgr_level.cuh"
#include "mgr_solve.cuh"

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

constexpr int kInterpNW = 8, kInterpRPW = 2;

template <typename TS, typename TW>
LevelArgs<TS, TW> level_args(const mgr_plan* p, int l) {
  const LevelGeom& g = p->geom[l];
  LevelArgs<TS, TW> a{};
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

// Number of z chunks for `tiles` xy tiles and mz coarse planes: minimise
// waves x planes streamed per CTA (each chunk also streams ~1.5 halo planes).
inline int choose_chunks(const mgr_plan* p, int64_t tiles, int mz, int ctas_per_sm) {
  const int64_t slots = int64_t(p->ctx->num_sms) * ctas_per_sm;
  int best = 1;
  double best_cost = 1e300;
  const int cmax = std::max(1, std::min(mz, 64));
  for (int c = 1; c <= cmax; ++c) {
    const int len = (mz + c - 1) / c;
    if (c > 1 && len < 4) break;
    const int cc = (mz + len - 1) / len;
    const int64_t waves = (tiles * cc + slots - 1) / slots;
    const double cost = double(waves) * (len + 1.5);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = c;
    }
  }
  return best;
}

template <typename TS, typename TW>
dim3 level_grid(const mgr_plan* p, LevelArgs<TS, TW>& a) {
  using C = LevelCfg<TS>;
  using G = LevelTile<C::NW, C::RPW>;
  const int gx = (a.m[2] + G::BX - 1) / G::BX, gy = (a.m[1] + G::BY - 1) / G::BY;
  const int chunks = choose_chunks(p, int64_t(gx) * gy, a.m[0], 2);
  a.qz_chunk = (a.m[0] + chunks - 1) / chunks;
  const int gz = (a.m[0] + a.qz_chunk - 1) / a.qz_chunk;
  return dim3(gx, gy, gz);
}

template <int MODE, typename TI, typename TD, typename TS, typename TW, bool PK, bool QZ = false>
void launch_level(const mgr_plan* p, LevelArgs<TS, TW>& a, cudaStream_t st) {
  using C = LevelCfg<TS>;
  constexpr size_t sm = level_smem_bytes<C::NW, C::RPW, C::STAGES, TI, TS>();
  auto kern = k_level<MODE, C::NW, C::RPW, C::STAGES, TI, TD, TS, TW, PK, QZ>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  dim3 grid = level_grid(p, a);
  kern<<<grid, C::NW * 32, sm, st>>>(a);
}

// c: nodal coefficients (PK false), the packed class of level l (PK true), or
// null for a dropped class (all coefficients zero); QZ: c holds codes of bin
// width qs
template <typename TD, typename TO, typename TS, typename TW, bool PK, bool QZ = false>
void launch_interp(const mgr_plan* p, int l, const void* c, const TW* w, void* out, int out_full, cudaStream_t st,
                   double qs = 1.0) {
  const LevelGeom& g = p->geom[l];
  const TS* T = table<TS>(p);
  InterpArgs<TS, TW> a{};
  for (int k = 0; k < 3; ++k) {
    a.n[k] = g.ax[k].n;
    a.m[k] = g.ax[k].m;
    a.s[k] = g.ax[k].s;
    a.N[k] = g.ax[k].N;
    a.wa[k] = T + g.ax[k].o_wa;
    a.wb[k] = T + g.ax[k].o_wb;
  }
  a.c = c;
  a.y_sz = PK ? int64_t(g.ax[1].n) * g.ax[2].n : p->full[1] * p->full[2];
  a.y_sy = PK ? int64_t(g.ax[2].n) : p->full[2];
  a.w = w;
  a.c_sz = int64_t(g.ax[1].m) * g.ax[2].m;
  a.c_sy = g.ax[2].m;
  a.out = out;
  a.out_full = out_full;
  a.qs = qs;
  a.o_sz = out_full ? a.y_sz : int64_t(g.ax[1].n) * g.ax[2].n;
  a.o_sy = out_full ? a.y_sy : int64_t(g.ax[2].n);
  constexpr int BY = kInterpNW * kInterpRPW;
  const int gx = (a.m[2] + 31) / 32, gy = (a.m[1] + BY - 1) / BY;
  const int chunks = choose_chunks(p, int64_t(gx) * gy, a.m[0], 2);
  a.qz_chunk = (a.m[0] + chunks - 1) / chunks;
  const int gz = (a.m[0] + a.qz_chunk - 1) / a.qz_chunk;
  constexpr size_t sm = interp_smem_bytes<kInterpNW, kInterpRPW, TD, TW>();
  auto kern = k_interp<kInterpNW, kInterpRPW, TD, TO, TS, TW, PK, QZ>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  kern<<<dim3(gx, gy, gz), kInterpNW * 32, sm, st>>>(a);
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
  const int64_t lines_x = int64_t(mz) * my;
  if (axis == 2 && sizeof(TW) * (size_t(mx | 1) + 2 * size_t(mx)) > 96 * 1024) {
    // lines too long to stage in shared memory: one thread per line from global memory
    const int threads = 128;
    const int blocks = int((lines_x + threads - 1) / threads);
    k_solve_strided<TW><<<blocks, threads, 0, st>>>(f, w, mx, 1, 1, lines_x, mx, ta, tb, op);
    return cudaGetLastError();
  }
  if (axis == 2) {
    const int pitch = mx | 1;
    // rows per CTA (one solving thread per row, 128 threads load and store):
    // up to 32 rows within 32 KB of shared memory, so several CTAs share an SM
    int R = int(std::min<size_t>(32, (32 * 1024) / (sizeof(TW) * pitch)));
    R = std::max(1, R);
    const size_t sm = sizeof(TW) * (size_t(R) * pitch + 2 * size_t(mx));
    const int blocks = int((lines_x + R - 1) / R);
    cudaFuncSetAttribute(k_solve_contig<TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    k_solve_contig<TW><<<blocks, 128, sm, st>>>(f, w, mx, lines_x, mx, R, ta, tb, op);
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
  k_solve_strided<TW><<<blocks, threads, 0, st>>>(f, w, mline, lstride, inner, outer, ostride, ta, tb, op);
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

// Coarsest grid <-> its place in the output: the nodal positions at stride
// 2^L (nodal layout) or class 0, the compact coarsest grid (packed layout).
template <typename TD, typename TW>
cudaError_t coarsest_copy_launch(const mgr_plan* p, TD* y, TW* w, bool packed, int dir, cudaStream_t st) {
  const int L = p->levels;
  const int3 n0 = make_int3(int(p->coarsest[0]), int(p->coarsest[1]), int(p->coarsest[2]));
  const int64_t s0 = packed ? 1 : (int64_t(1) << L);
  const longlong3 s = make_longlong3(p->full[0] > 1 ? s0 : 1, p->full[1] > 1 ? s0 : 1, s0);
  const longlong3 N = packed ? make_longlong3(n0.x, n0.y, n0.z) : make_longlong3(p->full[0], p->full[1], p->full[2]);
  const int64_t total = int64_t(n0.x) * n0.y * n0.z;
  rec_begin(st);
  k_coarsest<TD, TW><<<grid_1d(total, 256, p), 256, 0, st>>>(y, N.y * N.z, N.z, w, n0, s, N, dir);
  cudaError_t e = cudaGetLastError();
  rec_end(st, "coarsest", 0, double(total) * (sizeof(TD) + sizeof(TW)), 0.0);
  return e;
}

// Class 0 of a quantized decomposition: codes of the compact coarsest values
// v (dir 1) or those values from their codes (dir 0), arithmetic and rounding
// decision in TW.  v is the compact coarse workspace, or the field itself
// when the hierarchy has no level (L = 0).
template <typename TV, typename TW>
__global__ void k_coarsest_q(int* codes, TV* v, int64_t total, double q, int dir, unsigned long long* sat) {
  const TW qinv = TW(1.0 / q), qq = TW(q);
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    if (dir)
      codes[i] = quant_code(TW(v[i]), qinv, sat);
    else
      v[i] = TV(dequant(codes[i], qq));
  }
}

template <typename TV, typename TW>
cudaError_t coarsest_q_launch(const mgr_plan* p, int* codes, TV* v, double q, int dir, unsigned long long* sat,
                              cudaStream_t st) {
  const int64_t total = p->class_off[1];
  rec_begin(st);
  k_coarsest_q<TV, TW><<<grid_1d(total, 256, p), 256, 0, st>>>(codes, v, total, q, dir, sat);
  cudaError_t e = cudaGetLastError();
  rec_end(st, "coarsest", 0, double(total) * (sizeof(int) + sizeof(TV)), 0.0);
  return e;
}

// PK: write the coefficients in the class-packed layout (class l at
// p->class_off[l]; `out` must not overlap `in`).  QZ (with PK): write int32
// codes with the bin widths bins[0..L] instead, counting saturated codes in
// *sat (when not null).
template <typename TD, typename TS, typename TW, bool PK, bool QZ = false>
cudaError_t decompose_t(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st,
                        const double* bins = nullptr, unsigned long long* sat = nullptr) {
  static_assert(PK || !QZ, "quantized output is class-packed");
  using TY = std::conditional_t<QZ, int, TD>;  // coefficient output type
  const int L = p->levels;
  const size_t bytes = size_t(p->count) * sizeof(TD);
  if (L == 0) {
    // the whole field is the coarsest class
    if constexpr (QZ) {
      return coarsest_q_launch<TD, TW>(p, static_cast<int*>(out), const_cast<TD*>(static_cast<const TD*>(in)),
                                       bins[0], 1, sat, st);
    } else {
      if (in != out) return cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, st);
      return cudaSuccess;
    }
  }
  const bool inplace = !PK && (in == out);
  Bufs b = split_ws(p, ws);
  TW* F = static_cast<TW*>(b.F);
  TW* cur = nullptr;  // compact level-l values for l < L
  for (int l = L; l >= 1; --l) {
    TW* nxt = static_cast<TW*>(((L - l) % 2 == 0) ? b.A : b.B);
    auto a = level_args<TS, TW>(p, l);
    const LevelGeom& g = p->geom[l];
    a.y = out;
    if (PK) {
      a.y = static_cast<TY*>(out) + p->class_off[l];
      a.y_sz = int64_t(g.ax[1].n) * g.ax[2].n;
      a.y_sy = g.ax[2].n;
    }
    if (QZ) {
      a.qs = 1.0 / bins[l];
      a.qsat = sat;
    }
    a.w = nxt;
    a.f = F;
    a.write_y = (l == L && inplace) ? 0 : 1;
    rec_begin(st);
    if (l == L) {
      a.in = in;
      a.in_full = 1;
      a.in_sz = p->full[1] * p->full[2];
      a.in_sy = p->full[2];
      launch_level<0, TD, TY, TS, TW, PK, QZ>(p, a, st);
    } else {
      a.in = cur;
      a.in_full = 0;
      a.in_sz = int64_t(g.ax[1].n) * g.ax[2].n;
      a.in_sy = g.ax[2].n;
      launch_level<0, TW, TY, TS, TW, PK, QZ>(p, a, st);
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
  // coarsest values into their nodal positions / class 0
  if constexpr (QZ) return coarsest_q_launch<TW, TW>(p, static_cast<int*>(out), cur, bins[0], 1, sat, st);
  else return coarsest_copy_launch<TD, TW>(p, static_cast<TD*>(out), cur, PK, 1, st);
}

// Recompose from classes 0..ncls-1 (ncls = L+1: all of them).  Levels whose
// class is dropped have zero coefficients, hence a zero correction: they are
// interpolation only.  PK: `in` is class-packed (its first class_off[ncls]
// elements are read) and must not overlap `out`.
// QZ (with PK): `in` holds int32 codes with the bin widths bins[0..L].
template <typename TD, typename TS, typename TW, bool PK, bool QZ = false>
cudaError_t recompose_t(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st, int ncls,
                        const double* bins = nullptr) {
  static_assert(PK || !QZ, "quantized input is class-packed");
  using TY = std::conditional_t<QZ, int, TD>;  // coefficient input type
  const int L = p->levels;
  const size_t bytes = size_t(p->count) * sizeof(TD);
  if (L == 0) {
    if constexpr (QZ) {
      return coarsest_q_launch<TD, TW>(p, const_cast<int*>(static_cast<const int*>(in)), static_cast<TD*>(out),
                                       bins[0], 0, nullptr, st);
    } else {
      if (in != out) return cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, st);
      return cudaSuccess;
    }
  }
  Bufs b = split_ws(p, ws);
  TW* F = static_cast<TW*>(b.F);
  // coarsest grid from the nodal positions / class 0
  TW* cur = static_cast<TW*>((L % 2 == 1) ? b.A : b.B);  // level 0 lives where decompose left it
  {
    cudaError_t e;
    if constexpr (QZ) e = coarsest_q_launch<TW, TW>(p, const_cast<int*>(static_cast<const int*>(in)), cur, bins[0], 0,
                                                    nullptr, st);
    else e = coarsest_copy_launch<TD, TW>(p, const_cast<TD*>(static_cast<const TD*>(in)), cur, PK, 0, st);
    if (e != cudaSuccess) return e;
  }
  for (int l = 1; l <= L; ++l) {
    const LevelGeom& g = p->geom[l];
    const void* cl = PK ? static_cast<const void*>(static_cast<const TY*>(in) + p->class_off[l]) : in;
    const double qs = QZ ? bins[l] : 1.0;
    if (l >= ncls) {
      // dropped class: v = interpolant of the coarse values
      rec_begin(st);
      if (l == L) {
        launch_interp<TY, TD, TS, TW, PK, QZ>(p, l, nullptr, cur, out, 1, st, qs);
      } else {
        TW* nxt = static_cast<TW*>(cur == b.A ? b.B : b.A);
        launch_interp<TY, TW, TS, TW, PK, QZ>(p, l, nullptr, cur, nxt, 0, st, qs);
        cur = nxt;
      }
      cudaError_t e = cudaGetLastError();
      {
        const Work wk = work_interp(p, l);
        rec_end(st, "interp_zero", l, wk.bytes - double(g.fine_count()) * p->elem, wk.flops);
      }
      if (e != cudaSuccess) return e;
      continue;
    }
    auto a = level_args<TS, TW>(p, l);
    a.in = cl;
    if (PK) {
      a.in_full = 0;
      a.in_sz = int64_t(g.ax[1].n) * g.ax[2].n;
      a.in_sy = g.ax[2].n;
    } else {
      a.in_full = 1;
      a.in_sz = a.y_sz;
      a.in_sy = a.y_sy;
    }
    a.f = F;
    a.w = nullptr;
    a.y = nullptr;
    a.write_y = 0;
    a.qs = qs;
    rec_begin(st);
    launch_level<1, TY, TY, TS, TW, PK, QZ>(p, a, st);
    cudaError_t e = cudaGetLastError();
    {
      const Work wk = work_level_load(p, l, false);
      rec_end(st, "level_load_rec", l, wk.bytes, wk.flops);
    }
    if (e != cudaSuccess) return e;
    if ((e = solve_level<TW>(p, l, F, cur, SOLVE_SUB, st)) != cudaSuccess) return e;
    rec_begin(st);
    if (l == L) {
      launch_interp<TY, TD, TS, TW, PK, QZ>(p, l, cl, cur, out, 1, st, qs);
    } else {
      TW* nxt = static_cast<TW*>(cur == b.A ? b.B : b.A);
      launch_interp<TY, TW, TS, TW, PK, QZ>(p, l, cl, cur, nxt, 0, st, qs);
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
    case kFormF64: return decompose_t<double, double, double, false>(p, in, out, ws, st);
    case kFormF32: return decompose_t<float, float, float, false>(p, in, out, ws, st);
    default: return decompose_t<float, float, double, false>(p, in, out, ws, st);
  }
}

cudaError_t enqueue_recompose(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st) {
  const int all = p->levels + 1;
  switch (p->form) {
    case kFormF64: return recompose_t<double, double, double, false>(p, in, out, ws, st, all);
    case kFormF32: return recompose_t<float, float, float, false>(p, in, out, ws, st, all);
    default: return recompose_t<float, float, double, false>(p, in, out, ws, st, all);
  }
}

cudaError_t enqueue_decompose_packed(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st) {
  switch (p->form) {
    case kFormF64: return decompose_t<double, double, double, true>(p, in, out, ws, st);
    case kFormF32: return decompose_t<float, float, float, true>(p, in, out, ws, st);
    default: return decompose_t<float, float, double, true>(p, in, out, ws, st);
  }
}

cudaError_t enqueue_recompose_packed(const mgr_plan* p, const void* in, int ncls, void* out, void* ws,
                                     cudaStream_t st) {
  switch (p->form) {
    case kFormF64: return recompose_t<double, double, double, true>(p, in, out, ws, st, ncls);
    case kFormF32: return recompose_t<float, float, float, true>(p, in, out, ws, st, ncls);
    default: return recompose_t<float, float, double, true>(p, in, out, ws, st, ncls);
  }
}

cudaError_t enqueue_decompose_quantized(const mgr_plan* p, const void* in, int* codes, const double* bins,
                                        unsigned long long* sat, void* ws, cudaStream_t st) {
  switch (p->form) {
    case kFormF64: return decompose_t<double, double, double, true, true>(p, in, codes, ws, st, bins, sat);
    case kFormF32: return decompose_t<float, float, float, true, true>(p, in, codes, ws, st, bins, sat);
    default: return decompose_t<float, float, double, true, true>(p, in, codes, ws, st, bins, sat);
  }
}

cudaError_t enqueue_recompose_dequantized(const mgr_plan* p, const int* codes, int ncls, const double* bins,
                                          void* out, void* ws, cudaStream_t st) {
  switch (p->form) {
    case kFormF64: return recompose_t<double, double, double, true, true>(p, codes, out, ws, st, ncls, bins);
    case kFormF32: return recompose_t<float, float, float, true, true>(p, codes, out, ws, st, ncls, bins);
    default: return recompose_t<float, float, double, true, true>(p, codes, out, ws, st, ncls, bins);
  }
}

}  // namespace mgr
