// mgr_launch.cuh -- host-side launch helpers shared by the level loops of
// the single-field paths (mgr_core.cu: 1D-3D; mgr_st.cu: the spatiotemporal
// 4D form): per-launch event recording, plan tables, level arguments, grid
// choices, kernel launches of the level pass / interpolation / solves and the
// coarsest-grid copy.  Included inside an anonymous namespace after the kernel
// headers (mgr_device.cuh, mgr_level.cuh, mgr_solve.cuh).
#pragma once

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
// Chunks may be a single plane: on small levels the plane loop's latency, not
// the halo's extra work, bounds the pass, so the more CTAs the better.  Chunks
// are at most max_len planes long (the level pass tabulates its planes).
inline int choose_chunks(const mgr_plan* p, int64_t tiles, int mz, int ctas_per_sm, int max_len = 1 << 30) {
  const int64_t slots = int64_t(p->ctx->num_sms) * ctas_per_sm;
  const int cmin = std::max(1, (mz + max_len - 1) / max_len);
  int best = cmin;
  double best_cost = 1e300;
  const int cmax = std::max(cmin, std::min(mz, 64));
  for (int c = cmin; c <= cmax; ++c) {
    const int len = (mz + c - 1) / c;
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

template <int MODE, typename TS, typename TW>
dim3 level_grid(const mgr_plan* p, LevelArgs<TS, TW>& a) {
  using C = LevelCfgM<TS, MODE>;
  using G = LevelTile<C::NW, C::RPW>;
  const int gx = (a.m[2] + G::BX - 1) / G::BX, gy = (a.m[1] + G::BY - 1) / G::BY;
  const int chunks = choose_chunks(p, int64_t(gx) * gy, a.m[0], level_ctas_per_sm(C::NW), kLevelMaxChunk);
  a.qz_chunk = (a.m[0] + chunks - 1) / chunks;
  const int gz = (a.m[0] + a.qz_chunk - 1) / a.qz_chunk;
  return dim3(gx, gy, gz);
}

template <int MODE, typename TI, typename TD, typename TS, typename TW, bool PK, bool QZ = false>
void launch_level(const mgr_plan* p, LevelArgs<TS, TW>& a, cudaStream_t st) {
  using C = LevelCfgM<TS, MODE>;
  constexpr size_t sm = level_smem_bytes<C::NW, C::RPW, C::STAGES, TI, TS>();
  auto kern = k_level<MODE, C::NW, C::RPW, C::STAGES, TI, TD, TS, TW, PK, QZ>;
  raise_smem_limit(kern, sm);
  dim3 grid = level_grid<MODE>(p, a);
  kern<<<grid, C::NW * 32, sm, st>>>(a);
}

// z chunks [c0, c1) of the level pass's grid (the grid level_grid chooses):
// a level pass may run as several such launches, each as soon as its input
// planes are ready.
template <int MODE, typename TI, typename TD, typename TS, typename TW, bool PK, bool QZ = false>
void launch_level_chunks(const mgr_plan* p, LevelArgs<TS, TW>& a, int c0, int c1, cudaStream_t st) {
  using C = LevelCfgM<TS, MODE>;
  constexpr size_t sm = level_smem_bytes<C::NW, C::RPW, C::STAGES, TI, TS>();
  auto kern = k_level<MODE, C::NW, C::RPW, C::STAGES, TI, TD, TS, TW, PK, QZ>;
  raise_smem_limit(kern, sm);
  dim3 grid = level_grid<MODE>(p, a);
  if (c1 <= c0 || c1 > int(grid.z)) return;
  a.bz0 = c0;
  grid.z = unsigned(c1 - c0);
  kern<<<grid, C::NW * 32, sm, st>>>(a);
  a.bz0 = 0;
}

// c: nodal coefficients (PK false), the packed class of level l (PK true), or
// null for a dropped class (all coefficients zero); QZ: c holds codes of bin
// width qs
template <typename TD, typename TO, typename TS, typename TW, bool PK, bool QZ = false>
void launch_interp(const mgr_plan* p, int l, const void* c, const TW* w, void* out, int out_full, cudaStream_t st,
                   double qs = 1.0);

// Arguments of the interpolation of level l (spatial axes) and its (x, y)
// tile counts; the z chunking is left to the caller.
template <typename TS, typename TW, bool PK = false>
InterpArgs<TS, TW> interp_args(const mgr_plan* p, int l, const void* c, const TW* w, void* out, int out_full,
                               double qs, int* gx, int* gy) {
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
  *gx = (a.m[2] + 31) / 32;
  *gy = (a.m[1] + BY - 1) / BY;
  return a;
}

// z chunking of an interpolation launch (sets a.qz_chunk; returns the chunk count)
template <typename TS, typename TW>
int interp_chunks(const mgr_plan* p, InterpArgs<TS, TW>& a, int gx, int gy) {
  const int chunks = choose_chunks(p, int64_t(gx) * gy, a.m[0], 2, kLevelMaxChunk);
  a.qz_chunk = (a.m[0] + chunks - 1) / chunks;
  return (a.m[0] + a.qz_chunk - 1) / a.qz_chunk;
}

// z chunks [c0, c1) of the interpolation of level l (c1 < 0: all of them)
template <typename TD, typename TO, typename TS, typename TW, bool PK, bool QZ>
void launch_interp_chunks(const mgr_plan* p, int l, const void* c, const TW* w, void* out, int out_full,
                          cudaStream_t st, double qs, int c0, int c1) {
  int gx, gy;
  InterpArgs<TS, TW> a = interp_args<TS, TW, PK>(p, l, c, w, out, out_full, qs, &gx, &gy);
  const int gz = interp_chunks(p, a, gx, gy);
  if (c1 < 0) c1 = gz;
  if (c1 <= c0 || c1 > gz) return;
  a.bz0 = c0;
  constexpr size_t sm = interp_smem_bytes<kInterpNW, kInterpRPW, TD, TS, TW>();
  auto kern = k_interp<kInterpNW, kInterpRPW, TD, TO, TS, TW, PK, QZ>;
  raise_smem_limit(kern, sm);
  kern<<<dim3(gx, gy, c1 - c0), kInterpNW * 32, sm, st>>>(a);
}

template <typename TD, typename TO, typename TS, typename TW, bool PK, bool QZ>
void launch_interp(const mgr_plan* p, int l, const void* c, const TW* w, void* out, int out_full, cudaStream_t st,
                   double qs) {
  launch_interp_chunks<TD, TO, TS, TW, PK, QZ>(p, l, c, w, out, out_full, st, qs, 0, -1);
}

// Thomas solves along the contiguous axis: `lines` lines of length mx,
// consecutive in memory.  Build-time knobs: MGR_X_SOLVE_ROWS (1: FP64 with
// many lines through k_solve_rows), MGR_X_SOLVE_KB (shared memory per CTA of
// k_solve_contig).
#ifndef MGR_X_SOLVE_ROWS
#define MGR_X_SOLVE_ROWS 1
#endif
#ifndef MGR_X_SOLVE_KB
#define MGR_X_SOLVE_KB 32
#endif
template <typename TW>
cudaError_t launch_x_solve(const mgr_plan* p, TW* f, TW* w, int mx, int64_t lines, const TW* ta, const TW* tb, int op,
                           cudaStream_t st) {
  (void)p;
  if (MGR_X_SOLVE_ROWS && sizeof(TW) == 8 && lines >= 32768) {
    // lines through 32 x 32 tiles, the intermediate through memory
    const int64_t nwarps = (lines + 31) / 32;
    k_solve_rows<TW><<<int((nwarps + kRowsWarps - 1) / kRowsWarps), kRowsWarps * 32, 0, st>>>(f, w, mx, lines, mx, ta,
                                                                                             tb, op);
    return cudaGetLastError();
  }
  if (solve_contig_smem<TW>(mx, 1) > 96 * 1024) {
    // lines too long to stage in shared memory: one thread per line from global memory
    const int threads = 128;
    const int blocks = int((lines + threads - 1) / threads);
    k_solve_strided<TW><<<blocks, threads, 0, st>>>(f, w, mx, 1, 1, lines, mx, ta, tb, op);
    return cudaGetLastError();
  }
  const int pitch = contig_pitch<TW>(mx);
  // rows per CTA (one solving thread per row, 128 threads load and store): up
  // to 32, a whole warp of recurrences, within MGR_X_SOLVE_KB of shared memory
  int R = int(std::min<size_t>(32, (size_t(MGR_X_SOLVE_KB) * 1024) / (sizeof(TW) * pitch)));
  R = std::max(1, R);
  const size_t sm = solve_contig_smem<TW>(mx, R);
  const int blocks = int((lines + R - 1) / R);
  raise_smem_limit(k_solve_contig<TW>, sm);
  k_solve_contig<TW><<<blocks, 128, sm, st>>>(f, w, mx, lines, mx, R, ta, tb, op);
  return cudaGetLastError();
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

// Strided axes: whole lines staged in shared memory below this many lines
// (build-time knobs), one thread per line from global memory above.
#ifndef MGR_STAGED_LINES_F32
#define MGR_STAGED_LINES_F32 32768
#endif
#ifndef MGR_STAGED_LINES_F64
#define MGR_STAGED_LINES_F64 32768
#endif
template <typename TW>
cudaError_t solve_axis_launch(const mgr_plan* p, int l, int axis, TW* f, TW* w, int op, cudaStream_t st) {
  const LevelGeom& g = p->geom[l];
  const int mz = g.ax[0].m, my = g.ax[1].m, mx = g.ax[2].m;
  const TW* T = table<TW>(p);
  const TW* ta = T + g.ax[axis].o_ta;
  const TW* tb = T + g.ax[axis].o_tb;
  const int64_t lines_x = int64_t(mz) * my;
  if (axis == 2) return launch_x_solve<TW>(p, f, w, mx, lines_x, ta, tb, op, st);
  int mline, inner;
  int64_t lstride, outer, ostride;
  if (axis == 1) {
    mline = my; lstride = mx; inner = mx; outer = mz; ostride = int64_t(my) * mx;
  } else {
    mline = mz; lstride = int64_t(my) * mx; inner = mx; outer = my; ostride = mx;
  }
  const int64_t lines = int64_t(inner) * outer;
  const size_t ssm = solve_staged_smem<TW>(mline);
  const int64_t staged_below = sizeof(TW) == 4 ? int64_t(MGR_STAGED_LINES_F32) : int64_t(MGR_STAGED_LINES_F64);
  if (lines < staged_below && ssm <= size_t(100) * 1024 && ssm <= p->ctx->smem_optin) {
    // few lines (coarse levels): whole lines staged in shared memory, 32 per CTA
    raise_smem_limit(k_solve_staged<TW>, ssm);
    k_solve_staged<TW><<<int((lines + kStagedLines - 1) / kStagedLines), 128, ssm, st>>>(f, w, mline, lstride, inner,
                                                                                       outer, ostride, ta, tb, op);
    return cudaGetLastError();
  }
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
