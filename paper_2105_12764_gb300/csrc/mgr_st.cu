// mgr_st.cu -- spatiotemporal (3+1)-D refactoring (arXiv 2105.12764,
// Sec. III.E): a 4D field (t, z, y, x), time slowest, decomposed with the same
// tensor-product method in four dimensions (interpolation, mass transfer and
// Thomas solves along all four axes per level).
//
// Hierarchical batching, GB300 form.  The paper keeps shared memory at
// O(b^3) by batching three selected dimensions in a thread block and spreading
// the fourth over thread blocks.  Here every time slice is a 3D field for the
// spatial kernels (the z-streamed level pass and interpolation of
// mgr_level.cuh, unchanged, with the time slice as one more grid dimension of
// the launch), and the time axis is handled by separate passes over whole
// slices:
//
//   decomposition of level l (n_t slices -> m_t coarse slices)
//     D1  slices coarse in time: the 3D level pass.  In such a slice the 4D
//         coefficients are the 3D ones (the 4D interpolant of a node of a
//         coarse-time slice is its slice's 3D interpolant), and it writes the
//         coarse nodes and the 3D load vector g_t = (K_z x K_y x K_x) c_t.
//     D2  slices fine in time: a node's 4D interpolant is
//         wa P3(v_{t-1}) + wb P3(v_{t+1}), P3 the 3D interpolant of a slice's
//         coarse nodes, and P3(v_s) = v_s - c_s for the coarse slices' 3D
//         coefficients c_s (zero on their 3D-coarse nodes), so
//           c_t = v_t - wa (v_{t-1} - c_{t-1}) - wb (v_{t+1} - c_{t+1})
//         pointwise (k_time_fine).
//     D3  slices fine in time: g_t = (K_z x K_y x K_x) c_t by the level pass in
//         its load-vector mode, every node being a coefficient there.
//     D4  f = K_t g along time: five taps per coarse slice (k_time_stencil).
//     D5  Thomas solves along x, y, z and t on the coarse 4D grid; the last
//         adds the correction to the coarse nodes (Eq. (1)).
//   recomposition of level l: g_t for every slice (D3's mode, coarse-time
//   slices with the usual coarse-node zeros), D4, D5 subtracting, then the 3D
//   interpolation of the coarse-time slices and D2 inverted for the others:
//           v_t = c_t + wa (v_{t-1} - c_{t-1}) + wb (v_{t+1} - c_{t+1}).
//
// Layout: nodal, like the 3D form (time index t of level l at full-grid time
// index min(t * 2^(L-l), N_t - 1)).  The operations are out of place (the
// time passes read neighbouring slices' input values after their coefficients
// are written).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>

#include "mgr_internal.h"

namespace mgr {
namespace {

#include "mgr_device.cuh"
#include "mgr_level.cuh"
#include "mgr_solve.cuh"
#include "mgr_launch.cuh"

// Time slices of a batched spatial launch: blockIdx.z = j * zchunks + chunk,
// slice j is the level time index t = min(first + j * step, last).
struct Slabs {
  int zchunks;
  int first, step, last;
  int nt;                    // level time length n_t
  int64_t tS, tN;            // full-grid time map: index min(t * tS, tN - 1)
  int64_t in_ts, y_ts, o_ts; // element strides per time index of in / y (or c) / out
  int64_t w_ts, f_ts;        // per slice j of w, per time index t of f
  int in_tfull, out_tfull;   // in / out addressed through the full-grid time map
  int fine_all;              // load-vector mode: slices fine in time hold coefficients at every node
};

__device__ __forceinline__ int slab_time(const Slabs& sl, int j) { return min(sl.first + j * sl.step, sl.last); }
__device__ __forceinline__ int64_t slab_map(const Slabs& sl, int t, int full) {
  return full ? fmap(t, sl.tS, sl.tN) : int64_t(t);
}

template <int MODE, int NW, int RPW, int STAGES, typename TI, typename TD, typename TS, typename TW>
__global__ void __launch_bounds__(NW * 32, level_ctas_per_sm(NW)) k_level_st(const LevelArgs<TS, TW> a, const Slabs sl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int j = blockIdx.z / sl.zchunks, bz = blockIdx.z - j * sl.zchunks;
  const int t = slab_time(sl, j);
  LevelArgs<TS, TW> b = a;
  b.in = static_cast<const TI*>(a.in) + slab_map(sl, t, sl.in_tfull) * sl.in_ts;
  if (MODE == 0) {
    b.y = static_cast<TD*>(a.y) + slab_map(sl, t, 1) * sl.y_ts;
    b.w = a.w + int64_t(j) * sl.w_ts;
  }
  b.f = a.f + int64_t(t) * sl.f_ts;
  b.all_fine = (MODE == 1 && sl.fine_all) ? int(!is_coarse(t, sl.nt)) : 0;
  level_body<MODE, NW, RPW, STAGES, TI, TD, TS, TW, false, false, true>(b, blockIdx.x, blockIdx.y, bz, smem_raw);
}

template <int NW, int RPW, typename TD, typename TO, typename TS, typename TW>
__global__ void __launch_bounds__(NW * 32, level_ctas_per_sm(NW)) k_interp_st(const InterpArgs<TS, TW> a, const Slabs sl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int j = blockIdx.z / sl.zchunks, bz = blockIdx.z - j * sl.zchunks;
  const int t = slab_time(sl, j);
  InterpArgs<TS, TW> b = a;
  b.c = static_cast<const TD*>(a.c) + slab_map(sl, t, 1) * sl.y_ts;
  b.w = a.w + int64_t(j) * sl.w_ts;
  b.out = static_cast<TO*>(a.out) + slab_map(sl, t, sl.out_tfull) * sl.o_ts;
  interp_body<NW, RPW, TD, TO, TS, TW>(b, blockIdx.x, blockIdx.y, bz, smem_raw);
}

// Spatial addressing of one level for the elementwise time passes.
struct SpaceMap {
  int n[3];          // level sizes (z, y, x)
  int64_t s[3], N[3];
  int64_t full_sz, full_sy;  // full-grid strides of z and y
};

__device__ __forceinline__ int64_t space_full(const SpaceMap& g, int z, int y, int x) {
  return fmap(z, g.s[0], g.N[0]) * g.full_sz + fmap(y, g.s[1], g.N[1]) * g.full_sy + fmap(x, g.s[2], g.N[2]);
}

// D2 (DIR 0) and its inverse (DIR 1) on the slices fine in time, t = 2j + 1
// between the coarse slices t - 1 and t + 1.  v: level-l values (full grid
// through the maps when v_full, else compact), c: nodal coefficients.  One
// warp per (slice, z, y) row.
template <int DIR, typename TV, typename TC, typename TS>
__global__ void k_time_fine(TV* v, int v_full, TC* c, SpaceMap g, int nfine, int64_t tS, int64_t tN,
                            int64_t space_full_n, const TS* __restrict__ wa, const TS* __restrict__ wb) {
  const int nz = g.n[0], ny = g.n[1], nx = g.n[2];
  const int64_t rows = int64_t(nfine) * nz * ny;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int64_t Sn = int64_t(nz) * ny * nx;
  for (int64_t r = w0; r < rows; r += nw) {
    const int j = int(r / (int64_t(nz) * ny));
    const int64_t zy = r - int64_t(j) * nz * ny;
    const int z = int(zy / ny), y = int(zy - int64_t(z) * ny);
    const int t = 2 * j + 1;
    const TS ta = wa[t], tb = wb[t];
    const int64_t cT0 = fmap(t - 1, tS, tN) * space_full_n, cT = fmap(t, tS, tN) * space_full_n,
                  cT1 = fmap(t + 1, tS, tN) * space_full_n;
    const int64_t vT0 = v_full ? cT0 : int64_t(t - 1) * Sn, vT = v_full ? cT : int64_t(t) * Sn,
                  vT1 = v_full ? cT1 : int64_t(t + 1) * Sn;
    const bool yz_coarse = is_coarse(z, nz) && is_coarse(y, ny);
    for (int x = lane; x < nx; x += 32) {
      const int64_t cs = space_full(g, z, y, x);
      const int64_t vs = v_full ? cs : (int64_t(z) * ny + y) * nx + x;
      // coefficients of the coarse slices vanish on their 3D-coarse nodes (the
      // nodal array holds other levels' values there)
      const bool cc = yz_coarse && is_coarse(x, nx);
      const TS c0 = cc ? TS(0) : TS(c[cT0 + cs]), c1 = cc ? TS(0) : TS(c[cT1 + cs]);
      const TS d = ta * (TS(v[vT0 + vs]) - c0) + tb * (TS(v[vT1 + vs]) - c1);
      if (DIR == 0) {
        c[cT + cs] = TC(TS(v[vT + vs]) - d);
      } else {
        v[vT + vs] = TV(TS(c[cT + cs]) + d);
      }
    }
  }
}

// D4: f_q = sum_o Kt[q][o] g_{p(q)+o-2} along time for every coarse spatial
// node (Kt: the time axis' scaled mass-transfer rows).
template <typename TW>
__global__ void k_time_stencil(const TW* __restrict__ g, TW* __restrict__ f, int nt, int mt, int64_t Sm,
                               const TW* __restrict__ Kt) {
  const int64_t total = int64_t(mt) * Sm;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int q = int(e / Sm);
    const int64_t s = e - int64_t(q) * Sm;
    const int pq = pidx(q, nt);
    TW acc = TW(0);
#pragma unroll
    for (int o = 0; o < 5; ++o) {
      const int t = pq + o - 2;
      if (t >= 0 && t < nt) acc += Kt[5 * q + o] * g[int64_t(t) * Sm + s];
    }
    f[e] = acc;
  }
}

// Coarsest 4D grid <-> its nodal positions, one time slice per blockIdx.y.
template <typename TD, typename TW>
__global__ void k_coarsest_st(TD* y, int64_t y_sz, int64_t y_sy, TW* w, int3 n, longlong3 s, longlong3 N,
                              int64_t tS, int64_t tN, int64_t space_full_n, int dir) {
  const int t = blockIdx.y;
  const int64_t cnt = int64_t(n.x) * n.y * n.z;
  coarsest_copy<TD, TW>(y + fmap(t, tS, tN) * space_full_n, y_sz, y_sy, w + int64_t(t) * cnt, n, s, N, dir,
                        blockIdx.x * int64_t(blockDim.x) + threadIdx.x, int64_t(gridDim.x) * blockDim.x);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

SpaceMap space_map(const mgr_plan* p, int l) {
  const LevelGeom& g = p->geom[l];
  SpaceMap m{};
  for (int k = 0; k < 3; ++k) {
    m.n[k] = g.ax[k].n;
    m.s[k] = g.ax[k].s;
    m.N[k] = g.ax[k].N;
  }
  m.full_sz = p->full[1] * p->full[2];
  m.full_sy = p->full[2];
  return m;
}

int64_t space_full_count(const mgr_plan* p) { return p->full[0] * p->full[1] * p->full[2]; }

Slabs base_slabs(const mgr_plan* p, int l) {
  const AxisLevel& ta = p->geom[l].tax;
  Slabs sl{};
  sl.nt = ta.n;
  sl.tS = ta.s;
  sl.tN = ta.N;
  sl.y_ts = space_full_count(p);
  return sl;
}

// Batched spatial level pass over `slabs` time slices.
template <int MODE, typename TI, typename TD, typename TS, typename TW>
cudaError_t launch_level_st(const mgr_plan* p, LevelArgs<TS, TW>& a, Slabs sl, int slabs, cudaStream_t st) {
  if (slabs <= 0) return cudaSuccess;
  using C = LevelCfg<TS>;
  using G = LevelTile<C::NW, C::RPW>;
  constexpr size_t sm = level_smem_bytes<C::NW, C::RPW, C::STAGES, TI, TS>();
  const int gx = (a.m[2] + G::BX - 1) / G::BX, gy = (a.m[1] + G::BY - 1) / G::BY;
  const int chunks = choose_chunks(p, int64_t(gx) * gy * slabs, a.m[0], level_ctas_per_sm(C::NW), kLevelMaxChunk);
  a.qz_chunk = (a.m[0] + chunks - 1) / chunks;
  sl.zchunks = (a.m[0] + a.qz_chunk - 1) / a.qz_chunk;
  auto kern = k_level_st<MODE, C::NW, C::RPW, C::STAGES, TI, TD, TS, TW>;
  raise_smem_limit(kern, sm);
  kern<<<dim3(gx, gy, sl.zchunks * slabs), C::NW * 32, sm, st>>>(a, sl);
  return cudaGetLastError();
}

template <typename TD, typename TO, typename TS, typename TW>
cudaError_t launch_interp_st(const mgr_plan* p, int l, const TD* c, const TW* w, TO* out, int out_full, Slabs sl,
                             int slabs, cudaStream_t st) {
  if (slabs <= 0) return cudaSuccess;
  int gx, gy;
  InterpArgs<TS, TW> a = interp_args<TS, TW>(p, l, c, w, out, out_full, 1.0, &gx, &gy);
  const int chunks = choose_chunks(p, int64_t(gx) * gy * slabs, a.m[0], 2, kLevelMaxChunk);
  a.qz_chunk = (a.m[0] + chunks - 1) / chunks;
  sl.zchunks = (a.m[0] + a.qz_chunk - 1) / a.qz_chunk;
  constexpr size_t sm = interp_smem_bytes<kInterpNW, kInterpRPW, TD, TS, TW>();
  auto kern = k_interp_st<kInterpNW, kInterpRPW, TD, TO, TS, TW>;
  raise_smem_limit(kern, sm);
  kern<<<dim3(gx, gy, sl.zchunks * slabs), kInterpNW * 32, sm, st>>>(a, sl);
  return cudaGetLastError();
}

template <int DIR, typename TV, typename TC, typename TS>
cudaError_t launch_time_fine(const mgr_plan* p, int l, TV* v, int v_full, TC* c, cudaStream_t st) {
  const LevelGeom& g = p->geom[l];
  const int nfine = g.tax.n - g.tax.m;
  if (nfine <= 0) return cudaSuccess;
  const TS* T = table<TS>(p);
  const int64_t rows = int64_t(nfine) * g.ax[0].n * g.ax[1].n;
  const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((rows + 7) / 8, int64_t(p->ctx->num_sms) * 16)));
  k_time_fine<DIR, TV, TC, TS><<<blocks, 256, 0, st>>>(v, v_full, c, space_map(p, l), nfine, g.tax.s, g.tax.N,
                                                        space_full_count(p), T + g.tax.o_wa, T + g.tax.o_wb);
  return cudaGetLastError();
}

template <typename TW>
cudaError_t launch_time_stencil(const mgr_plan* p, int l, const TW* G, TW* F, cudaStream_t st) {
  const LevelGeom& g = p->geom[l];
  const int64_t Sm = g.space_coarse();
  const TW* T = table<TW>(p);
  k_time_stencil<TW><<<grid_1d(int64_t(g.tax.m) * Sm, 256, p), 256, 0, st>>>(G, F, g.tax.n, g.tax.m, Sm,
                                                                             T + g.tax.o_k);
  return cudaGetLastError();
}

// Solves of level l along x, y, z (each time slice) and t; the last applies
// `final_op` into w.
template <typename TW>
cudaError_t solve_level_st(const mgr_plan* p, int l, TW* f, TW* w, int final_op, cudaStream_t st) {
  const LevelGeom& g = p->geom[l];
  const int mt = g.tax.m, mz = g.ax[0].m, my = g.ax[1].m, mx = g.ax[2].m;
  const int64_t Sm = g.space_coarse();
  const TW* T = table<TW>(p);
  auto name_of = [](int axis) { return axis == 3 ? "solve_t" : (axis == 0 ? "solve_z" : axis == 1 ? "solve_y" : "solve_x"); };
  for (int axis : {2, 1, 0, 3}) {
    const AxisLevel& ax = axis == 3 ? g.tax : g.ax[axis];
    if (!ax.active) continue;
    const int op = axis == 3 ? final_op : SOLVE_INPLACE;
    const TW* ta = T + ax.o_ta;
    const TW* tb = T + ax.o_tb;
    const int64_t m = int64_t(mt) * Sm;
    rec_begin(st);
    if (axis == 2) {
      launch_x_solve<TW>(p, f, w, mx, int64_t(mt) * mz * my, ta, tb, op, st);
    } else {
      int mline, inner;
      int64_t lstride, outer, ostride;
      if (axis == 1) {
        mline = my; lstride = mx; inner = mx; outer = int64_t(mt) * mz; ostride = int64_t(my) * mx;
      } else if (axis == 0) {
        mline = mz; lstride = int64_t(my) * mx; inner = my * mx; outer = mt; ostride = Sm;
      } else {
        mline = mt; lstride = Sm; inner = int(Sm); outer = 1; ostride = 0;
      }
      const int64_t lines = int64_t(inner) * outer;
      k_solve_strided<TW><<<int((lines + 127) / 128), 128, 0, st>>>(f, w, mline, lstride, inner, outer, ostride, ta,
                                                                    tb, op);
    }
    cudaError_t e = cudaGetLastError();
    rec_end(st, name_of(axis), l, double(m) * sizeof(TW) * (op != SOLVE_INPLACE ? 4 : 2),
            double(m) * (op != SOLVE_INPLACE ? 5 : 4));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename TD, typename TW>
cudaError_t coarsest_st(const mgr_plan* p, TD* y, TW* w, int dir, cudaStream_t st) {
  const int L = p->levels;
  const int3 n0 = make_int3(int(p->coarsest[0]), int(p->coarsest[1]), int(p->coarsest[2]));
  const int64_t s0 = int64_t(1) << L;
  const longlong3 s = make_longlong3(p->full[0] > 1 ? s0 : 1, p->full[1] > 1 ? s0 : 1, s0);
  const longlong3 N = make_longlong3(p->full[0], p->full[1], p->full[2]);
  const int64_t cnt = int64_t(n0.x) * n0.y * n0.z;
  const int bx = int(std::max<int64_t>(1, std::min<int64_t>((cnt + 255) / 256, 1024)));
  rec_begin(st);
  k_coarsest_st<TD, TW><<<dim3(bx, unsigned(p->coarsest_t)), 256, 0, st>>>(
      y, p->full[1] * p->full[2], p->full[2], w, n0, s, N, s0, p->full_t, space_full_count(p), dir);
  cudaError_t e = cudaGetLastError();
  rec_end(st, "coarsest", 0, double(cnt) * p->coarsest_t * (sizeof(TD) + sizeof(TW)), 0.0);
  return e;
}

// Algorithmic bytes / flops of the spatial passes of one 4D level: the 3D
// figures of one slice times the number of slices.
Work slab_work(const mgr_plan* p, int l, bool dec, int slabs, double s_in) {
  const LevelGeom& g = p->geom[l];
  const double n = double(g.space_fine()), m = double(g.space_coarse());
  const double sd = double(p->elem), sw = double(p->welem);
  Work w;
  w.bytes = slabs * (dec ? n * s_in + (n - m) * sd + 2.0 * m * sw : n * sd + m * sw);
  w.flops = slabs * 2.0 * (5.0 * n);  // about 5 stencil FMAs per node (plus coefficients in the level pass)
  return w;
}

template <typename TD, typename TS, typename TW>
cudaError_t decompose_st_t(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st) {
  const int L = p->levels;
  if (L == 0) return cudaMemcpyAsync(out, in, size_t(p->count) * sizeof(TD), cudaMemcpyDeviceToDevice, st);
  Bufs b = split_ws(p, ws);
  TW* F = static_cast<TW*>(b.F);
  TW* G = reinterpret_cast<TW*>(static_cast<char*>(ws) + p->ws_a + p->ws_b + p->ws_f);
  TD* y = static_cast<TD*>(out);
  const int64_t Fsp = space_full_count(p);
  TW* cur = nullptr;
  NvtxRange op_range("mgr decompose 4D");
  for (int l = L; l >= 1; --l) {
    NvtxRange level_range("decompose 4D level %d", l);
    const LevelGeom& g = p->geom[l];
    const int nt = g.tax.n, mt = g.tax.m;
    const int64_t Sn = g.space_fine(), Sm = g.space_coarse();
    TW* nxt = static_cast<TW*>(((L - l) % 2 == 0) ? b.A : b.B);
    cudaError_t e;
    // D1: coarse-time slices, level pass
    {
      auto a = level_args<TS, TW>(p, l);
      a.y = out;
      a.w = nxt;
      a.f = G;
      a.write_y = 1;
      Slabs sl = base_slabs(p, l);
      sl.first = 0;
      sl.step = 2;
      sl.last = nt - 1;
      sl.w_ts = Sm;
      sl.f_ts = Sm;
      rec_begin(st);
      if (l == L) {
        a.in = in;
        a.in_full = 1;
        a.in_sz = p->full[1] * p->full[2];
        a.in_sy = p->full[2];
        sl.in_tfull = 1;
        sl.in_ts = Fsp;
        e = launch_level_st<0, TD, TD, TS, TW>(p, a, sl, mt, st);
      } else {
        a.in = cur;
        a.in_full = 0;
        a.in_sz = int64_t(g.ax[1].n) * g.ax[2].n;
        a.in_sy = g.ax[2].n;
        sl.in_tfull = 0;
        sl.in_ts = Sn;
        e = launch_level_st<0, TW, TD, TS, TW>(p, a, sl, mt, st);
      }
      const Work wk = slab_work(p, l, true, mt, double(l == L ? sizeof(TD) : sizeof(TW)));
      rec_end(st, "level_load_dec", l, wk.bytes, wk.flops);
      if (e != cudaSuccess) return e;
    }
    // D2: coefficients of the fine-time slices
    rec_begin(st);
    if (l == L)
      e = launch_time_fine<0, TD, TD, TS>(p, l, const_cast<TD*>(static_cast<const TD*>(in)), 1, y, st);
    else
      e = launch_time_fine<0, TW, TD, TS>(p, l, cur, 0, y, st);
    rec_end(st, "time_coef", l, double(nt - mt) * Sn * (3.0 * (l == L ? sizeof(TD) : sizeof(TW)) + 3.0 * sizeof(TD)),
            double(nt - mt) * Sn * 6.0);
    if (e != cudaSuccess) return e;
    // D3: load vectors of the fine-time slices
    {
      auto a = level_args<TS, TW>(p, l);
      a.in = out;
      a.in_full = 1;
      a.in_sz = p->full[1] * p->full[2];
      a.in_sy = p->full[2];
      a.f = G;
      Slabs sl = base_slabs(p, l);
      sl.first = 1;
      sl.step = 2;
      sl.last = nt - 1;
      sl.in_tfull = 1;
      sl.in_ts = Fsp;
      sl.f_ts = Sm;
      sl.fine_all = 1;
      rec_begin(st);
      e = launch_level_st<1, TD, TD, TS, TW>(p, a, sl, nt - mt, st);
      const Work wk = slab_work(p, l, false, nt - mt, 0.0);
      rec_end(st, "level_load_rec", l, wk.bytes, wk.flops);
      if (e != cudaSuccess) return e;
    }
    // D4: along time
    rec_begin(st);
    e = launch_time_stencil<TW>(p, l, G, F, st);
    rec_end(st, "time_stencil", l, double(nt + mt) * Sm * sizeof(TW), 10.0 * mt * Sm);
    if (e != cudaSuccess) return e;
    // D5: solves, correction added to the coarse nodes
    if ((e = solve_level_st<TW>(p, l, F, nxt, SOLVE_ADD, st)) != cudaSuccess) return e;
    cur = nxt;
  }
  return coarsest_st<TD, TW>(p, y, cur, 1, st);
}

template <typename TD, typename TS, typename TW>
cudaError_t recompose_st_t(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st) {
  const int L = p->levels;
  if (L == 0) return cudaMemcpyAsync(out, in, size_t(p->count) * sizeof(TD), cudaMemcpyDeviceToDevice, st);
  Bufs b = split_ws(p, ws);
  TW* F = static_cast<TW*>(b.F);
  TW* G = reinterpret_cast<TW*>(static_cast<char*>(ws) + p->ws_a + p->ws_b + p->ws_f);
  TD* c = const_cast<TD*>(static_cast<const TD*>(in));
  const int64_t Fsp = space_full_count(p);
  TW* cur = static_cast<TW*>((L % 2 == 1) ? b.A : b.B);
  cudaError_t e = coarsest_st<TD, TW>(p, c, cur, 0, st);
  if (e != cudaSuccess) return e;
  NvtxRange op_range("mgr recompose 4D");
  for (int l = 1; l <= L; ++l) {
    NvtxRange level_range("recompose 4D level %d", l);
    const LevelGeom& g = p->geom[l];
    const int nt = g.tax.n, mt = g.tax.m;
    const int64_t Sn = g.space_fine(), Sm = g.space_coarse();
    // load vectors of every slice (coarse-time slices: coefficients on their
    // 3D-fine nodes only; fine-time slices: on every node)
    {
      auto a = level_args<TS, TW>(p, l);
      a.in = in;
      a.in_full = 1;
      a.in_sz = p->full[1] * p->full[2];
      a.in_sy = p->full[2];
      a.f = G;
      Slabs sl = base_slabs(p, l);
      sl.first = 0;
      sl.step = 1;
      sl.last = nt - 1;
      sl.in_tfull = 1;
      sl.in_ts = Fsp;
      sl.f_ts = Sm;
      sl.fine_all = 1;
      rec_begin(st);
      e = launch_level_st<1, TD, TD, TS, TW>(p, a, sl, nt, st);
      const Work wk = slab_work(p, l, false, nt, 0.0);
      rec_end(st, "level_load_rec", l, wk.bytes, wk.flops);
      if (e != cudaSuccess) return e;
    }
    rec_begin(st);
    e = launch_time_stencil<TW>(p, l, G, F, st);
    rec_end(st, "time_stencil", l, double(nt + mt) * Sm * sizeof(TW), 10.0 * mt * Sm);
    if (e != cudaSuccess) return e;
    if ((e = solve_level_st<TW>(p, l, F, cur, SOLVE_SUB, st)) != cudaSuccess) return e;
    // interpolation of the coarse-time slices, then the fine-time slices
    TW* nxt = static_cast<TW*>(cur == b.A ? b.B : b.A);
    Slabs sl = base_slabs(p, l);
    sl.first = 0;
    sl.step = 2;
    sl.last = nt - 1;
    sl.w_ts = Sm;
    rec_begin(st);
    if (l == L) {
      sl.out_tfull = 1;
      sl.o_ts = Fsp;
      e = launch_interp_st<TD, TD, TS, TW>(p, l, c, cur, static_cast<TD*>(out), 1, sl, mt, st);
    } else {
      sl.out_tfull = 0;
      sl.o_ts = Sn;
      e = launch_interp_st<TD, TW, TS, TW>(p, l, c, cur, nxt, 0, sl, mt, st);
    }
    rec_end(st, "interp", l, double(mt) * Sn * (2.0 * p->elem) + double(mt) * Sm * p->welem, 2.0 * 3.0 * mt * Sn);
    if (e != cudaSuccess) return e;
    rec_begin(st);
    if (l == L)
      e = launch_time_fine<1, TD, TD, TS>(p, l, static_cast<TD*>(out), 1, c, st);
    else
      e = launch_time_fine<1, TW, TD, TS>(p, l, nxt, 0, c, st);
    rec_end(st, "time_interp", l, double(nt - mt) * Sn * (3.0 * (l == L ? sizeof(TD) : sizeof(TW)) + 3.0 * sizeof(TD)),
            double(nt - mt) * Sn * 6.0);
    if (e != cudaSuccess) return e;
    cur = nxt;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t enqueue_decompose_st(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st) {
  switch (p->form) {
    case kFormF64: return decompose_st_t<double, double, double>(p, in, out, ws, st);
    case kFormF32: return decompose_st_t<float, float, float>(p, in, out, ws, st);
    default: return decompose_st_t<float, float, double>(p, in, out, ws, st);
  }
}

cudaError_t enqueue_recompose_st(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st) {
  switch (p->form) {
    case kFormF64: return recompose_st_t<double, double, double>(p, in, out, ws, st);
    case kFormF32: return recompose_st_t<float, float, float>(p, in, out, ws, st);
    default: return recompose_st_t<float, float, double>(p, in, out, ws, st);
  }
}


// Read and clear this translation unit's bounds-check record (MGR_DEBUG_BOUNDS).
unsigned long long debug_take_st(DebugRecord* first) {
#ifdef MGR_DEBUG_BOUNDS
  DebugRecord r{};
  if (cudaMemcpyFromSymbol(&r, g_debug_record, sizeof(r)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (r.count) {
    const DebugRecord zero{};
    cudaMemcpyToSymbol(g_debug_record, &zero, sizeof(zero));
    if (first) *first = r;
  }
  return r.count;
#else
  (void)first;
  return 0;
#endif
}

}  // namespace mgr
