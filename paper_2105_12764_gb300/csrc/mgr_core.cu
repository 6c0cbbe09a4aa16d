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

#include "mgr_device.cuh"
#include "mgr_level.cuh"
#include "mgr_solve.cuh"
#include "mgr_launch.cuh"
#include "mgr_small.cuh"

// Number of coarse levels (1..ls) the single-CTA kernels take: the largest ls
// whose level grid (a few thousand nodes) and work arrays fit in shared memory.
template <typename TS, typename TW>
int small_levels(const mgr_plan* p) {
  int ls = 0;
  for (int l = 1; l <= p->levels && l <= kSmallMaxLevels; ++l) {
    const LevelGeom& g = p->geom[l];
    const size_t sm =
        small_smem_bytes<TS, TW>(g.ax[0].n, g.ax[1].n, g.ax[2].n, g.ax[0].m, g.ax[1].m, g.ax[2].m);
    if (g.space_fine() > 8192 || sm > size_t(200) * 1024 || sm > p->ctx->smem_optin) break;
    ls = l;
  }
  return ls;
}

template <typename TS, typename TW>
SmallArgs<TS, TW> small_args(const mgr_plan* p, int ls) {
  SmallArgs<TS, TW> a{};
  const TS* T = table<TS>(p);
  const TW* Tw = table<TW>(p);
  a.levels = ls;
  for (int l = 1; l <= ls; ++l)
    for (int k = 0; k < 3; ++k) {
      const AxisLevel& ax = p->geom[l].ax[k];
      a.n[l][k] = ax.n;
      a.m[l][k] = ax.m;
      a.active[l][k] = ax.active ? 1 : 0;
      a.s[l][k] = ax.s;
      a.wa[l][k] = T + ax.o_wa;
      a.wb[l][k] = T + ax.o_wb;
      a.k[l][k] = T + ax.o_k;
      a.ta[l][k] = Tw + ax.o_ta;
      a.tb[l][k] = Tw + ax.o_tb;
    }
  const int64_t s0 = int64_t(1) << p->levels;
  for (int k = 0; k < 3; ++k) {
    a.N[k] = p->full[k];
    a.n0[k] = int(p->coarsest[k]);
    a.s0[k] = p->full[k] > 1 ? s0 : 1;
  }
  a.sz = p->full[1] * p->full[2];
  a.sy = p->full[2];
  return a;
}

template <typename TD, typename TS, typename TW, bool DEC>
cudaError_t launch_small(const mgr_plan* p, SmallArgs<TS, TW>& a, cudaStream_t st) {
  const int ls = a.levels;
  const size_t sm = small_smem_bytes<TS, TW>(a.n[ls][0], a.n[ls][1], a.n[ls][2], a.m[ls][0], a.m[ls][1], a.m[ls][2]);
  auto kern = DEC ? k_small_dec<TD, TS, TW> : k_small_rec<TD, TS, TW>;
  raise_smem_limit(kern, sm);
  rec_begin(st);
  kern<<<1, kSmallThreads, sm, st>>>(a);
  cudaError_t e = cudaGetLastError();
  double nodes = 0;
  for (int l = 1; l <= ls; ++l) nodes += double(p->geom[l].fine_count());
  rec_end(st, DEC ? "small_levels_dec" : "small_levels_rec", ls, nodes * (2.0 * p->elem), 0.0);
  return e;
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

// The finest level pass of a pipelined host-buffer decomposition: part k
// covers the pass's z chunks [c0[k], c0[k+1]), waits for wait[k] (its input
// planes are on the device) and records done[k].
struct PipeParts {
  int parts;
  const int* c0;
  const cudaEvent_t* wait;
  const cudaEvent_t* done;
};

// PK: write the coefficients in the class-packed layout (class l at
// p->class_off[l]; `out` must not overlap `in`).  QZ (with PK): write int32
// codes with the bin widths bins[0..L] instead, counting saturated codes in
// *sat (when not null).  pp: run the finest level pass in parts (nodal, out
// of place, finest level tiled).
template <typename TD, typename TS, typename TW, bool PK, bool QZ = false>
cudaError_t decompose_t(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st,
                        const double* bins = nullptr, unsigned long long* sat = nullptr,
                        const PipeParts* pp = nullptr) {
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
  const int ls = (PK || QZ) ? 0 : small_levels<TS, TW>(p);  // levels ls..1 run in one CTA
  NvtxRange op_range("mgr decompose %s", PK ? (QZ ? "quantized" : "packed") : "nodal");
  for (int l = L; l > ls; --l) {
    NvtxRange level_range("decompose level %d", l);
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
      if (pp) {
        for (int k = 0; k < pp->parts; ++k) {
          if (cudaStreamWaitEvent(st, pp->wait[k], 0) != cudaSuccess) return cudaGetLastError();
          launch_level_chunks<0, TD, TY, TS, TW, PK, QZ>(p, a, pp->c0[k], pp->c0[k + 1], st);
          if (cudaEventRecord(pp->done[k], st) != cudaSuccess) return cudaGetLastError();
        }
      } else {
        launch_level<0, TD, TY, TS, TW, PK, QZ>(p, a, st);
      }
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
  if (ls >= 1) {
    NvtxRange small_range("decompose levels %d..1 in one CTA", ls);
    SmallArgs<TS, TW> sa = small_args<TS, TW>(p, ls);
    sa.vin = ls == L ? in : static_cast<const void*>(cur);
    sa.vin_full = ls == L;
    sa.out = out;
    return launch_small<TD, TS, TW, true>(p, sa, st);
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
// fk (graph capture only): the load-vector passes of all levels run on
// fk->side (the finest level's on fk->side2) ahead of the solve /
// interpolation chain on st, each level into its own load-vector buffer; st
// waits for level l's before its solves.
// The recomposition of a pipelined host-buffer call: every pass waits for
// `even` (the planes holding the coefficients of the coarser levels are on the
// device); the finest level's load-vector pass runs in parts over its z chunks
// [c0[k], c0[k+1]), part k after odd[k] (the odd planes it reads); the finest
// interpolation runs in parts over its z chunks [ic0[k], ic0[k+1]), recording
// done[k] after part k.
struct RecPipe {
  cudaEvent_t even;
  int parts;
  const int* c0;
  const cudaEvent_t* odd;
  int iparts;
  const int* ic0;
  const cudaEvent_t* done;
};

template <typename TD, typename TS, typename TW, bool PK, bool QZ = false>
cudaError_t recompose_t(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st, int ncls,
                        const double* bins = nullptr, const ForkCtx* fk = nullptr, const RecPipe* rp = nullptr) {
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
  auto Fl = [&](int l) { return reinterpret_cast<TW*>(static_cast<char*>(b.F) + p->f_off[l]); };
  // load vector of level l (Sec. II.A.2) from its coefficients, on stream s
  auto load_vector = [&](int l, cudaStream_t s) -> cudaError_t {
    NvtxRange lv_range("recompose level %d load vector", l);
    const LevelGeom& g = p->geom[l];
    auto a = level_args<TS, TW>(p, l);
    a.in = PK ? static_cast<const void*>(static_cast<const TY*>(in) + p->class_off[l]) : in;
    if (PK) {
      a.in_full = 0;
      a.in_sz = int64_t(g.ax[1].n) * g.ax[2].n;
      a.in_sy = g.ax[2].n;
    } else {
      a.in_full = 1;
      a.in_sz = a.y_sz;
      a.in_sy = a.y_sy;
    }
    a.f = Fl(l);
    a.w = nullptr;
    a.y = nullptr;
    a.write_y = 0;
    a.qs = QZ ? bins[l] : 1.0;
    rec_begin(s);
    if (rp && l == L) {
      for (int k = 0; k < rp->parts; ++k) {
        if (cudaStreamWaitEvent(s, rp->odd[k], 0) != cudaSuccess) return cudaGetLastError();
        launch_level_chunks<1, TY, TY, TS, TW, PK, QZ>(p, a, rp->c0[k], rp->c0[k + 1], s);
      }
    } else {
      launch_level<1, TY, TY, TS, TW, PK, QZ>(p, a, s);
    }
    cudaError_t e = cudaGetLastError();
    const Work wk = work_level_load(p, l, false);
    rec_end(s, "level_load_rec", l, wk.bytes, wk.flops);
    return e;
  };
  const int last_lv = std::min(L, ncls - 1);  // levels 1..last_lv have their coefficient class
  const int ls = (PK || QZ) ? 0 : small_levels<TS, TW>(p);  // levels 1..ls run in one CTA
  const bool fork = fk != nullptr && last_lv > ls && t_recorder == nullptr;
  NvtxRange op_range("mgr recompose %s", PK ? (QZ ? "dequantized" : "packed") : "nodal");
  if (rp && cudaStreamWaitEvent(st, rp->even, 0) != cudaSuccess) return cudaGetLastError();
  if (fork) {
    if (cudaEventRecord(fk->ev[0], st) != cudaSuccess || cudaStreamWaitEvent(fk->side, fk->ev[0], 0) != cudaSuccess)
      return cudaGetLastError();
    // the finest level's pass (most of the work, needed last) on its own
    // stream from the start, the coarser levels' passes in chain order on the other
    const bool finest_apart = fk->side2 != nullptr && last_lv == L && L > ls + 1;
    if (finest_apart) {
      if (cudaStreamWaitEvent(fk->side2, fk->ev[0], 0) != cudaSuccess) return cudaGetLastError();
      cudaError_t e = load_vector(L, fk->side2);
      if (e != cudaSuccess) return e;
      if ((e = cudaEventRecord(fk->ev[L], fk->side2)) != cudaSuccess) return e;
    }
    for (int l = ls + 1; l <= (finest_apart ? L - 1 : last_lv); ++l) {
      cudaError_t e = load_vector(l, fk->side);
      if (e != cudaSuccess) return e;
      if ((e = cudaEventRecord(fk->ev[l], fk->side)) != cudaSuccess) return e;
    }
  }
  // coarsest grid from the nodal positions / class 0
  TW* cur = static_cast<TW*>((L % 2 == 1) ? b.A : b.B);  // level 0 lives where decompose left it
  if (ls >= 1) {
    // levels 1..ls in one CTA; level ls's values go where the level loop keeps them
    TW* lsbuf = (ls % 2 == 1) ? static_cast<TW*>(cur == b.A ? b.B : b.A) : cur;
    SmallArgs<TS, TW> sa = small_args<TS, TW>(p, ls);
    sa.cin = in;
    sa.vout = ls == L ? out : static_cast<void*>(lsbuf);
    sa.vout_full = ls == L;
    cudaError_t e = launch_small<TD, TS, TW, false>(p, sa, st);
    if (e != cudaSuccess || ls == L) return e;
    cur = lsbuf;
  } else {
    cudaError_t e;
    if constexpr (QZ) e = coarsest_q_launch<TW, TW>(p, const_cast<int*>(static_cast<const int*>(in)), cur, bins[0], 0,
                                                    nullptr, st);
    else e = coarsest_copy_launch<TD, TW>(p, const_cast<TD*>(static_cast<const TD*>(in)), cur, PK, 0, st);
    if (e != cudaSuccess) return e;
  }
  for (int l = ls + 1; l <= L; ++l) {
    NvtxRange level_range("recompose level %d", l);
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
    cudaError_t e = fork ? cudaStreamWaitEvent(st, fk->ev[l], 0) : load_vector(l, st);
    if (e != cudaSuccess) return e;
    if ((e = solve_level<TW>(p, l, Fl(l), cur, SOLVE_SUB, st)) != cudaSuccess) return e;
    rec_begin(st);
    if (l == L && rp) {
      for (int k = 0; k < rp->iparts; ++k) {
        launch_interp_chunks<TY, TD, TS, TW, PK, QZ>(p, l, cl, cur, out, 1, st, qs, rp->ic0[k], rp->ic0[k + 1]);
        if (cudaEventRecord(rp->done[k], st) != cudaSuccess) return cudaGetLastError();
      }
    } else if (l == L) {
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

template <typename TD, typename TS, typename TW>
bool pipe_eligible_t(const mgr_plan* p) {
  const int L = p->levels;
  return L >= 1 && small_levels<TS, TW>(p) < L;
}

// Pipelined decomposition with host buffers (see PipeCtx).  Part k of the
// finest level pass covers coarse z planes [qz0, qz1); it reads level planes
// up to p(min(qz1, mz-1)) and finishes the planes 2t-1, t in (qz0, qz1],
// that are fine in z.
template <typename TD, typename TS, typename TW>
cudaError_t host_pipe_t(const mgr_plan* p, const void* host_in, void* host_out, const void* dev_in, void* dev_out,
                        void* ws, cudaStream_t st, const PipeCtx& pc) {
  const int L = p->levels;
  const int nz = int(p->full[0]), mz = p->geom[L].ax[0].m;
  const size_t plane = size_t(p->full[1]) * size_t(p->full[2]) * sizeof(TD);
  auto a = level_args<TS, TW>(p, L);
  const dim3 grid = level_grid<0>(p, a);
  const int gz = int(grid.z), qc = a.qz_chunk;
  const int parts = std::min(gz, kPipeParts);
  int c0[kPipeParts + 1];
  for (int k = 0; k <= parts; ++k) c0[k] = int((int64_t(k) * gz) / parts);
  // events: [0] start, [1 .. kPipeParts] slabs copied, [kPipeParts+1 .. 2 kPipeParts] parts done,
  // [2 kPipeParts+1] operation done, [2 kPipeParts+2] copies back done
  cudaEvent_t* h2d_ev = pc.ev + 1;
  cudaEvent_t* done_ev = pc.ev + 1 + kPipeParts;
  const cudaEvent_t end_ev = pc.ev[2 * kPipeParts + 1], back_ev = pc.ev[2 * kPipeParts + 2];
  const char* hin = static_cast<const char*>(host_in);
  char* hout = static_cast<char*>(host_out);
  char* din = static_cast<char*>(const_cast<void*>(dev_in));
  char* dout = static_cast<char*>(dev_out);
  cudaError_t e;
  if ((e = cudaEventRecord(pc.ev[0], st)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(pc.h2d, pc.ev[0], 0)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(pc.d2h, pc.ev[0], 0)) != cudaSuccess) return e;
  int next = 0;  // first plane not yet copied in
  for (int k = 0; k < parts; ++k) {
    const int qz1 = std::min(c0[k + 1] * qc, mz);
    const int hi = (k == parts - 1) ? nz - 1 : std::min(2 * std::min(qz1, mz - 1), nz - 1);
    if (hi >= next) {
      if ((e = cudaMemcpyAsync(din + size_t(next) * plane, hin + size_t(next) * plane, size_t(hi - next + 1) * plane,
                               cudaMemcpyHostToDevice, pc.h2d)) != cudaSuccess)
        return e;
      next = hi + 1;
    }
    if ((e = cudaEventRecord(h2d_ev[k], pc.h2d)) != cudaSuccess) return e;
  }
  const PipeParts pp{parts, c0, h2d_ev, done_ev};
  if ((e = decompose_t<TD, TS, TW, false>(p, dev_in, dev_out, ws, st, nullptr, nullptr, &pp)) != cudaSuccess) return e;
  for (int k = 0; k < parts; ++k) {
    if ((e = cudaStreamWaitEvent(pc.d2h, done_ev[k], 0)) != cudaSuccess) return e;
    const int qz0 = c0[k] * qc, qz1 = std::min(c0[k + 1] * qc, mz);
    const int t0 = qz0 + 1, t1 = std::min(std::min(qz1, mz - 1), (nz - 1) / 2);
    if (t1 >= t0 &&
        (e = cudaMemcpy2DAsync(hout + size_t(2 * t0 - 1) * plane, 2 * plane, dout + size_t(2 * t0 - 1) * plane,
                               2 * plane, plane, size_t(t1 - t0 + 1), cudaMemcpyDeviceToHost, pc.d2h)) != cudaSuccess)
      return e;
  }
  // the even planes, and the last plane when it has an odd index (it is coarse)
  if ((e = cudaEventRecord(end_ev, st)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(pc.d2h, end_ev, 0)) != cudaSuccess) return e;
  if ((e = cudaMemcpy2DAsync(hout, 2 * plane, dout, 2 * plane, plane, size_t((nz + 1) / 2), cudaMemcpyDeviceToHost,
                             pc.d2h)) != cudaSuccess)
    return e;
  if (nz % 2 == 0 && (e = cudaMemcpyAsync(hout + size_t(nz - 1) * plane, dout + size_t(nz - 1) * plane, plane,
                                          cudaMemcpyDeviceToHost, pc.d2h)) != cudaSuccess)
    return e;
  if ((e = cudaEventRecord(back_ev, pc.d2h)) != cudaSuccess) return e;
  return cudaStreamWaitEvent(st, back_ev, 0);
}

// Pipelined recomposition with host buffers: the even planes first (they hold
// every coefficient of the coarser levels, and the last plane of an even
// plane count), then the odd planes in slabs, each slab releasing a part of
// the finest load-vector pass; the output planes go back as each part of the
// finest interpolation finishes (part k writes planes [2 qz0, 2 qz1) , the
// last part up to the last plane).
template <typename TD, typename TS, typename TW>
cudaError_t host_rec_pipe_t(const mgr_plan* p, const void* host_in, void* host_out, const void* dev_in,
                            void* dev_out, void* ws, cudaStream_t st, const PipeCtx& pc, const ForkCtx& fk) {
  const int L = p->levels;
  const int nz = int(p->full[0]), mz = p->geom[L].ax[0].m;
  const size_t plane = size_t(p->full[1]) * size_t(p->full[2]) * sizeof(TD);
  auto a = level_args<TS, TW>(p, L);
  const int gz = int(level_grid<1>(p, a).z), qc = a.qz_chunk;
  const int parts = std::min(gz, kPipeParts);
  int c0[kPipeParts + 1];
  for (int k = 0; k <= parts; ++k) c0[k] = int((int64_t(k) * gz) / parts);
  int gx, gy;
  auto ia = interp_args<TS, TW, false>(p, L, nullptr, nullptr, nullptr, 1, 1.0, &gx, &gy);
  const int giz = interp_chunks(p, ia, gx, gy), iqc = ia.qz_chunk;
  const int iparts = std::min(giz, kPipeParts);
  int ic0[kPipeParts + 1];
  for (int k = 0; k <= iparts; ++k) ic0[k] = int((int64_t(k) * giz) / iparts);
  // events: [0] start, [1] even planes in, [2 .. kPipeParts+1] odd slabs in,
  // [kPipeParts+2 .. 2 kPipeParts+1] interpolation parts done, [2 kPipeParts+2] copies back done
  const cudaEvent_t even_ev = pc.ev[1], back_ev = pc.ev[2 * kPipeParts + 2];
  cudaEvent_t* odd_ev = pc.ev + 2;
  cudaEvent_t* done_ev = pc.ev + 2 + kPipeParts;
  const char* hin = static_cast<const char*>(host_in);
  char* hout = static_cast<char*>(host_out);
  char* din = static_cast<char*>(const_cast<void*>(dev_in));
  const char* dout = static_cast<const char*>(dev_out);
  cudaError_t e;
  if ((e = cudaEventRecord(pc.ev[0], st)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(pc.h2d, pc.ev[0], 0)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(pc.d2h, pc.ev[0], 0)) != cudaSuccess) return e;
  if ((e = cudaMemcpy2DAsync(din, 2 * plane, hin, 2 * plane, plane, size_t((nz + 1) / 2), cudaMemcpyHostToDevice,
                             pc.h2d)) != cudaSuccess)
    return e;
  if (nz % 2 == 0 && (e = cudaMemcpyAsync(din + size_t(nz - 1) * plane, hin + size_t(nz - 1) * plane, plane,
                                          cudaMemcpyHostToDevice, pc.h2d)) != cudaSuccess)
    return e;
  if ((e = cudaEventRecord(even_ev, pc.h2d)) != cudaSuccess) return e;
  int tlo = 1;  // odd planes 2t-1 not yet copied in start at t = tlo
  for (int k = 0; k < parts; ++k) {
    const int qz1 = std::min(c0[k + 1] * qc, mz);
    const int thi = (k == parts - 1) ? (nz - 1) / 2 : std::min(std::min(qz1, mz - 1), (nz - 1) / 2);
    if (thi >= tlo) {
      if ((e = cudaMemcpy2DAsync(din + size_t(2 * tlo - 1) * plane, 2 * plane, hin + size_t(2 * tlo - 1) * plane,
                                 2 * plane, plane, size_t(thi - tlo + 1), cudaMemcpyHostToDevice, pc.h2d)) !=
          cudaSuccess)
        return e;
      tlo = thi + 1;
    }
    if ((e = cudaEventRecord(odd_ev[k], pc.h2d)) != cudaSuccess) return e;
  }
  const RecPipe rp{even_ev, parts, c0, odd_ev, iparts, ic0, done_ev};
  if ((e = recompose_t<TD, TS, TW, false>(p, dev_in, dev_out, ws, st, L + 1, nullptr, &fk, &rp)) != cudaSuccess)
    return e;
  for (int k = 0; k < iparts; ++k) {
    if ((e = cudaStreamWaitEvent(pc.d2h, done_ev[k], 0)) != cudaSuccess) return e;
    const int z0 = 2 * ic0[k] * iqc;
    const int z1 = (k == iparts - 1) ? nz : std::min(2 * std::min(ic0[k + 1] * iqc, mz), nz);
    if (z1 > z0 && (e = cudaMemcpyAsync(hout + size_t(z0) * plane, dout + size_t(z0) * plane, size_t(z1 - z0) * plane,
                                        cudaMemcpyDeviceToHost, pc.d2h)) != cudaSuccess)
      return e;
  }
  if ((e = cudaEventRecord(back_ev, pc.d2h)) != cudaSuccess) return e;
  return cudaStreamWaitEvent(st, back_ev, 0);
}

}  // namespace

cudaError_t enqueue_recompose_host_pipe(const mgr_plan* p, const void* host_in, void* host_out, const void* dev_in,
                                        void* dev_out, void* ws, cudaStream_t st, const PipeCtx& pc,
                                        const ForkCtx& fk) {
  switch (p->form) {
    case kFormF64: return host_rec_pipe_t<double, double, double>(p, host_in, host_out, dev_in, dev_out, ws, st, pc, fk);
    case kFormF32: return host_rec_pipe_t<float, float, float>(p, host_in, host_out, dev_in, dev_out, ws, st, pc, fk);
    default: return host_rec_pipe_t<float, float, double>(p, host_in, host_out, dev_in, dev_out, ws, st, pc, fk);
  }
}

bool pipe_eligible(const mgr_plan* p, const void* dev_in, const void* dev_out) {
  if (!p || p->desc.ndim != 3 || dev_in == dev_out || p->levels < 1 || p->full[0] < 32) return false;
  switch (p->form) {
    case kFormF64: return pipe_eligible_t<double, double, double>(p);
    case kFormF32: return pipe_eligible_t<float, float, float>(p);
    default: return pipe_eligible_t<float, float, double>(p);
  }
}

cudaError_t enqueue_decompose_host_pipe(const mgr_plan* p, const void* host_in, void* host_out, const void* dev_in,
                                        void* dev_out, void* ws, cudaStream_t st, const PipeCtx& pc) {
  switch (p->form) {
    case kFormF64: return host_pipe_t<double, double, double>(p, host_in, host_out, dev_in, dev_out, ws, st, pc);
    case kFormF32: return host_pipe_t<float, float, float>(p, host_in, host_out, dev_in, dev_out, ws, st, pc);
    default: return host_pipe_t<float, float, double>(p, host_in, host_out, dev_in, dev_out, ws, st, pc);
  }
}

cudaError_t enqueue_decompose(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st) {
  if (p->desc.ndim == 4) return enqueue_decompose_st(p, in, out, ws, st);
  switch (p->form) {
    case kFormF64: return decompose_t<double, double, double, false>(p, in, out, ws, st);
    case kFormF32: return decompose_t<float, float, float, false>(p, in, out, ws, st);
    default: return decompose_t<float, float, double, false>(p, in, out, ws, st);
  }
}

cudaError_t enqueue_recompose(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st) {
  if (p->desc.ndim == 4) return enqueue_recompose_st(p, in, out, ws, st);
  const int all = p->levels + 1;
  switch (p->form) {
    case kFormF64: return recompose_t<double, double, double, false>(p, in, out, ws, st, all);
    case kFormF32: return recompose_t<float, float, float, false>(p, in, out, ws, st, all);
    default: return recompose_t<float, float, double, false>(p, in, out, ws, st, all);
  }
}

cudaError_t enqueue_recompose_fork(const mgr_plan* p, int kind, const void* in, int ncls, const double* bins, void* out,
                                   void* ws, cudaStream_t st, const ForkCtx& fk) {
  const ForkCtx* f = &fk;
  if (kind == 0) {
    switch (p->form) {
      case kFormF64: return recompose_t<double, double, double, false>(p, in, out, ws, st, ncls, nullptr, f);
      case kFormF32: return recompose_t<float, float, float, false>(p, in, out, ws, st, ncls, nullptr, f);
      default: return recompose_t<float, float, double, false>(p, in, out, ws, st, ncls, nullptr, f);
    }
  }
  if (kind == 1) {
    switch (p->form) {
      case kFormF64: return recompose_t<double, double, double, true>(p, in, out, ws, st, ncls, nullptr, f);
      case kFormF32: return recompose_t<float, float, float, true>(p, in, out, ws, st, ncls, nullptr, f);
      default: return recompose_t<float, float, double, true>(p, in, out, ws, st, ncls, nullptr, f);
    }
  }
  switch (p->form) {
    case kFormF64: return recompose_t<double, double, double, true, true>(p, in, out, ws, st, ncls, bins, f);
    case kFormF32: return recompose_t<float, float, float, true, true>(p, in, out, ws, st, ncls, bins, f);
    default: return recompose_t<float, float, double, true, true>(p, in, out, ws, st, ncls, bins, f);
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


// Read and clear this translation unit's bounds-check record (MGR_DEBUG_BOUNDS).
unsigned long long debug_take_core(DebugRecord* first) {
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
