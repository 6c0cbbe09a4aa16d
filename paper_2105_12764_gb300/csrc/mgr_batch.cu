// mgr_batch.cu -- batched refactoring of many independent fields of uneven
// sizes: one persistent, descriptor-driven launch per phase of the level
// loop, the whole phase sequence captured once into a CUDA graph, and tile
// shapes chosen by an autotuner.
//
// Phases follow the level loop of Sec. II.A for all fields at once, aligned by
// depth d (depth 0 = every field's finest level): for decomposition, for d =
// 0..D-1, the level pass (coefficients + load vector) of every field that has
// a level L_f - d, then the x, y and z solves of those fields (the last axis
// of each field adds the correction); then the coarsest-grid scatter.
// Recomposition runs the depths in reverse with the interpolation pass.
// Every phase is a single persistent launch whose CTAs walk a list of work
// items (field descriptor, tile, z chunk); ordering between phases comes from
// stream order inside the graph, so no CTA ever waits on another.
//
// Autotuning (Sec. III.B: an analytic model ranks the candidate launch
// shapes, the best few are measured): candidates are the level-pass tile
// (8 warps x 2 row pairs = 30x14 coarse nodes, 4 warps x 2 = 30x6, or 4 warps
// in half-warp row groups x 2 = 14x14, for fields whose coarse rows are
// short) and the z-chunk length (at most 8, 16 or 32 coarse planes, split evenly over a
// field's items).  The model charges each work item the shared-memory slots
// it streams (halo and padding included) and takes the longer of the memory
// time and the longest-processing-time schedule of the items over the
// persistent CTAs; the model's best candidate of each tile shape, the next
// best up to three, and the other chunk lengths of the fastest tile shape are
// timed on the real batch and the fastest is cached per batch shape.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <queue>
#include <string>
#include <thread>
#include <vector>

#include "mgr_internal.h"

namespace mgr {
namespace {

#include "mgr_device.cuh"
#include "mgr_level.cuh"
#include "mgr_solve.cuh"
#include "mgr_small.cuh"

// ---------------------------------------------------------------------------
// Descriptor-driven kernels (one CTA per work item, persistent grid)
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ void copy_words(T* dst, const T* src) {
  static_assert(sizeof(T) % 4 == 0, "descriptor size");
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(dst);
  for (int i = threadIdx.x; i < int(sizeof(T) / 4); i += blockDim.x) d[i] = s[i];
}

template <int MODE, int NW, int RPW, int STAGES, typename TI, typename TD, typename TS, typename TW, int LX = 32>
__global__ void __launch_bounds__(NW * 32, level_ctas_per_sm(NW)) kb_level(const LevelArgs<TS, TW>* __restrict__ args,
                                                       const int4* __restrict__ items, int n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) LevelArgs<TS, TW> sa;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int4 it = items[i];
    copy_words(&sa, args + it.x);
    __syncthreads();
    level_body<MODE, NW, RPW, STAGES, TI, TD, TS, TW, false, false, false, LX>(sa, it.y, it.z, it.w, smem_raw);
    __syncthreads();
  }
}

template <int NW, int RPW, typename TD, typename TO, typename TS, typename TW, int LX = 32>
__global__ void __launch_bounds__(NW * 32, level_ctas_per_sm(NW)) kb_interp(const InterpArgs<TS, TW>* __restrict__ args,
                                                        const int4* __restrict__ items, int n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) InterpArgs<TS, TW> sa;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int4 it = items[i];
    copy_words(&sa, args + it.x);
    __syncthreads();
    interp_body<NW, RPW, TD, TO, TS, TW, false, false, LX>(sa, it.y, it.z, it.w, smem_raw);
    __syncthreads();
  }
}

template <typename TW>
struct SolveDesc {
  TW* f;
  TW* w;
  const TW* ta;
  const TW* tb;
  int64_t lstride, ostride, count, row_pitch;  // count: lines (strided) or rows (contiguous)
  int mline, inner, op, R;
};

// Elements of a line loaded ahead of the recurrence per thread in the batched
// strided solves (build-time tunable).
#ifndef MGR_BATCH_SOLVE_U32
#define MGR_BATCH_SOLVE_U32 8
#endif
template <typename TW>
constexpr int kBatchSolveU() {
  return sizeof(TW) == 4 ? MGR_BATCH_SOLVE_U32 : 8;
}

template <typename TW>
__global__ void __launch_bounds__(128) kb_solve_strided(const SolveDesc<TW>* __restrict__ d,
                                                        const int2* __restrict__ items, int n) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int2 it = items[i];
    const SolveDesc<TW> s = d[it.x];
    const int64_t line = int64_t(it.y) * blockDim.x + threadIdx.x;
    if (line < s.count)
      solve_strided_line<TW, kBatchSolveU<TW>()>(s.f, s.w, s.mline, s.lstride, s.inner, s.ostride, s.ta, s.tb, s.op,
                                                 line,
                             max(int64_t(s.mline) * s.lstride, (s.count / s.inner) * s.ostride));
  }
}

template <typename TW>
__global__ void __launch_bounds__(128) kb_solve_contig(const SolveDesc<TW>* __restrict__ d,
                                                       const int2* __restrict__ items, int n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int2 it = items[i];
    const SolveDesc<TW> s = d[it.x];
    solve_contig_rows<TW>(s.f, s.w, s.mline, s.count, s.row_pitch, s.R, s.ta, s.tb, s.op, int64_t(it.y) * s.R,
                          smem_raw);
    __syncthreads();
  }
}

// The coarse end of every field's hierarchy (its levels of at most a few
// thousand nodes), one field per CTA: the one-CTA coarse-level bodies of the
// single-field path, over a list of fields (largest first).
#ifndef MGR_BATCH_SMALL_THREADS
#define MGR_BATCH_SMALL_THREADS 256
#endif
#ifndef MGR_BATCH_SMALL_SMEM_KB
#define MGR_BATCH_SMALL_SMEM_KB 50
#endif
constexpr int kBatchSmallThreads = MGR_BATCH_SMALL_THREADS;
constexpr int kBatchSmallCtas = 1024 / MGR_BATCH_SMALL_THREADS;  // CTAs per SM it is compiled for

template <bool DEC, typename TD, typename TS, typename TW>
__global__ void __launch_bounds__(kBatchSmallThreads, kBatchSmallCtas) kb_small(const SmallArgs<TS, TW>* __restrict__ args, int n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) SmallArgs<TS, TW> sa;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    copy_words(&sa, args + i);
    __syncthreads();
    if (DEC) small_dec_body<TD, TS, TW>(sa, smem_raw);
    else small_rec_body<TD, TS, TW>(sa, smem_raw);
    __syncthreads();
  }
}

template <typename TD, typename TW>
struct CopyDesc {
  TD* y;
  TW* w;
  int64_t y_sz, y_sy;
  int3 n;
  longlong3 s, N;
  int dir;
};

template <typename TD, typename TW>
__global__ void __launch_bounds__(256) kb_coarsest(const CopyDesc<TD, TW>* __restrict__ d, int n) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const CopyDesc<TD, TW> c = d[i];
    coarsest_copy<TD, TW>(c.y, c.y_sz, c.y_sy, c.w, c.n, c.s, c.N, c.dir, threadIdx.x, blockDim.x);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

template <typename T>
const T* table_of(const mgr_plan* p);
template <>
const double* table_of<double>(const mgr_plan* p) { return p->tables.d64; }
template <>
const float* table_of<float>(const mgr_plan* p) { return p->tables.d32; }

// Host staging of the device descriptor/item blob.
struct Blob {
  std::vector<unsigned char> host;
  size_t put(const void* p, size_t n, size_t align = 16) {
    size_t off = (host.size() + align - 1) & ~(align - 1);
    host.resize(off + n);
    std::memcpy(host.data() + off, p, n);
    return off;
  }
};

struct FieldRef {
  const mgr_plan* p;
  const void* in;
  void* out;
  char* ws;
};

// Level-pass tile candidates (NW warps x RPW row pairs per row group of LX
// lanes); chunk lengths.
struct TileCand {
  int cfg;    // 0: 8 warps x 2 row pairs (30 x 14), 1: 4 warps x 2 (30 x 6),
              // 2: 4 warps as 8 half-warp row groups x 2 (14 x 14)
  int chunk;  // coarse z planes per work item
};
constexpr int kNumCfg = 3;
inline int cfg_bx(int cfg) { return cfg == 2 ? 14 : 30; }
inline int cfg_by(int cfg) { return cfg == 1 ? 6 : 14; }
inline const char* cfg_name(int cfg) { return cfg == 0 ? "30x14" : cfg == 1 ? "30x6" : "14x14"; }

inline int ctas_per_sm(int cfg) { return cfg == 0 ? 2 : 4; }

// z-chunk length candidates of the autotuner (coarse planes per work item, at most)
#ifndef MGR_BATCH_CHUNK_MAX
#define MGR_BATCH_CHUNK_MAX 32
#endif
static_assert(MGR_BATCH_CHUNK_MAX <= kLevelMaxChunk, "level-pass chunks are at most kLevelMaxChunk planes");
#if MGR_BATCH_CHUNK_MAX > 32
constexpr int kChunks[] = {8, 16, 32, MGR_BATCH_CHUNK_MAX};
#else
constexpr int kChunks[] = {8, 16, 32};
#endif

// Coarse z planes per work item: at most `chunk`, split evenly over the items
// (33 planes in chunks of 32 are 17 + 16, not 32 + 1).
inline int balanced_chunk(int chunk, int mz) {
  mz = std::max(1, mz);
  const int items = (mz + chunk - 1) / chunk;
  return (mz + items - 1) / items;
}

template <typename TD, typename TS, typename TW>
struct Builder {
  const std::vector<FieldRef>& fields;
  int op;
  TileCand cand;
  int num_sms;
  Blob blob;
  struct PendingPhase {
    const void* fn;
    int kind;            // 0 level, 1 interp, 2 strided, 3 contig, 4 coarsest, 5 coarse levels in one CTA
    size_t desc_off, items_off;
    int n_items;
    int block;
    size_t smem;
    int grid;
  };
  std::vector<PendingPhase> pending;
  std::vector<std::function<cudaError_t(cudaStream_t)>> copies;  // levels == 0 fields

  std::vector<int> small;  // per field: its levels 1..small[f] run in one CTA (kb_small)
  size_t smem_optin;

  Builder(const std::vector<FieldRef>& f, int o, TileCand c, int sms, size_t optin)
      : fields(f), op(o), cand(c), num_sms(sms), smem_optin(optin) {
    for (const FieldRef& fr : fields) small.push_back(small_levels_of(fr.p));
  }

  // Coarse levels taken by the one-CTA phase: the largest ls whose level grid
  // has at most 8192 nodes and whose work arrays fit in kSmallSmemCap bytes
  // (two CTAs per SM).
  static constexpr size_t kSmallSmemCap = size_t(MGR_BATCH_SMALL_SMEM_KB) * 1024;
  int small_levels_of(const mgr_plan* p) const {
    int ls = 0;
    for (int l = 1; l <= p->levels && l <= kSmallMaxLevels; ++l) {
      const LevelGeom& g = p->geom[l];
      const size_t sm =
          small_smem_bytes<TS, TW>(g.ax[0].n, g.ax[1].n, g.ax[2].n, g.ax[0].m, g.ax[1].m, g.ax[2].m);
      if (g.space_fine() > 8192 || sm > kSmallSmemCap || sm > smem_optin) break;
      ls = l;
    }
    return ls;
  }
  // whether field i runs level L - d in the tiled phases
  bool tiled(size_t i, int d) const { return fields[i].p->levels - d > small[i]; }

  static char* bufA(const FieldRef& fr) { return fr.ws; }
  static char* bufB(const FieldRef& fr) { return fr.ws + fr.p->ws_a; }
  static char* bufF(const FieldRef& fr) { return fr.ws + fr.p->ws_a + fr.p->ws_b; }

  LevelArgs<TS, TW> level_args(const FieldRef& fr, int l) const {
    const mgr_plan* p = fr.p;
    const LevelGeom& g = p->geom[l];
    LevelArgs<TS, TW> a{};
    const TS* T = table_of<TS>(p);
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
    a.qz_chunk = balanced_chunk(cand.chunk, g.ax[0].m);
    return a;
  }

  // Level-pass phase for all fields at depth d.
  template <int MODE, typename TI>
  void level_phase(int d, bool first_dec) {
    std::vector<LevelArgs<TS, TW>> descs;
    std::vector<int4> items;
    const int BX = cfg_bx(cand.cfg), BY = cfg_by(cand.cfg);
    for (size_t fi = 0; fi < fields.size(); ++fi) {
      const FieldRef& fr = fields[fi];
      const int L = fr.p->levels;
      if (!tiled(fi, d)) continue;
      const int l = L - d;
      LevelArgs<TS, TW> a = level_args(fr, l);
      if (MODE == 0) {
        char* nxt = ((L - l) % 2 == 0) ? bufA(fr) : bufB(fr);
        char* cur = ((L - l - 1) % 2 == 0) ? bufA(fr) : bufB(fr);
        a.y = fr.out;
        a.w = reinterpret_cast<TW*>(nxt);
        a.f = reinterpret_cast<TW*>(bufF(fr));
        a.write_y = 1;
        if (l == L) {
          a.in = fr.in;
          a.in_full = 1;
          a.in_sz = a.y_sz;
          a.in_sy = a.y_sy;
        } else {
          const LevelGeom& g = fr.p->geom[l];
          a.in = cur;
          a.in_full = 0;
          a.in_sz = int64_t(g.ax[1].n) * g.ax[2].n;
          a.in_sy = g.ax[2].n;
        }
      } else {
        a.in = fr.in;
        a.in_full = 1;
        a.in_sz = a.y_sz;
        a.in_sy = a.y_sy;
        a.f = reinterpret_cast<TW*>(bufF(fr));
        a.w = nullptr;
        a.y = nullptr;
        a.write_y = 0;
      }
      const int di = int(descs.size());
      descs.push_back(a);
      const int gx = (a.m[2] + BX - 1) / BX, gy = (a.m[1] + BY - 1) / BY, gz = (a.m[0] + a.qz_chunk - 1) / a.qz_chunk;
      for (int z = 0; z < gz; ++z)
        for (int y = 0; y < gy; ++y)
          for (int x = 0; x < gx; ++x) items.push_back(make_int4(di, x, y, z));
    }
    (void)first_dec;
    if (items.empty()) return;
    PendingPhase ph{};
    ph.kind = 0;
    ph.desc_off = blob.put(descs.data(), descs.size() * sizeof(descs[0]));
    ph.items_off = blob.put(items.data(), items.size() * sizeof(int4));
    ph.n_items = int(items.size());
    if (cand.cfg == 0) {
      using C = LevelCfg<TS>;
      ph.fn = reinterpret_cast<const void*>(kb_level<MODE, C::NW, C::RPW, C::STAGES, TI, TD, TS, TW>);
      ph.block = C::NW * 32;
      ph.smem = level_smem_bytes<C::NW, C::RPW, C::STAGES, TI, TS>();
    } else if (cand.cfg == 1) {
      constexpr int ST = LevelCfg<TS>::STAGES;
      ph.fn = reinterpret_cast<const void*>(kb_level<MODE, 4, 2, ST, TI, TD, TS, TW>);
      ph.block = 128;
      ph.smem = level_smem_bytes<4, 2, ST, TI, TS>();
    } else {
      constexpr int ST = LevelCfg<TS>::STAGES;
      ph.fn = reinterpret_cast<const void*>(kb_level<MODE, 4, 2, ST, TI, TD, TS, TW, 16>);
      ph.block = 128;
      ph.smem = level_smem_bytes<4, 2, ST, TI, TS, 16>();
    }
    ph.grid = std::min(ph.n_items, num_sms * ctas_per_sm(cand.cfg));
    pending.push_back(ph);
  }

  template <typename TO>
  void interp_phase(int d) {
    std::vector<InterpArgs<TS, TW>> descs;
    std::vector<int4> items;
#ifndef MGR_BATCH_INTERP_NW
#define MGR_BATCH_INTERP_NW 1
#endif
#ifndef MGR_BATCH_INTERP_LX
#define MGR_BATCH_INTERP_LX 16
#endif
    // tiles of LX x BY coarse nodes: half-warp row groups fit the short coarse
    // rows of the batch's fields better than whole warps
    constexpr int NW = MGR_BATCH_INTERP_NW, RPW = 2, LX = MGR_BATCH_INTERP_LX, BY = NW * 32 / LX * RPW;
    for (size_t fi = 0; fi < fields.size(); ++fi) {
      const FieldRef& fr = fields[fi];
      const int L = fr.p->levels;
      if (!tiled(fi, d)) continue;
      const int l = L - d;
      const mgr_plan* p = fr.p;
      const LevelGeom& g = p->geom[l];
      const TS* T = table_of<TS>(p);
      InterpArgs<TS, TW> a{};
      for (int k = 0; k < 3; ++k) {
        a.n[k] = g.ax[k].n;
        a.m[k] = g.ax[k].m;
        a.s[k] = g.ax[k].s;
        a.N[k] = g.ax[k].N;
        a.wa[k] = T + g.ax[k].o_wa;
        a.wb[k] = T + g.ax[k].o_wb;
      }
      // the coarse values of level l-1 and the level-l destination
      char* cur = ((L - l) % 2 == 0) ? bufA(fr) : bufB(fr);
      char* nxt = ((L - l + 1) % 2 == 0) ? bufA(fr) : bufB(fr);
      a.c = fr.in;
      a.y_sz = p->full[1] * p->full[2];
      a.y_sy = p->full[2];
      a.w = reinterpret_cast<const TW*>(cur);
      a.c_sz = int64_t(g.ax[1].m) * g.ax[2].m;
      a.c_sy = g.ax[2].m;
      const bool last = (l == L);
      a.out = last ? fr.out : static_cast<void*>(nxt);
      a.out_full = last ? 1 : 0;
      a.o_sz = last ? a.y_sz : int64_t(g.ax[1].n) * g.ax[2].n;
      a.o_sy = last ? a.y_sy : int64_t(g.ax[2].n);
      a.qz_chunk = balanced_chunk(cand.chunk, g.ax[0].m);
      const int di = int(descs.size());
      descs.push_back(a);
      const int gx = (a.m[2] + LX - 1) / LX, gy = (a.m[1] + BY - 1) / BY, gz = (a.m[0] + a.qz_chunk - 1) / a.qz_chunk;
      for (int z = 0; z < gz; ++z)
        for (int y = 0; y < gy; ++y)
          for (int x = 0; x < gx; ++x) items.push_back(make_int4(di, x, y, z));
    }
    if (items.empty()) return;
    PendingPhase ph{};
    ph.kind = 1;
    ph.desc_off = blob.put(descs.data(), descs.size() * sizeof(descs[0]));
    ph.items_off = blob.put(items.data(), items.size() * sizeof(int4));
    ph.n_items = int(items.size());
    ph.fn = reinterpret_cast<const void*>(kb_interp<NW, RPW, TD, TO, TS, TW, LX>);
    ph.block = NW * 32;
    ph.smem = interp_smem_bytes<NW, RPW, TD, TS, TW, LX>();
    ph.grid = std::min(ph.n_items, num_sms * level_ctas_per_sm(NW));
    pending.push_back(ph);
  }

  // Solves of all fields at depth d along `axis`; fields whose last active
  // axis is `axis` apply the correction with `final_op`.
  void solve_phase(int d, int axis, int final_op) {
    std::vector<SolveDesc<TW>> sdesc, cdesc;
    std::vector<int2> sitems, citems;
    size_t csmem = 0;
    for (size_t fi = 0; fi < fields.size(); ++fi) {
      const FieldRef& fr = fields[fi];
      const int L = fr.p->levels;
      if (!tiled(fi, d)) continue;
      const int l = L - d;
      const LevelGeom& g = fr.p->geom[l];
      if (!g.ax[axis].active) continue;
      int last = -1;
      for (int a2 = 2; a2 >= 0; --a2)
        if (g.ax[a2].active) last = a2;
      const TW* T = table_of<TW>(fr.p);
      const int mz = g.ax[0].m, my = g.ax[1].m, mx = g.ax[2].m;
      SolveDesc<TW> s{};
      s.f = reinterpret_cast<TW*>(bufF(fr));
      s.w = reinterpret_cast<TW*>(((L - l) % 2 == 0) ? bufA(fr) : bufB(fr));
      s.ta = T + g.ax[axis].o_ta;
      s.tb = T + g.ax[axis].o_tb;
      s.op = (axis == last) ? final_op : SOLVE_INPLACE;
      if (axis == 2 && solve_contig_smem<TW>(mx, 1) <= 96 * 1024) {
        const int pitch = contig_pitch<TW>(mx);
        int R = int(std::min<size_t>(32, (32 * 1024) / (sizeof(TW) * pitch)));
        R = std::max(1, R);
        s.mline = mx;
        s.count = int64_t(mz) * my;
        s.row_pitch = mx;
        s.R = R;
        csmem = std::max(csmem, solve_contig_smem<TW>(mx, R));
        const int di = int(cdesc.size());
        cdesc.push_back(s);
        const int64_t blocks = (s.count + R - 1) / R;
        for (int64_t b = 0; b < blocks; ++b) citems.push_back(make_int2(di, int(b)));
      } else {
        if (axis == 2) {
          s.mline = mx; s.lstride = 1; s.inner = 1; s.ostride = mx; s.count = int64_t(mz) * my;
        } else if (axis == 1) {
          s.mline = my; s.lstride = mx; s.inner = mx; s.ostride = int64_t(my) * mx; s.count = int64_t(mz) * mx;
        } else {
          s.mline = mz; s.lstride = int64_t(my) * mx; s.inner = mx; s.ostride = mx; s.count = int64_t(my) * mx;
        }
        const int di = int(sdesc.size());
        sdesc.push_back(s);
        const int64_t blocks = (s.count + 127) / 128;
        for (int64_t b = 0; b < blocks; ++b) sitems.push_back(make_int2(di, int(b)));
      }
    }
    if (!citems.empty()) {
      PendingPhase ph{};
      ph.kind = 3;
      ph.desc_off = blob.put(cdesc.data(), cdesc.size() * sizeof(cdesc[0]));
      ph.items_off = blob.put(citems.data(), citems.size() * sizeof(int2));
      ph.n_items = int(citems.size());
      ph.fn = reinterpret_cast<const void*>(kb_solve_contig<TW>);
      ph.block = 128;
      ph.smem = csmem;
      ph.grid = std::min<int>(ph.n_items, num_sms * 6);
      pending.push_back(ph);
    }
    if (!sitems.empty()) {
      PendingPhase ph{};
      ph.kind = 2;
      ph.desc_off = blob.put(sdesc.data(), sdesc.size() * sizeof(sdesc[0]));
      ph.items_off = blob.put(sitems.data(), sitems.size() * sizeof(int2));
      ph.n_items = int(sitems.size());
      ph.fn = reinterpret_cast<const void*>(kb_solve_strided<TW>);
      ph.block = 128;
      ph.smem = 0;
      ph.grid = std::min<int>(ph.n_items, num_sms * 8);
      pending.push_back(ph);
    }
  }

  void coarsest_phase(int dir) {
    std::vector<CopyDesc<TD, TW>> descs;
    for (size_t fi = 0; fi < fields.size(); ++fi) {
      const FieldRef& fr = fields[fi];
      const mgr_plan* p = fr.p;
      const int L = p->levels;
      if (L == 0 || small[fi] > 0) continue;  // the one-CTA phase handles the coarsest grid
      CopyDesc<TD, TW> c{};
      c.y = static_cast<TD*>(dir == 1 ? fr.out : const_cast<void*>(fr.in));
      // level-0 values: where the last decomposition level wrote them / where
      // the first recomposition level reads them (same ping-pong rule)
      c.w = reinterpret_cast<TW*>((L % 2 == 1) ? bufA(fr) : bufB(fr));
      c.y_sz = p->full[1] * p->full[2];
      c.y_sy = p->full[2];
      c.n = make_int3(int(p->coarsest[0]), int(p->coarsest[1]), int(p->coarsest[2]));
      const int64_t s0 = int64_t(1) << L;
      c.s = make_longlong3(p->full[0] > 1 ? s0 : 1, p->full[1] > 1 ? s0 : 1, s0);
      c.N = make_longlong3(p->full[0], p->full[1], p->full[2]);
      c.dir = dir;
      descs.push_back(c);
    }
    if (descs.empty()) return;
    PendingPhase ph{};
    ph.kind = 4;
    ph.desc_off = blob.put(descs.data(), descs.size() * sizeof(descs[0]));
    ph.items_off = 0;
    ph.n_items = int(descs.size());
    ph.fn = reinterpret_cast<const void*>(kb_coarsest<TD, TW>);
    ph.block = 256;
    ph.smem = 0;
    ph.grid = std::min(ph.n_items, num_sms * 8);
    pending.push_back(ph);
  }

  // The one-CTA phase: every field's levels small[f]..1 (decomposition: after
  // its tiled levels; recomposition: before them), largest first.
  void small_phase(bool dec) {
    std::vector<std::pair<size_t, size_t>> order;  // (shared memory, field)
    for (size_t fi = 0; fi < fields.size(); ++fi) {
      const int ls = small[fi];
      if (ls < 1) continue;
      const LevelGeom& g = fields[fi].p->geom[ls];
      order.push_back({small_smem_bytes<TS, TW>(g.ax[0].n, g.ax[1].n, g.ax[2].n, g.ax[0].m, g.ax[1].m, g.ax[2].m), fi});
    }
    if (order.empty()) return;
    std::sort(order.begin(), order.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    std::vector<SmallArgs<TS, TW>> descs;
    for (const auto& o : order) {
      const FieldRef& fr = fields[o.second];
      const mgr_plan* p = fr.p;
      const int L = p->levels, ls = small[o.second];
      SmallArgs<TS, TW> a{};
      const TS* T = table_of<TS>(p);
      const TW* Tw = table_of<TW>(p);
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
      const int64_t s0 = int64_t(1) << L;
      for (int k = 0; k < 3; ++k) {
        a.N[k] = p->full[k];
        a.n0[k] = int(p->coarsest[k]);
        a.s0[k] = p->full[k] > 1 ? s0 : 1;
      }
      a.sz = p->full[1] * p->full[2];
      a.sy = p->full[2];
      // level-ls values: the field itself when every level is small, else the
      // coarse buffer the tiled level ls+1 writes (decomposition) / the
      // interpolation of level ls+1 reads (recomposition)
      char* lsbuf = ((L - ls - 1) % 2 == 0) ? bufA(fr) : bufB(fr);
      if (dec) {
        a.vin = ls == L ? fr.in : static_cast<const void*>(lsbuf);
        a.vin_full = ls == L;
        a.out = fr.out;
      } else {
        a.cin = fr.in;
        a.vout = ls == L ? fr.out : static_cast<void*>(lsbuf);
        a.vout_full = ls == L;
      }
      descs.push_back(a);
    }
    PendingPhase ph{};
    ph.kind = 5;
    ph.desc_off = blob.put(descs.data(), descs.size() * sizeof(descs[0]));
    ph.items_off = 0;
    ph.n_items = int(descs.size());
    ph.fn = dec ? reinterpret_cast<const void*>(kb_small<true, TD, TS, TW>)
                : reinterpret_cast<const void*>(kb_small<false, TD, TS, TW>);
    ph.block = kBatchSmallThreads;
    ph.smem = order.front().first;
    ph.grid = std::min(ph.n_items, num_sms * kBatchSmallCtas);
    pending.push_back(ph);
  }

  void build() {
    int D = 0;
    for (const FieldRef& fr : fields) D = std::max(D, fr.p->levels);
    for (const FieldRef& fr : fields) {
      if (fr.p->levels == 0 && fr.in != fr.out) {
        const FieldRef f = fr;
        copies.push_back([f](cudaStream_t st) {
          return cudaMemcpyAsync(f.out, f.in, size_t(f.p->count) * f.p->elem, cudaMemcpyDeviceToDevice, st);
        });
      }
    }
    if (op == 0) {
      for (int d = 0; d < D; ++d) {
        if (d == 0) level_phase<0, TD>(d, true);
        else level_phase<0, TW>(d, false);
        solve_phase(d, 2, SOLVE_ADD);
        solve_phase(d, 1, SOLVE_ADD);
        solve_phase(d, 0, SOLVE_ADD);
      }
      small_phase(true);
      coarsest_phase(1);
    } else {
      coarsest_phase(0);
      small_phase(false);
      for (int d = D - 1; d >= 0; --d) {
        level_phase<1, TD>(d, false);
        solve_phase(d, 2, SOLVE_SUB);
        solve_phase(d, 1, SOLVE_SUB);
        solve_phase(d, 0, SOLVE_SUB);
        if (d == 0) interp_phase<TD>(d);
        else interp_phase<TW>(d);
      }
    }
  }

  // Estimated time of this candidate (model of Sec. III.B, restated): every
  // level-pass item streams RR x RC slots per plane pair (halo and padding
  // included); the phase takes the longer of that traffic at HBM speed and
  // the LPT schedule of the items over the persistent CTAs.
  double model_cost(double hbm_bytes_per_us) const {
    double total = 0;
    const int BX = cfg_bx(cand.cfg), BY = cfg_by(cand.cfg);
    const int RR = 2 * (BY + 2), RC = 2 * (BX + 2);
    const int slots = num_sms * ctas_per_sm(cand.cfg);
    const double t_iter_us = (cand.cfg == 0 ? 1.6 : 1.0);
    int D = 0;
    for (const FieldRef& fr : fields) D = std::max(D, fr.p->levels);
    for (int d = 0; d < D; ++d) {
      std::vector<double> jobs;
      double bytes = 0;
      for (size_t fi = 0; fi < fields.size(); ++fi) {
        const FieldRef& fr = fields[fi];
        const int L = fr.p->levels;
        if (!tiled(fi, d)) continue;
        const LevelGeom& g = fr.p->geom[L - d];
        const int chunk = balanced_chunk(cand.chunk, g.ax[0].m);
        const int gx = (g.ax[2].m + BX - 1) / BX, gy = (g.ax[1].m + BY - 1) / BY;
        const int gz = (g.ax[0].m + chunk - 1) / chunk;
        for (int z = 0; z < gz; ++z) {
          const int planes = std::min(chunk, g.ax[0].m - z * chunk) + 1;
          for (int i = 0; i < gx * gy; ++i) {
            jobs.push_back(planes * t_iter_us + 2.0);
            bytes += double(planes) * 2.0 * RR * RC * fr.p->elem;
          }
        }
      }
      std::sort(jobs.begin(), jobs.end(), std::greater<double>());
      std::priority_queue<double, std::vector<double>, std::greater<double>> q;
      for (int i = 0; i < std::min<int>(slots, int(jobs.size())); ++i) q.push(0.0);
      for (double j : jobs) {
        double t = q.top();
        q.pop();
        q.push(t + j);
      }
      double makespan = 0;
      while (!q.empty()) {
        makespan = std::max(makespan, q.top());
        q.pop();
      }
      total += std::max(makespan, bytes / hbm_bytes_per_us);
    }
    return total;
  }
};

// Launch-ready batch: device blob (descriptors, items) and the phase list.
struct BatchExec {
  void* dev = nullptr;
  size_t dev_bytes = 0;
  struct L {
    const void* fn;
    int kind;
    const void* desc;
    const void* items;
    int n;
    dim3 grid, block;
    size_t smem;
  };
  std::vector<L> launches;
  std::vector<std::function<cudaError_t(cudaStream_t)>> copies;
  cudaGraphExec_t graph = nullptr;
  mutable std::string failed;  // the launch that failed last, for the tuning report
  ~BatchExec() {
    if (graph) cudaGraphExecDestroy(graph);
    if (dev) cudaFree(dev);
  }
  cudaError_t enqueue(cudaStream_t st) const {
    static const char* kinds[] = {"level pass", "interpolation", "strided solves", "contiguous solves",
                                  "coarsest copy", "coarse levels in one CTA"};
    NvtxRange op_range("mgr batch: %d phases", int(launches.size()));
    for (auto& c : copies) {
      const cudaError_t e = c(st);
      if (e != cudaSuccess) {
        failed = std::string("copy of a field without levels: ") + cudaGetErrorName(e);
        return e;
      }
    }
    for (const L& l : launches) {
      NvtxRange phase_range("batch phase: %s", kinds[l.kind]);
      cudaError_t e = raise_smem_limit(l.fn, l.smem);
      if (e == cudaSuccess) {
        if (l.kind == 4 || l.kind == 5) {
          void* args[] = {const_cast<void**>(&l.desc), const_cast<int*>(&l.n)};
          e = cudaLaunchKernel(l.fn, l.grid, l.block, args, l.smem, st);
        } else {
          void* args[] = {const_cast<void**>(&l.desc), const_cast<void**>(&l.items), const_cast<int*>(&l.n)};
          e = cudaLaunchKernel(l.fn, l.grid, l.block, args, l.smem, st);
        }
      }
      if (e != cudaSuccess) {
        char b[192];
        std::snprintf(b, sizeof(b), "%s (grid %u, block %u, %zu B shared memory, %d items): %s", kinds[l.kind],
                      l.grid.x, l.block.x, l.smem, l.n, cudaGetErrorName(e));
        failed = b;
        return e;
      }
    }
    return cudaGetLastError();
  }
};

template <typename TD, typename TS, typename TW>
int make_exec(const std::vector<FieldRef>& fields, int op, TileCand cand, int num_sms, size_t optin,
              std::unique_ptr<BatchExec>& out) {
  Builder<TD, TS, TW> b(fields, op, cand, num_sms, optin);
  b.build();
  auto ex = std::make_unique<BatchExec>();
  ex->dev_bytes = std::max<size_t>(b.blob.host.size(), 16);
  if (cudaMalloc(&ex->dev, ex->dev_bytes) != cudaSuccess) {
    cudaGetLastError();
    return MGR_ENOMEM;
  }
  if (!b.blob.host.empty() &&
      cudaMemcpy(ex->dev, b.blob.host.data(), b.blob.host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return MGR_ECUDA;
  char* base = static_cast<char*>(ex->dev);
  for (auto& ph : b.pending) {
    BatchExec::L l{};
    l.fn = ph.fn;
    l.kind = ph.kind;
    l.desc = base + ph.desc_off;
    l.items = base + ph.items_off;
    l.n = ph.n_items;
    l.grid = dim3(std::max(1, ph.grid));
    l.block = dim3(ph.block);
    l.smem = ph.smem;
    ex->launches.push_back(l);
  }
  ex->copies = std::move(b.copies);
  out = std::move(ex);
  return MGR_OK;
}

template <typename TD, typename TS, typename TW>
double model_of(const std::vector<FieldRef>& fields, int op, TileCand cand, int num_sms, size_t optin) {
  Builder<TD, TS, TW> b(fields, op, cand, num_sms, optin);
  return b.model_cost(6.79e6 * 0.6);  // bytes per microsecond at ~60% of the measured copy bandwidth
}

}  // namespace

// ---------------------------------------------------------------------------
// Batch state owned by the context
// ---------------------------------------------------------------------------
struct BatchState {
  cudaStream_t stream = nullptr;
  std::mutex mu;
  uint64_t next_ticket = 1;
  struct Ticket {
    cudaEvent_t done;
    int n;
  };
  std::map<uint64_t, Ticket> tickets;
  // executable batches keyed by the request list
  struct Entry {
    std::vector<const void*> key;  // op, then (plan, in, out) of every request
    void* ws = nullptr;
    size_t ws_bytes = 0;
    std::unique_ptr<BatchExec> exec;
    uint64_t last_use = 0;
  };
  std::vector<std::unique_ptr<Entry>> entries;
  size_t held_bytes = 0;
  uint64_t clock = 0;
  // autotune decisions keyed by the batch shape
  std::map<std::string, TileCand> tuned;
  std::map<std::string, std::vector<std::pair<TileCand, double>>> tune_log;
  std::map<std::string, bool> from_file;  // decision read from the persisted cache
  std::map<std::string, std::string> tune_note;  // the launch a failed candidate stopped at
};

namespace {

std::string shape_key(const std::vector<const mgr_plan*>& plans, int op, int form) {
  std::string k = std::to_string(op) + ":" + std::to_string(form) + ":";
  std::vector<std::string> parts;
  for (const mgr_plan* p : plans) {
    char buf[96];
    std::snprintf(buf, sizeof(buf), "%lldx%lldx%lld/%d", (long long)p->full[0], (long long)p->full[1],
                  (long long)p->full[2], p->levels);
    parts.push_back(buf);
  }
  std::sort(parts.begin(), parts.end());
  for (auto& s : parts) k += s + ",";
  return k;
}

template <typename TD, typename TS, typename TW>
int exec_for(mgr_ctx* ctx, BatchState& B, const std::vector<FieldRef>& fields, int op, const std::string& skey,
             TileCand cand, std::unique_ptr<BatchExec>& out) {
  (void)B;
  (void)skey;
  return make_exec<TD, TS, TW>(fields, op, cand, ctx->num_sms, ctx->smem_optin, out);
}

// Time one candidate on the real batch (graph-less, after one warm-up run).
// A candidate that fails (a launch refused, or any CUDA error while it runs)
// returns minus its CUDA error code: it is never the fastest, and the tuning
// report names the error.
template <typename TD, typename TS, typename TW>
double time_candidate(mgr_ctx* ctx, const std::vector<FieldRef>& fields, int op, TileCand cand, cudaStream_t st,
                      std::string* failed) {
  std::unique_ptr<BatchExec> ex;
  if (make_exec<TD, TS, TW>(fields, op, cand, ctx->num_sms, ctx->smem_optin, ex) != MGR_OK)
    return -double(cudaErrorMemoryAllocation);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaError_t e = ex->enqueue(st);
  cudaEventRecord(a, st);
  if (e == cudaSuccess) e = ex->enqueue(st);
  cudaEventRecord(b, st);
  float ms = 0.f;
  const cudaError_t es = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = es;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaGetLastError();
  if (e != cudaSuccess && failed && !ex->failed.empty()) *failed = ex->failed;
  return e == cudaSuccess ? double(ms) : -double(e);
}

// Persisted decisions: the environment variable MGR_AUTOTUNE_CACHE names a
// text file of lines "<gpu> <shape> <tile> <chunk>" -- the GPU as its name
// (spaces as '_') and SM count, the batch shape as the FNV-1a hash of its key
// (operation, form, every field's shape and depth), the tile shape index and
// the chunk length.  A decision found there is used without timing; a new
// one is appended.  Read and written on each tuning (no file: nothing kept).
std::string gpu_key(int device) {
  cudaDeviceProp pr{};
  if (cudaGetDeviceProperties(&pr, device) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string k = pr.name;
  for (char& ch : k)
    if (ch == ' ' || ch == '\t') ch = '_';
  return k + "_sm" + std::to_string(pr.multiProcessorCount);
}

unsigned long long shape_hash(const std::string& skey) {
  unsigned long long h = 1469598103934665603ull;
  for (unsigned char ch : skey) {
    h ^= ch;
    h *= 1099511628211ull;
  }
  return h;
}

bool cache_lookup(const char* path, const std::string& gk, unsigned long long h, TileCand* out) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char g[256];
  unsigned long long hh = 0;
  int cfg = 0, chunk = 0;
  bool found = false;
  while (std::fscanf(f, "%255s %llx %d %d", g, &hh, &cfg, &chunk) == 4) {
    bool known = false;
    for (int c : kChunks) known |= chunk == c;
    if (gk == g && hh == h && cfg >= 0 && cfg < kNumCfg && known) {
      *out = TileCand{cfg, chunk};  // the last matching line wins
      found = true;
    }
  }
  std::fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& gk, unsigned long long h, TileCand c) {
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %llx %d %d\n", gk.c_str(), h, c.cfg, c.chunk);
  std::fclose(f);
}

template <typename TD, typename TS, typename TW>
TileCand autotune(mgr_ctx* ctx, BatchState& B, const std::vector<FieldRef>& fields, int op, const std::string& skey) {
  auto it = B.tuned.find(skey);
  if (it != B.tuned.end()) return it->second;
  const char* path = std::getenv("MGR_AUTOTUNE_CACHE");
  const bool persist = path && *path;
  const std::string gk = persist ? gpu_key(ctx->device) : std::string();
  const unsigned long long h = persist ? shape_hash(skey) : 0ull;
  if (persist) {
    TileCand c{};
    if (cache_lookup(path, gk, h, &c)) {
      B.tuned[skey] = c;
      B.tune_log[skey] = {};
      B.from_file[skey] = true;
      return c;
    }
  }
  std::vector<std::pair<double, TileCand>> ranked;
  for (int cfg = 0; cfg < kNumCfg; ++cfg)
    for (int chunk : kChunks) {
      TileCand c{cfg, chunk};
      ranked.push_back({model_of<TD, TS, TW>(fields, op, c, ctx->num_sms, ctx->smem_optin), c});
    }
  std::sort(ranked.begin(), ranked.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
  // measured: the model's best candidate of every tile shape, then the next
  // best overall up to three, then every other chunk length of the fastest
  // tile shape
  std::vector<TileCand> timed;
  for (int cfg = 0; cfg < kNumCfg; ++cfg)
    for (const auto& r : ranked)
      if (r.second.cfg == cfg) {
        timed.push_back(r.second);
        break;
      }
  for (const auto& r : ranked) {
    if (timed.size() >= 3) break;
    bool seen = false;
    for (const TileCand& c : timed) seen |= c.cfg == r.second.cfg && c.chunk == r.second.chunk;
    if (!seen) timed.push_back(r.second);
  }
  TileCand best = ranked[0].second;
  double best_ms = 1e30;
  std::vector<std::pair<TileCand, double>> log;
  auto time_one = [&](const TileCand& c) {
    std::string why;
    const double ms = time_candidate<TD, TS, TW>(ctx, fields, op, c, B.stream, &why);
    log.push_back({c, ms});
    if (!why.empty()) B.tune_note[skey] = why;
    if (ms >= 0.0 && ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  };
  for (const TileCand& c : timed) time_one(c);
  // then the other chunk lengths of the fastest tile shape
  if (best_ms < 1e30) {
    const int cfg = best.cfg;
    for (int chunk : kChunks) {
      bool seen = false;
      for (const TileCand& c : timed) seen |= c.cfg == cfg && c.chunk == chunk;
      if (!seen) time_one(TileCand{cfg, chunk});
    }
  }
  B.tuned[skey] = best;
  B.tune_log[skey] = log;
  if (persist) cache_store(path, gk, h, best);
  return best;
}

template <typename TD, typename TS, typename TW>
int run_group(mgr_ctx* ctx, BatchState& B, const std::vector<const mgr_request*>& reqs, int op) {
  // workspace / executable lookup keyed by the exact request list (a vector of
  // pointers: a resubmitted list is found with one comparison per entry)
  std::vector<const void*> key;
  key.reserve(1 + 3 * reqs.size());
  key.push_back(reinterpret_cast<const void*>(uintptr_t(op)));
  size_t ws_total = 0;
  for (const mgr_request* r : reqs) {
    key.push_back(r->plan);
    key.push_back(r->in);
    key.push_back(r->out);
    ws_total += (r->plan->ws_bytes + 255) & ~size_t(255);
  }
  BatchState::Entry* ent = nullptr;
  for (auto& e : B.entries)
    if (e->key == key) ent = e.get();
  if (!ent) {
    std::vector<const mgr_plan*> plans;
    plans.reserve(reqs.size());
    for (const mgr_request* r : reqs) plans.push_back(r->plan);
    const std::string skey = shape_key(plans, op, reqs[0]->plan->form);
    if (ctx->budget && ws_total > ctx->budget) return MGR_EBUDGET;
    // evict least recently used entries until the new workspace fits the budget
    while (ctx->budget && B.held_bytes + ws_total > ctx->budget && !B.entries.empty()) {
      cudaStreamSynchronize(B.stream);
      auto victim = std::min_element(B.entries.begin(), B.entries.end(),
                                     [](const auto& x, const auto& y) { return x->last_use < y->last_use; });
      B.held_bytes -= (*victim)->ws_bytes;
      cudaFree((*victim)->ws);
      B.entries.erase(victim);
    }
    auto e = std::make_unique<BatchState::Entry>();
    e->key = std::move(key);
    e->ws_bytes = std::max<size_t>(ws_total, 256);
    if (fault_injected("alloc")) return MGR_ENOMEM;
    if (cudaMalloc(&e->ws, e->ws_bytes) != cudaSuccess) {
      cudaGetLastError();
      return MGR_ENOMEM;
    }
    std::vector<FieldRef> fields;
    char* w = static_cast<char*>(e->ws);
    for (const mgr_request* r : reqs) {
      fields.push_back(FieldRef{r->plan, r->in, r->out, w});
      w += (r->plan->ws_bytes + 255) & ~size_t(255);
    }
    const TileCand cand = autotune<TD, TS, TW>(ctx, B, fields, op, skey);
    int rc = exec_for<TD, TS, TW>(ctx, B, fields, op, skey, cand, e->exec);
    if (rc != MGR_OK) {
      cudaFree(e->ws);
      return rc;
    }
    // capture the phase sequence once
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
      cudaFree(e->ws);
      return MGR_ECUDA;
    }
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
      cudaError_t e2 = e->exec->enqueue(cs);
      ce = cudaStreamEndCapture(cs, &g);
      if (e2 != cudaSuccess) ce = e2;
    }
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&e->exec->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (ce != cudaSuccess) {
      cudaGetLastError();
      cudaFree(e->ws);
      return MGR_ECUDA;
    }
    B.held_bytes += e->ws_bytes;
    ent = e.get();
    B.entries.push_back(std::move(e));
  }
  ent->last_use = ++B.clock;
  return cudaGraphLaunch(ent->exec->graph, B.stream) == cudaSuccess ? MGR_OK : MGR_ECUDA;
}

BatchState* state_of(mgr_ctx* ctx) {
  if (!ctx->batch) {
    auto* s = new BatchState();
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete s;
      return nullptr;
    }
    ctx->batch = s;
  }
  return static_cast<BatchState*>(ctx->batch);
}

}  // namespace

void batch_destroy(mgr_ctx* ctx) {
  if (!ctx->batch) return;
  BatchState* s = static_cast<BatchState*>(ctx->batch);
  cudaStreamSynchronize(s->stream);
  for (auto& t : s->tickets) cudaEventDestroy(t.second.done);
  for (auto& e : s->entries) cudaFree(e->ws);
  s->entries.clear();
  cudaStreamDestroy(s->stream);
  delete s;
  ctx->batch = nullptr;
}

int batch_submit(mgr_ctx* ctx, const mgr_request* reqs, int n, uint64_t* ticket) {
  if (!ctx || !ticket || n < 0 || (n > 0 && !reqs)) return MGR_EINVAL;
  *ticket = 0;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return MGR_ECUDA;
  BatchState* B = state_of(ctx);
  if (!B) return MGR_ECUDA;
  std::lock_guard<std::mutex> lk(B->mu);
  std::vector<const mgr_request*> dec, rec;
  int form = -1;
  for (int i = 0; i < n; ++i) {
    const mgr_request& r = reqs[i];
    if (!r.plan || !r.in || !r.out || r.in == r.out) return MGR_EINVAL;
    if (r.plan->ctx != ctx) return MGR_EINVAL;
    if (r.plan->desc.ndim == 4) return MGR_EINVAL;  // the batched kernels are 1D-3D
    if (form < 0) form = r.plan->form;
    if (r.plan->form != form) return MGR_EINVAL;
    if (r.op == 0) dec.push_back(&r);
    else if (r.op == 1) rec.push_back(&r);
    else return MGR_EINVAL;
  }
  if (fault_injected("launch")) return MGR_ECUDA;
  int rc = MGR_OK;
  for (int pass = 0; pass < 2 && rc == MGR_OK; ++pass) {
    auto& grp = pass == 0 ? dec : rec;
    if (grp.empty()) continue;
    switch (form) {
      case kFormF64: rc = run_group<double, double, double>(ctx, *B, grp, pass); break;
      case kFormF32: rc = run_group<float, float, float>(ctx, *B, grp, pass); break;
      default: rc = run_group<float, float, double>(ctx, *B, grp, pass); break;
    }
  }
  if (rc != MGR_OK) return rc;
  BatchState::Ticket t{};
  if (cudaEventCreateWithFlags(&t.done, cudaEventDisableTiming) != cudaSuccess) return MGR_ECUDA;
  cudaEventRecord(t.done, B->stream);
  t.n = n;
  *ticket = B->next_ticket++;
  B->tickets[*ticket] = t;
  return MGR_OK;
}

int batch_poll(mgr_ctx* ctx, uint64_t ticket, int64_t timeout_us, int* n_done) {
  if (!ctx || !n_done) return MGR_EINVAL;
  *n_done = 0;
  BatchState* B = static_cast<BatchState*>(ctx->batch);
  if (!B) return MGR_ENOTFOUND;
  cudaEvent_t ev;
  int n;
  {
    std::lock_guard<std::mutex> lk(B->mu);
    auto it = B->tickets.find(ticket);
    if (it == B->tickets.end()) return MGR_ENOTFOUND;
    ev = it->second.done;
    n = it->second.n;
  }
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t q = cudaEventQuery(ev);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) {
      cudaGetLastError();
      return MGR_ECUDA;
    }
    if (timeout_us == 0) return MGR_EPENDING;
    const auto el = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0);
    if (timeout_us > 0 && el.count() >= timeout_us) return MGR_ETIMEDOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  {
    std::lock_guard<std::mutex> lk(B->mu);
    auto it = B->tickets.find(ticket);
    if (it != B->tickets.end()) {
      cudaEventDestroy(it->second.done);
      B->tickets.erase(it);
    }
  }
  *n_done = n;
#ifdef MGR_DEBUG_BOUNDS
  // bounds-checking builds: an out-of-bounds access of the finished batch
  DebugRecord r{};
  if (debug_take(&r)) {
    std::lock_guard<std::mutex> lk(g_dbg_mu);
    g_dbg_last = r;
    g_dbg_have = true;
    return MGR_EDEVICE;
  }
#endif
  return MGR_OK;
}

int batch_tuning(mgr_ctx* ctx, char* buf, size_t len) {
  BatchState* B = ctx ? static_cast<BatchState*>(ctx->batch) : nullptr;
  std::string s;
  if (B) {
    std::lock_guard<std::mutex> lk(B->mu);
    for (auto& kv : B->tune_log) {
      s += "shape[" + std::to_string(kv.first.size()) + " chars]";
      const TileCand c = B->tuned[kv.first];
      char line[128];
      std::snprintf(line, sizeof(line), " chosen tile=%s chunk=%d;%s", cfg_name(c.cfg), c.chunk,
                    B->from_file.count(kv.first) ? " (from the persisted cache)" : "");
      s += line;
      for (auto& m : kv.second) {
        if (m.second >= 0.0)
          std::snprintf(line, sizeof(line), " [%s/%d: %.3f ms]", cfg_name(m.first.cfg), m.first.chunk, m.second);
        else
          std::snprintf(line, sizeof(line), " [%s/%d: failed, %s]", cfg_name(m.first.cfg), m.first.chunk,
                        cudaGetErrorName(cudaError_t(int(-m.second))));
        s += line;
      }
      auto nt = B->tune_note.find(kv.first);
      if (nt != B->tune_note.end()) s += " failed at: " + nt->second;
      s += "\n";
    }
  }
  if (buf && len) {
    std::snprintf(buf, len, "%s", s.c_str());
  }
  return int(s.size());
}


// Read and clear this translation unit's bounds-check record (MGR_DEBUG_BOUNDS).
unsigned long long debug_take_batch(DebugRecord* first) {
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
