// mgr_level.cuh -- the level pass of decomposition (coefficients + load
// vector) and the load-vector pass of recomposition, for sm_103a.
//
// Per level l (level grid n -> coarse grid m), a CTA owns BX x BY coarse
// (y, x) nodes and a chunk of coarse z planes.  It streams the fine z planes
// of its region (the owned fine nodes plus the two-node halo the 5-tap
// mass-transfer stencil needs) in pairs: the coarse-in-z plane p(t) and the
// fine-in-z plane p(t)-1 between p(t-1) and p(t).
//
// Thread mapping (fixed for the CTA's lifetime, so every per-row and
// per-column weight and address is computed once): the CTA's threads form
// row groups of LX lanes (a whole warp, LX = 32, or half of one, LX = 16:
// a tile 14 coarse nodes wide, for fields whose coarse rows are short);
// lane l of a group owns the fine column pair (rx0 + 2l, rx0 + 2l + 1) of
// the region, group w owns RPW fine row pairs.  Below, "lane" and "warp"
// are a thread's lane in its group and its group.  The region starts on a
// coarse node, so the first node of every pair is coarse and the second is
// the fine node between two coarse ones (or, at the end of an axis whose
// length is even, the last coarse node).
//
// Coefficients (Sec. II.A.1), separable and in the paper's FMA form
// (Table "fma"): on a coarse-z plane the x interpolant of a coarse row uses
// the right neighbour's value (warp shuffle), the y interpolant of a fine row
// uses the next coarse row's interpolant (the next pair of the same thread,
// or the next warp's first pair through shared memory); a fine-z plane
// interpolates between the xy interpolants of its two coarse planes, which
// each thread keeps in registers.
//
// Load vector f' = (x_k D_k^-1 K_k) c (Sec. II.A.2, III.A.2): c goes to
// shared memory, the x stencil runs on rows (5 taps; in FP64 2 on rows that
// are coarse in y and z, where c vanishes on coarse nodes), the y stencil on
// the x results, and the z stencil accumulates in registers over the
// streamed planes.  FP32 keeps the two planes interleaved in its tiles
// ({coarse, fine} per node) and runs both planes' stencils as paired FMAs.
// The per-plane-pair constants come from a table the CTA fills once.  Two
// CTA barriers per plane pair.
//
// Coefficient addressing.  Nodal (PK = false): a coefficient sits at its node's
// full-grid position.  Class-packed (PK = true, Sec. I coefficient classes): the
// coefficients of level l form one contiguous class, in row-major order of the
// level grid with the nodes of the coarser grid left out.  With cb(i) = (i+1)/2
// coarse nodes before index i, node (i, j, k) of class l is at
//   i*n1*n2 - cb(i)*m1*m2 + (i fine ? j*n2 + k
//                                   : j*n2 - cb(j)*m2 + (j fine ? k : k - cb(k)))
// from the class start, so plane and row offsets stay separable.
//
// Quantized coefficients (QZ, class-packed only): decomposition writes the
// int32 code round_half_even(c * (1/q_l)) of each coefficient (the rounding
// decision in the stencil type TS) and recomposition reads codes and uses
// code * q_l; q_l is the bin width of the level's class.
#pragma once

template <int NW, int RPW, int LX = 32>
struct LevelTile {
  static_assert(LX == 32 || LX == 16, "row groups of a warp or half a warp");
  static constexpr int NT = NW * 32;
  static constexpr int NG = NT / LX;       // row groups
  static constexpr int BX = LX - 2;        // coarse x outputs per CTA
  static constexpr int BY = NG * RPW - 2;  // coarse y outputs per CTA
  static constexpr int RC = 2 * LX;        // fine column slots (region width <= 2*BX+3 = RC-1)
  static constexpr int RR = 2 * NG * RPW;  // fine row slots (region height <= 2*BY+3 = RR-1)
  static constexpr int CP = RC + 2;        // c row pitch: even, so column pairs stay 8/16-byte aligned
  // x-stencil result row pitch: with half-warp groups the two halves of a warp
  // work 2*RPW rows apart, and a pitch of 4 (mod 8) words puts them in
  // different banks
  static constexpr int GP = LX == 32 ? 32 : LX + 4;
};

// Tile configuration of the level pass per stencil type: 8 warps with two
// row pairs each (two CTAs per SM); FP64 uses a single cp.async stage (the
// FP64 pipe, not memory latency, bounds it, and the smaller footprint keeps
// two CTAs per SM), FP32 two stages.  The MGR_LEVEL_* macros override the
// defaults at build time (tuning sweeps).
#ifndef MGR_LEVEL_F64_NW
#define MGR_LEVEL_F64_NW 8
#endif
#ifndef MGR_LEVEL_F64_RPW
#define MGR_LEVEL_F64_RPW 2
#endif
#ifndef MGR_LEVEL_F64_STAGES
#define MGR_LEVEL_F64_STAGES 1
#endif
#ifndef MGR_LEVEL_F32_NW
#define MGR_LEVEL_F32_NW 8
#endif
#ifndef MGR_LEVEL_F32_RPW
#define MGR_LEVEL_F32_RPW 2
#endif
#ifndef MGR_LEVEL_F32_STAGES
#define MGR_LEVEL_F32_STAGES 2
#endif
template <typename TS>
struct LevelCfg;
template <>
struct LevelCfg<double> {
  static constexpr int NW = MGR_LEVEL_F64_NW, RPW = MGR_LEVEL_F64_RPW, STAGES = MGR_LEVEL_F64_STAGES;
};
template <>
struct LevelCfg<float> {
  static constexpr int NW = MGR_LEVEL_F32_NW, RPW = MGR_LEVEL_F32_RPW, STAGES = MGR_LEVEL_F32_STAGES;
};

// Tile configuration per pass: the recomposition load pass (MODE 1) computes
// no coefficients and keeps fewer values per row pair in registers, so in FP32
// it also fits three row pairs per warp (a taller tile, less repeated halo
// work) within the same 128 registers; MGR_LEVEL_F32_REC_RPW selects it at
// build time (measured: faster at 1000x700x300, slower at 513^3; default two).
#ifndef MGR_LEVEL_F32_REC_RPW
#define MGR_LEVEL_F32_REC_RPW 2
#endif
template <typename TS, int MODE>
struct LevelCfgM {
  static constexpr int NW = LevelCfg<TS>::NW, STAGES = LevelCfg<TS>::STAGES;
  static constexpr int RPW = (MODE == 1 && sizeof(TS) == 4) ? MGR_LEVEL_F32_REC_RPW : LevelCfg<TS>::RPW;
};

// CTAs per SM a level-pass or interpolation CTA of NW warps is compiled for:
// 16 warps per SM in every configuration, so each thread may use up to 128
// registers.
#ifndef MGR_LEVEL_CTAS_16W
#define MGR_LEVEL_CTAS_16W 1
#endif
constexpr int level_ctas_per_sm(int nw) { return nw >= 16 ? MGR_LEVEL_CTAS_16W : 16 / nw; }
template <typename T>
struct Pair;
template <>
struct Pair<float> {
  using type = float2;
};
template <>
struct Pair<double> {
  using type = double2;
};
template <>
struct Pair<int> {
  using type = int2;
};

// int32 code of value v for 1/bin width qinv: v * qinv rounded to FP32 / FP64
// (no contraction), then rounded half to even; values whose code does not fit
// in (-2^31, 2^31) (and NaN) become +-(2^31-1) and are counted.
__device__ __forceinline__ int quant_code(float v, float qinv, unsigned long long* sat) {
  const float t = __fmul_rn(v, qinv);
  const float r = rintf(t);
  if (!(fabsf(r) < 2147483648.0f)) {
    if (sat) atomicAdd(sat, 1ull);
    return t > 0.0f ? 2147483647 : -2147483647;
  }
  return int(r);
}
// FP64: the product is the only FP64 operation; t is rounded to an integer
// from its IEEE-754 fields with integer instructions (the FP64 pipe, which
// bounds the FP64 level pass, has a small fraction of the integer pipes'
// throughput).  With t = 1.m * 2^e and the 53-bit significand M = 1m,
// |t| < 0.5 for e < -1; otherwise floor|t| = M >> (52 - e) and the
// remainder decides round-half-to-even.
__device__ __forceinline__ int quant_code(double v, double qinv, unsigned long long* sat) {
  const double t = __dmul_rn(v, qinv);
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(t));
  const int e = int((b >> 52) & 0x7ffu) - 1023;
  if (e < -1) return 0;
  const bool neg = (b >> 63) != 0;
  if (e <= 30) {
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = 52 - e;  // 22 .. 53
    unsigned long long q = m >> sh;
    const unsigned long long rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
    if (q < (1ull << 31)) return neg ? -int(q) : int(q);
  }
  if (sat) atomicAdd(sat, 1ull);
  const bool nan = e == 1024 && (b & 0xFFFFFFFFFFFFFull) != 0;
  return (!neg && !nan) ? 2147483647 : -2147483647;
}

// Code k as a value of the stencil type.  FP64 assembles the IEEE-754 fields
// of the (exactly representable) integer with integer instructions: sign,
// exponent 1023 + msb(|k|), and |k| shifted up to the 52-bit fraction.
template <typename TS>
__device__ __forceinline__ TS code_value(int k);
template <>
__device__ __forceinline__ float code_value<float>(int k) {
  return float(k);
}
template <>
__device__ __forceinline__ double code_value<double>(int k) {
  const unsigned s = unsigned(k) & 0x80000000u;
  const unsigned a = k < 0 ? 0u - unsigned(k) : unsigned(k);
  const int e = 31 - __clz(a | 1u);
  const unsigned long long m = (static_cast<unsigned long long>(a) << (52 - e)) & 0xFFFFFFFFFFFFFull;
  const unsigned long long bits =
      (static_cast<unsigned long long>(s) << 32) | (static_cast<unsigned long long>(1023 + e) << 52) | m;
  return k == 0 ? 0.0 : __longlong_as_double(static_cast<long long>(bits));
}
// Dequantized value k * q.
template <typename TS>
__device__ __forceinline__ TS dequant(int k, TS q) {
  return code_value<TS>(k) * q;
}

template <typename TS, typename TW>
struct LevelArgs {
  const void* in;  // DEC: level-l values; REC: nodal coefficients (full grid)
  int64_t in_sz, in_sy;
  int in_full;     // 1: `in` is addressed through the full-grid map min(i*s, N-1)
  void* y;         // DEC: nodal output (full grid)
  int64_t y_sz, y_sy;
  TW* w;           // DEC: coarse nodal values (compact m grid)
  TW* f;           // load vector (compact m grid)
  int64_t c_sz, c_sy;
  int n[3], m[3];
  int64_t s[3], N[3];
  const TS* wa[3];
  const TS* wb[3];
  const TS* k[3];
  int qz_chunk;
  int bz0;         // first z chunk of this launch (a launch may cover a subset of the chunks)
  int write_y;
  double qs;                // QZ: 1/bin width (MODE 0) or bin width (MODE 1)
  unsigned long long* qsat; // QZ, MODE 0: saturated-code counter (may be null)
  int all_fine;             // MODE 1: every node holds a coefficient (a time slice of a
                            // 4D field that is fine in time), not only the fine ones
};

// FP64 keeps the x / y stencil weights in shared memory (the FP64 pass is
// bound by the FP64 pipe and short of registers), FP32 in registers (its
// pass is bound by instruction issue).
template <typename TS>
constexpr bool weights_in_smem() {
  return sizeof(TS) == 8;
}

// Plane pairs a level-pass CTA streams at most (its z chunk plus the halo
// planes before it): the per-plane-pair constants are tabulated once per CTA
// in shared memory, so the hosts cap the chunk length at kLevelMaxChunk.
constexpr int kLevelPlanes = 64;
constexpr int kLevelMaxChunk = kLevelPlanes - 2;

// Byte offset of the plane table in the level pass's shared memory (after the
// stage buffers, coefficient tiles, x-stencil results and weights).
template <int NW, int RPW, int STAGES, typename TI, typename TS, int LX = 32>
constexpr size_t level_table_offset() {
  using G = LevelTile<NW, RPW, LX>;
  return (sizeof(TI) * STAGES * 2 * G::RR * G::RC +
          sizeof(TS) * (2 * G::RR * G::CP + 2 * G::RR * G::GP + 5 * LX + 5 * G::NG * RPW +
                        (sizeof(TS) == 8 ? G::NG * G::RC : 0)) +
          15) / 16 * 16;
}
// per plane pair: four plane offsets (int64), eight weights (TS), a flag (int)
template <typename TS>
constexpr size_t level_table_bytes() {
  return kLevelPlanes * (4 * sizeof(int64_t) + 8 * sizeof(TS) + sizeof(int));
}
template <int NW, int RPW, int STAGES, typename TI, typename TS, int LX = 32>
constexpr size_t level_smem_bytes() {
  return level_table_offset<NW, RPW, STAGES, TI, TS, LX>() + level_table_bytes<TS>();
}

// Copy the element pair (c0, c0+1) of one row into shared memory: one
// 2-element cp.async when both are in the region, adjacent in memory and
// aligned (uniform across a warp: every lane of a row has the same parity),
// else one copy per element.
template <typename T>
__device__ __forceinline__ void load_pair(T* dst, const T* src0, const T* src1, bool v0, bool v1, bool contig) {
  if (v0 && v1 && contig && ((reinterpret_cast<uintptr_t>(src0) & (2 * sizeof(T) - 1)) == 0)) {
    cp_async(dst, src0, int(2 * sizeof(T)));
  } else {
    if (v0) cp_async(dst, src0, int(sizeof(T)));
    if (v1) cp_async(dst + 1, src1, int(sizeof(T)));
  }
}

// Store a pair of output values (to adjacent or separate addresses).  4-byte
// values are always stored one by one: the warp's stores still coalesce, and
// the FP32 level pass, bound by instruction issue, saves the alignment test
// and its branch (measured 7% faster at 513^3).
template <typename T>
__device__ __forceinline__ void store_pair(T* p0, T* p1, T a0, T a1, bool w0, bool w1, bool contig) {
  if constexpr (sizeof(T) == 4) {
    if (w0) *p0 = a0;
    if (w1) *p1 = a1;
    return;
  }
  if (w0 && w1 && contig && ((reinterpret_cast<uintptr_t>(p0) & (2 * sizeof(T) - 1)) == 0)) {
    typename Pair<T>::type v;
    v.x = a0;
    v.y = a1;
    *reinterpret_cast<typename Pair<T>::type*>(p0) = v;
  } else {
    if (w0) *p0 = a0;
    if (w1) *p1 = a1;
  }
}

// One CTA's work: coarse tile (bx, by) and z chunk bz of level args `a`,
// with `smem_raw` the CTA's dynamic shared memory (level_smem_bytes).
// PK: coefficients in the class-packed layout (MODE 0 writes `y`, MODE 1 reads
// `in` as the class of this level; y_sz / in_sz = n1*n2, y_sy / in_sy = n2).
// QZ (with PK): those coefficients are int32 codes (TD = int in MODE 0, TI =
// int in MODE 1).
// AF: honour `all_fine` (the 4D form's time slices; a runtime flag read once).
// LX: lanes per row group (32 or 16).
template <int MODE, int NW, int RPW, int STAGES, typename TI, typename TD, typename TS, typename TW, bool PK = false,
          bool QZ = false, bool AF = false, int LX = 32>
__device__ __forceinline__ void level_body(const LevelArgs<TS, TW>& a, int bx, int by, int bz,
                                           unsigned char* smem_raw) {
  using G = LevelTile<NW, RPW, LX>;
  using TS2 = typename Pair<TS>::type;
  using TI2 = typename Pair<TI>::type;
  constexpr int RR = G::RR, RC = G::RC, CP = G::CP, GP = G::GP, NG = G::NG;
  constexpr unsigned FULL = 0xffffffffu;
  TI* stage = reinterpret_cast<TI*>(smem_raw);                                       // [STAGES][2][RR][RC]
  TS* cbuf = reinterpret_cast<TS*>(smem_raw + sizeof(TI) * STAGES * 2 * RR * RC);  // [2][RR][CP]
  TS* gxb = cbuf + 2 * RR * CP;                                                     // [2][RR][GP]
  TS* kxs = gxb + 2 * RR * GP;                                                      // [5][LX]
  TS* kys = kxs + 5 * LX;                                                           // [5][NG*RPW]
  TS* xch = kys + 5 * NG * RPW;  // [NG][RC] FP64 only: x interpolants of each group's first coarse row
  // plane table (kLevelPlanes entries): offsets of the input's coarse and fine
  // planes and of the output's; weights wzc[3], wzf[2], za, zb; has-fine flag
  int64_t* ptab = reinterpret_cast<int64_t*>(smem_raw + level_table_offset<NW, RPW, STAGES, TI, TS, LX>());
  TS* pwt = reinterpret_cast<TS*>(ptab + 4 * kLevelPlanes);
  int* pfl = reinterpret_cast<int*>(pwt + 8 * kLevelPlanes);

  const int lane = threadIdx.x % LX, warp = threadIdx.x / LX;  // lane in the row group, row group
  const int nz = a.n[0], ny = a.n[1], nx = a.n[2];
  const int mz = a.m[0], my = a.m[1], mx = a.m[2];
  const int qx0 = bx * G::BX, qx1 = min(qx0 + G::BX, mx);
  const int qy0 = by * G::BY, qy1 = min(qy0 + G::BY, my);
  const int qz0 = bz * a.qz_chunk, qz1 = min(qz0 + a.qz_chunk, mz);
  const int rx0 = max(region_start(qx0, nx), 0), rx1 = min(pidx(qx1 - 1, nx) + 2, nx - 1);
  const int ry0 = max(region_start(qy0, ny), 0), ry1 = min(pidx(qy1 - 1, ny) + 2, ny - 1);
  const int ox0 = pidx(qx0, nx), ox1 = (qx1 == mx) ? nx : pidx(qx1, nx);
  const int oy0 = pidx(qy0, ny), oy1 = (qy1 == my) ? ny : pidx(qy1, ny);
  int t_start = qz0 > 0 ? qz0 - 1 : 0;
  if (qz0 >= 2 && pidx(qz0, nz) - pidx(qz0 - 1, nz) == 1) t_start = qz0 - 2;
  const int t_end = min(qz1, mz - 1);

  const TI* __restrict__ in = static_cast<const TI*>(a.in);
  TD* __restrict__ yout = static_cast<TD*>(a.y);
  const bool wy = (MODE == 0) && a.write_y;
  // bounds-checking builds: extents (elements) of the buffers this CTA
  // addresses; the LVL_* statements below check against them (other builds
  // run the plain statements)
#ifdef MGR_DEBUG_BOUNDS
  const long long n_in = (PK && MODE == 1) ? (long long)nz * a.in_sz - (long long)mz * a.c_sz
                                           : (long long)(a.in_full ? a.N[0] : nz) * a.in_sz;
  const long long n_y = PK ? (long long)nz * a.y_sz - (long long)mz * a.c_sz : (long long)a.N[0] * a.y_sz;
  const long long n_c = (long long)mz * a.c_sz;
  constexpr long long n_stage = (long long)STAGES * 2 * RR * RC;
#endif
#define LVL_CP(dst, src) \
  MGR_GUARD(MGR_PIN(src, in, n_in, kDbgLevelIn) && MGR_PIN(dst, stage, n_stage, kDbgLevelStage), \
            cp_async(dst, src, int(sizeof(TI))))
#define LVL_CPZ(dst, src, valid) \
  MGR_GUARD(MGR_PIN(src, in, n_in, kDbgLevelIn) && MGR_PIN(dst, stage, n_stage, kDbgLevelStage), \
            cp_async_zf(dst, src, int(sizeof(TI)), valid))
#define LVL_Y(q, v) MGR_GUARD(MGR_PIN(q, yout, n_y, kDbgLevelY), *(q) = (v))
#define LVL_YP(p0, p1, a0, a1, w0, w1, contig)                                                                  \
  MGR_GUARD((!(w0) || MGR_PIN(p0, yout, n_y, kDbgLevelY)) && (!(w1) || MGR_PIN(p1, yout, n_y, kDbgLevelY)), \
            store_pair<TD>(p0, p1, a0, a1, w0, w1, contig))
#define LVL_W(wz, i, v) MGR_GUARD(MGR_IN((wz) - a.w + (i), n_c, kDbgLevelW), (wz)[i] = (v))
#define LVL_F(i, v) MGR_GUARD(MGR_IN(i, n_c, kDbgLevelF), a.f[i] = (v))
  const bool afine = AF && MODE == 1 && a.all_fine;
  const TS qs = QZ ? TS(a.qs) : TS(1);
  // value written for coefficient v when `st` (the node is stored: values of
  // nodes that are not stored are never quantized, so never counted as
  // saturated) (MODE 0); value of a read coefficient (MODE 1)
  auto yval = [&](TS v, bool st) -> TD {
    if constexpr (QZ) return st ? TD(quant_code(v, qs, a.qsat)) : TD(0);
    else return TD(v);
  };
  // (MODE 1 with QZ: the code itself; the bin width scales the load vector
  // once per coarse node instead, see fout)
  auto cval = [&](TI v) -> TS {
    if constexpr (QZ && MODE == 1) return code_value<TS>(int(v));
    else return TS(v);
  };
  auto fout = [&](TS acc) -> TW {
    if constexpr (QZ && MODE == 1) return TW(acc) * TW(a.qs);
    else return TW(acc);
  };

  // ---- per-lane column constants (in-plane offsets fit in 32 bits)
  const int cx0 = 2 * lane;
  const int gx0 = rx0 + cx0, gx1 = gx0 + 1;
  const bool vx0 = gx0 <= rx1, vx1 = gx1 <= rx1;
  const bool fx1 = vx1 && gx1 < nx - 1;  // gx1 is odd: fine unless it is the last node
  const TS wax1 = fx1 ? a.wa[2][gx1] : TS(0), wbx1 = fx1 ? a.wb[2][gx1] : TS(0);
  const bool owx0 = vx0 && gx0 >= ox0 && gx0 < ox1, owx1 = vx1 && gx1 >= ox0 && gx1 < ox1;
  // input columns, clamped into the grid (slots past its end load zeros from a valid address)
  const int ic0 = a.in_full ? int(fmap(min(gx0, nx - 1), a.s[2], a.N[2])) : min(gx0, nx - 1);
  const int ic1 = a.in_full ? int(fmap(min(gx1, nx - 1), a.s[2], a.N[2])) : min(gx1, nx - 1);
  const int yc0 = PK ? gx0 : int(fmap(min(gx0, nx - 1), a.s[2], a.N[2]));
  const int yc1 = PK ? gx1 : int(fmap(min(gx1, nx - 1), a.s[2], a.N[2]));
  const bool ycontig = yc1 == yc0 + 1;
  const int pcx1 = gx1 - cidx(gx1);  // packed column of gx1 in a row coarse in y and z

  // ---- x stencil of this lane's output column
  const int nbx = qx1 - qx0;
  const bool kxo = lane < nbx;
  const int qxo = min(qx0 + lane, mx - 1);
  const int px = pidx(qxo, nx);
  const int dx = px - rx0;  // slot of the stencil centre
  TS kxr[weights_in_smem<TS>() ? 1 : 5];
  unsigned kxm = 0;  // taps inside the grid
#pragma unroll
  for (int o = 0; o < 5; ++o) {
    const TS kw = a.k[2][5 * qxo + o];
    if constexpr (weights_in_smem<TS>()) {
      if (warp == 0) kxs[o * LX + lane] = kw;
    } else {
      kxr[o] = kw;
    }
    const int j = px + o - 2;
    if (j >= 0 && j < nx) kxm |= 1u << o;
  }
  auto kx = [&](int o) -> TS {
    if constexpr (weights_in_smem<TS>()) return kxs[o * LX + lane];
    else return kxr[o];
  };
  // interior column: taps px +- 1 fine, px and px +- 2 coarse, even slot
  const bool kx_generic = kxm == 31u && (px & 1) == 0 && px + 1 < nx - 1;
  // FP32 (BF): the x / y stencils run without per-row branches, always five
  // taps (weight 0 outside the grid) over tiles whose slots outside the region
  // hold zeros, so their 8 independent FMA chains per thread interleave (the
  // FP32 pass is latency-bound); FP64, bound by its FP64 pipe, keeps the
  // reduced tap counts of rows whose coefficients vanish.
  constexpr bool BF = sizeof(TS) == 4;
  // FP32 nodal decomposition (RS): the coefficients go out after the
  // coefficient phase, row by row from the shared tile, each lane storing
  // output columns ox0 + lane and ox0 + LX + lane (consecutive lanes,
  // consecutive addresses): the coefficient phase then keeps no output
  // addresses or values live (it is short of registers).  All-coarse nodes
  // get 0 there, a placeholder a coarser level overwrites.
  constexpr bool RS = BF && !PK && MODE == 0;
  const int oc0 = ox0 + lane, oc1 = oc0 + LX;
  const bool rs0 = oc0 < ox1, rs1 = oc1 < ox1;
  const int ro0 = int(fmap(min(oc0, nx - 1), a.s[2], a.N[2])), ro1 = int(fmap(min(oc1, nx - 1), a.s[2], a.N[2]));
  const int rsl0 = oc0 - rx0, rsl1 = oc1 - rx0;

  // ---- per-row constants (RPW row pairs per warp)
  int gy0[RPW];
  bool vy0[RPW], vy1[RPW], fy1[RPW], owy0[RPW], owy1[RPW];
  TS way1[RPW], wby1[RPW];
  int ir0[RPW], ir1[RPW], yr0[RPW], yr1[RPW];
  // y stencil of this thread's output rows
  const int nby = qy1 - qy0;
  TS kyr[RPW][weights_in_smem<TS>() ? 1 : 5];
  unsigned kym[RPW];
  int dyo[RPW];
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    gy0[k] = ry0 + 2 * (warp * RPW + k);
    const int g1 = gy0[k] + 1;
    vy0[k] = gy0[k] <= ry1;
    vy1[k] = g1 <= ry1;
    fy1[k] = vy1[k] && g1 < ny - 1;
    way1[k] = fy1[k] ? a.wa[1][g1] : TS(0);
    wby1[k] = fy1[k] ? a.wb[1][g1] : TS(0);
    owy0[k] = vy0[k] && gy0[k] >= oy0 && gy0[k] < oy1;
    owy1[k] = vy1[k] && g1 >= oy0 && g1 < oy1;
    const int c0 = min(gy0[k], ny - 1), c1 = min(g1, ny - 1);
    ir0[k] = int(a.in_full ? fmap(c0, a.s[1], a.N[1]) * a.in_sy : int64_t(c0) * a.in_sy);
    ir1[k] = int(a.in_full ? fmap(c1, a.s[1], a.N[1]) * a.in_sy : int64_t(c1) * a.in_sy);
    yr0[k] = PK ? c0 * nx : int(fmap(c0, a.s[1], a.N[1]) * a.y_sy);
    yr1[k] = PK ? c1 * nx : int(fmap(c1, a.s[1], a.N[1]) * a.y_sy);
    const int qy = min(qy0 + warp * RPW + k, my - 1);
    const int py = pidx(qy, ny);
    dyo[k] = py - ry0;
    kym[k] = 0;
#pragma unroll
    for (int o = 0; o < 5; ++o) {
      const TS kw = a.k[1][5 * qy + o];
      if constexpr (weights_in_smem<TS>()) {
        if (lane == 0) kys[o * (NG * RPW) + warp * RPW + k] = kw;
      } else {
        kyr[k][o] = kw;
      }
      const int jj = py + o - 2;
      if (jj >= 0 && jj < ny) kym[k] |= 1u << o;
    }
    // rows past the tile's outputs (the last warp's, in all but the last tile
    // row) are never stored: not interior, so no stencil form reads past the tile
    if (warp * RPW + k >= nby) kym[k] = 0;
  }
  auto ky = [&](int k, int o) -> TS {
    if constexpr (weights_in_smem<TS>()) return kys[o * (NG * RPW) + warp * RPW + k];
    else return kyr[k][o];
  };
#ifdef MGR_DEBUG_BOUNDS
  // the shared-tile indices below are a per-thread constant plus the loop's
  // row and tap offsets: checking the constants' ranges once covers them all
  (void)MGR_IN(2 * (warp * RPW + RPW - 1) + 1, RR, kDbgLevelTile);  // stage / tile rows
  (void)MGR_IN(cx0 + 1, RC, kDbgLevelTile);                           // stage / tile columns
  if (kxo && kx_generic) {
    (void)MGR_IN(dx - 2, RC, kDbgLevelTile);  // five x taps
    (void)MGR_IN(dx + 2, RC, kDbgLevelTile);
  }
#pragma unroll
  for (int k = 0; k < RPW; ++k)
    if (kym[k] == 31u && kxo) {
      (void)MGR_IN(dyo[k] - 2, RR, kDbgLevelTile);  // five y taps
      (void)MGR_IN(dyo[k] + 2, RR, kDbgLevelTile);
    }
#endif
  auto iplane = [&](int g) -> int64_t {
    if (PK && MODE == 1) return int64_t(g) * a.in_sz - int64_t(cidx(g)) * a.c_sz;
    return a.in_full ? fmap(g, a.s[0], a.N[0]) * a.in_sz : int64_t(g) * a.in_sz;
  };
  auto yplane = [&](int g) -> int64_t {
    return PK ? int64_t(g) * a.y_sz - int64_t(cidx(g)) * a.c_sz : fmap(g, a.s[0], a.N[0]) * a.y_sz;
  };
  // ---- plane table, computed once by the CTA (every warp would otherwise
  // recompute these on each plane pair): plane pair t -- the coarse plane p(t)
  // and, when a fine plane lies between p(t-1) and p(t), that fine plane -- is
  // entry t - t_start
  (void)MGR_IN(t_end - t_start, kLevelPlanes, kDbgLevelTile);
  for (int e = threadIdx.x; e <= t_end - t_start && e < kLevelPlanes; e += G::NT) {
    const int t = t_start + e;
    const int Pc = pidx(t, nz), Pf = Pc - 1;
    const bool hf = t > t_start && Pc - pidx(t - 1, nz) == 2;
    ptab[4 * e + 0] = iplane(Pc);
    ptab[4 * e + 1] = hf ? iplane(Pf) : 0;
    ptab[4 * e + 2] = yplane(Pc);
    ptab[4 * e + 3] = yplane(max(Pf, 0));
    // z stencil weights of both planes for the coarse planes t-1, t, t+1
    TS* w = pwt + 8 * e;
#pragma unroll
    for (int dq = -1; dq <= 1; ++dq) {
      const int q = t + dq;
      const bool qv = q >= 0 && q < mz;
      const int pq = qv ? pidx(q, nz) : 0;
      const int oc = Pc - pq;
      w[dq + 1] = (qv && oc >= -2 && oc <= 2) ? a.k[0][5 * q + oc + 2] : TS(0);
      if (dq < 1) {
        const int of = Pf - pq;
        w[dq + 4] = (hf && qv && of >= -2 && of <= 2) ? a.k[0][5 * q + of + 2] : TS(0);
      }
    }
    // z interpolation weights of the fine plane (decomposition)
    w[6] = (MODE == 0 && hf) ? a.wa[0][Pf] : TS(0);
    w[7] = (MODE == 0 && hf) ? a.wb[0][Pf] : TS(0);
    pfl[e] = hf ? 1 : 0;
  }
  __syncthreads();  // stencil weights and plane table staged
  // poff: the plane's offset (plane table); zc: it is a coarse plane (a packed
  // class then holds only its fine nodes)
  auto load_plane = [&](TI* sb, int64_t poff, bool zc) {
    const TI* base = in + poff;
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
      TI* d0 = sb + 2 * (warp * RPW + k) * RC + cx0;
      if (PK && MODE == 1 && zc) {
        // rows of a coarse plane: the coarse row gy0 holds its fine columns only
        const int r0 = ir0[k] - cidx(gy0[k]) * mx, r1 = ir1[k] - cidx(gy0[k] + 1) * mx;
        if (vy0[k] && fx1) LVL_CP(d0 + 1, base + r0 + pcx1);
        if (vy1[k]) {
          if (fy1[k]) {
            if (vx0) LVL_CP(d0 + RC, base + r1 + ic0);
            if (vx1) LVL_CP(d0 + RC + 1, base + r1 + ic1);
          } else if (fx1) {
            LVL_CP(d0 + RC + 1, base + r1 + pcx1);
          }
        }
        continue;
      }
      if constexpr (MODE == 1) {
        // branch-free: every slot is copied, slots outside the region as zeros
        // (their addresses are clamped into the grid, so they are valid)
        LVL_CPZ(d0, base + ir0[k] + ic0, vy0[k] && vx0);
        LVL_CPZ(d0 + 1, base + ir0[k] + ic1, vy0[k] && vx1);
        LVL_CPZ(d0 + RC, base + ir1[k] + ic0, vy1[k] && vx0);
        LVL_CPZ(d0 + RC + 1, base + ir1[k] + ic1, vy1[k] && vx1);
      } else {
        // (the decomposition pass is short of registers: copying only the slots
        // inside the region keeps its per-slot predicates out of the loop)
        if (vy0[k]) {
          if (vx0) LVL_CP(d0, base + ir0[k] + ic0);
          if (vx1) LVL_CP(d0 + 1, base + ir0[k] + ic1);
        }
        if (vy1[k]) {
          if (vx0) LVL_CP(d0 + RC, base + ir1[k] + ic0);
          if (vx1) LVL_CP(d0 + RC + 1, base + ir1[k] + ic1);
        }
      }
    }
  };
  static_assert(STAGES == 1 || STAGES == 2, "one or two stage buffers");
  // stage buffer of plane pair t (two in rotation, or one)
  auto stage_of = [&](int t) { return stage + ((STAGES == 2) ? ((t - t_start) & 1) * 2 * RR * RC : 0); };
  auto issue = [&](int t) {
    TI* sb = stage_of(t);
    const int e = t - t_start;
    const longlong2 off = *reinterpret_cast<const longlong2*>(ptab + 4 * e);
    load_plane(sb, off.x, true);
    if (pfl[e]) load_plane(sb + RR * RC, off.y, false);
    cp_commit();
  };

  TS Ip[RPW][4], In[RPW][4];
  TS acc0[RPW], acc1[RPW], acc2[RPW];
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    acc0[k] = acc1[k] = acc2[k] = TS(0);
#pragma unroll
    for (int e = 0; e < 4; ++e) Ip[k][e] = In[k][e] = TS(0);
  }

  // two stages: the next plane pair is in flight while this one is processed;
  // one stage: the next is issued once every thread is done with the stage
  issue(t_start);
  for (int t = t_start; t <= t_end; ++t) {
    if (STAGES == 2) {
      if (t < t_end) {
        issue(t + 1);  // into the buffer plane pair t-1 used
        cp_wait<1>();
      } else {
        cp_wait<0>();
      }
    } else {
      cp_wait<0>();
    }
    // Every thread copies, and later reads, only its own slots of the stage
    // buffer; the one exception is FP32's read of the next warp's first row
    // (nxt0 / nxt1 below), which needs the CTA barrier.
    if constexpr (BF) __syncthreads();
    else __syncwarp();
    const TI* sc = stage_of(t);
    const TI* sf = sc + RR * RC;
    const int te = t - t_start;
    const bool hf = pfl[te] != 0;
    const bool own_c = (t >= qz0) && (t < qz1);
    const bool own_f = hf && (t > qz0) && (t <= qz1);

    // ---- this thread's values of both planes (pairs from shared memory)
    TS vc[RPW][4];
    TI rc[RPW][4];  // raw coarse-plane values: exact copies for the coarse workspace
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
      const int r0 = 2 * (warp * RPW + k);
      const TI2 p0 = *reinterpret_cast<const TI2*>(sc + r0 * RC + cx0);
      const TI2 p1 = *reinterpret_cast<const TI2*>(sc + (r0 + 1) * RC + cx0);
      rc[k][0] = p0.x;
      rc[k][1] = p0.y;
      rc[k][2] = p1.x;
      rc[k][3] = p1.y;
#pragma unroll
      for (int e = 0; e < 4; ++e) vc[k][e] = cval(rc[k][e]);
    }
    // ---- coarse-z plane: x interpolants of the coarse rows
    TS v12[RPW];
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
      const TS v02 = __shfl_down_sync(FULL, vc[k][0], 1, LX);
      v12[k] = __shfl_down_sync(FULL, vc[k][2], 1, LX);
      if (MODE == 0) {
        In[k][0] = vc[k][0];
        In[k][1] = fx1 ? wax1 * vc[k][0] + wbx1 * v02 : vc[k][1];
      }
    }
    // the x interpolant of the coarse row below this warp's last pair (the next
    // warp's first row), for the y interpolation of this warp's last fine row.
    // FP32: computed here from the staged tile (the same operations as the next
    // warp's), so no exchange and no barrier is needed; FP64, bound by its FP64
    // pipe, takes it from the next warp through shared memory instead.
    TS nxt0 = TS(0), nxt1 = TS(0);
    if constexpr (!BF) {
      if (MODE == 0) *reinterpret_cast<TS2*>(xch + warp * RC + cx0) = TS2{In[0][0], In[0][1]};
      __syncthreads();
    } else if (MODE == 0 && (LX < 32 || warp + 1 < NG)) {
      // (half-warp groups: both halves of a warp take this branch, so that the
      // shuffle below runs on every lane; the last group's result is unused)
      const int wn = LX < 32 ? min(warp + 1, NG - 1) : warp + 1;
      const TI2 pn = *reinterpret_cast<const TI2*>(sc + 2 * wn * RPW * RC + cx0);
      const TS vn0 = cval(pn.x), vn1 = cval(pn.y);
      const TS vn2 = __shfl_down_sync(FULL, vn0, 1, LX);
      nxt0 = vn0;
      nxt1 = fx1 ? wax1 * vn0 + wbx1 * vn2 : vn1;
    }

    // ---- coefficients of both planes -> shared memory and the nodal output
    TS* cc = cbuf;
    TS* cf = cbuf + RR * CP;
    const longlong2 yoff = *reinterpret_cast<const longlong2*>(ptab + 4 * te + 2);
    TD* yzc = yout + yoff.x;
    TD* yzf = yout + yoff.y;
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
      const int r0 = 2 * (warp * RPW + k);
      TS c[4];
      if (MODE == 0) {
        TS n0, n1;
        if (k + 1 < RPW) {
          n0 = In[k + 1 < RPW ? k + 1 : k][0];
          n1 = In[k + 1 < RPW ? k + 1 : k][1];
        } else if (warp + 1 < NG) {
          if constexpr (BF) {
            n0 = nxt0;
            n1 = nxt1;
          } else {
            const TS2 nx2 = *reinterpret_cast<const TS2*>(xch + (warp + 1) * RC + cx0);
            n0 = nx2.x;
            n1 = nx2.y;
          }
        } else {
          n0 = n1 = TS(0);
        }
        if (fy1[k]) {
          In[k][2] = way1[k] * In[k][0] + wby1[k] * n0;
          In[k][3] = way1[k] * In[k][1] + wby1[k] * n1;
        } else {
          In[k][2] = vc[k][2];
          In[k][3] = fx1 ? wax1 * vc[k][2] + wbx1 * v12[k] : vc[k][3];
        }
        c[0] = TS(0);
        c[1] = vc[k][1] - In[k][1];
        c[2] = vc[k][2] - In[k][2];
        c[3] = vc[k][3] - In[k][3];
      } else if (afine) {
        c[0] = (vx0 && vy0[k]) ? vc[k][0] : TS(0);
        c[1] = (vx1 && vy0[k]) ? vc[k][1] : TS(0);
        c[2] = (vx0 && vy1[k]) ? vc[k][2] : TS(0);
        c[3] = (vx1 && vy1[k]) ? vc[k][3] : TS(0);
      } else {
        c[0] = TS(0);
        c[1] = fx1 ? vc[k][1] : TS(0);
        c[2] = fy1[k] ? vc[k][2] : TS(0);
        c[3] = (fx1 || fy1[k]) ? vc[k][3] : TS(0);
      }
      if constexpr (BF && (PK || MODE == 0)) {
        // slots outside the region hold zeros, not values of unloaded slots (the
        // nodal recomposition loads zero-fill them; the other loads skip them)
        c[0] = (vx0 && vy0[k]) ? c[0] : TS(0);
        c[1] = (vx1 && vy0[k]) ? c[1] : TS(0);
        c[2] = (vx0 && vy1[k]) ? c[2] : TS(0);
        c[3] = (vx1 && vy1[k]) ? c[3] : TS(0);
      }
      if constexpr (!BF) {
        *reinterpret_cast<TS2*>(cc + r0 * CP + cx0) = TS2{c[0], c[1]};
        *reinterpret_cast<TS2*>(cc + (r0 + 1) * CP + cx0) = TS2{c[2], c[3]};
      }
      TS dd[4] = {TS(0), TS(0), TS(0), TS(0)};  // fine-plane coefficients (zeros without a fine plane)
      if (PK && wy && own_c) {
        // packed class: the coarse row gy0 keeps only its fine column gx1
        const int r0 = yr0[k] - cidx(gy0[k]) * mx, r1 = yr1[k] - cidx(gy0[k] + 1) * mx;
        if (owy0[k] && owx1 && fx1) LVL_Y(yzc + r0 + pcx1, yval(c[1], true));
        if (owy1[k]) {
          if (fy1[k]) {
            LVL_YP(yzc + r1 + yc0, yzc + r1 + yc1, yval(c[2], owx0), yval(c[3], owx1), owx0, owx1, true);
          } else if (owx1 && fx1) {
            LVL_Y(yzc + r1 + pcx1, yval(c[3], true));
          }
        }
      } else if (!RS && wy && own_c) {
        // all-coarse nodes get their (uncorrected) value as a placeholder that a
        // coarser level overwrites; it keeps the row's sectors fully written
        LVL_YP(yzc + yr0[k] + yc0, yzc + yr0[k] + yc1, TD(vc[k][0]), TD(fx1 ? c[1] : vc[k][1]),
                       owy0[k] && owx0, owy0[k] && owx1, ycontig);
        LVL_YP(yzc + yr1[k] + yc0, yzc + yr1[k] + yc1, TD(fy1[k] ? c[2] : vc[k][2]),
                       TD((fx1 || fy1[k]) ? c[3] : vc[k][3]), owy1[k] && owx0, owy1[k] && owx1, ycontig);
      }
      if (MODE == 0 && own_c) {
        // coarse nodal values of the owned all-coarse nodes
        TW* wz = a.w + int64_t(t) * a.c_sz;
        if (owy0[k] && owx0) LVL_W(wz, int64_t(cidx(gy0[k])) * a.c_sy + cidx(gx0), TW(rc[k][0]));
        if (owy0[k] && owx1 && !fx1) LVL_W(wz, int64_t(cidx(gy0[k])) * a.c_sy + cidx(gx1), TW(rc[k][1]));
        if (owy1[k] && !fy1[k]) {
          if (owx0) LVL_W(wz, int64_t(cidx(gy0[k] + 1)) * a.c_sy + cidx(gx0), TW(rc[k][2]));
          if (owx1 && !fx1) LVL_W(wz, int64_t(cidx(gy0[k] + 1)) * a.c_sy + cidx(gx1), TW(rc[k][3]));
        }
      }
      if (hf) {
        TS vf[4];
        {
          const TI2 f0 = *reinterpret_cast<const TI2*>(sf + r0 * RC + cx0);
          const TI2 f1 = *reinterpret_cast<const TI2*>(sf + (r0 + 1) * RC + cx0);
          vf[0] = cval(f0.x);
          vf[1] = cval(f0.y);
          vf[2] = cval(f1.x);
          vf[3] = cval(f1.y);
        }
        TS d[4];
        if (MODE == 0) {
          const TS za = pwt[8 * te + 6], zb = pwt[8 * te + 7];
#pragma unroll
          for (int e = 0; e < 4; ++e) d[e] = vf[e] - za * Ip[k][e] - zb * In[k][e];
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) d[e] = vf[e];
        }
        if constexpr (BF && (PK || MODE == 0)) {
          d[0] = (vx0 && vy0[k]) ? d[0] : TS(0);
          d[1] = (vx1 && vy0[k]) ? d[1] : TS(0);
          d[2] = (vx0 && vy1[k]) ? d[2] : TS(0);
          d[3] = (vx1 && vy1[k]) ? d[3] : TS(0);
        }
        if constexpr (!BF) {
          *reinterpret_cast<TS2*>(cf + r0 * CP + cx0) = TS2{d[0], d[1]};
          *reinterpret_cast<TS2*>(cf + (r0 + 1) * CP + cx0) = TS2{d[2], d[3]};
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) dd[e] = d[e];
        if (!RS && wy && own_f) {
          LVL_YP(yzf + yr0[k] + yc0, yzf + yr0[k] + yc1, yval(d[0], owy0[k] && owx0), yval(d[1], owy0[k] && owx1), owy0[k] && owx0,
                         owy0[k] && owx1, ycontig);
          LVL_YP(yzf + yr1[k] + yc0, yzf + yr1[k] + yc1, yval(d[2], owy1[k] && owx0), yval(d[3], owy1[k] && owx1), owy1[k] && owx0,
                         owy1[k] && owx1, ycontig);
        }
      }
      if constexpr (BF) {
        // FP32: both planes interleaved, {coarse plane, fine plane} per node
        *reinterpret_cast<float4*>(cbuf + 2 * (r0 * CP + cx0)) = make_float4(c[0], dd[0], c[1], dd[1]);
        *reinterpret_cast<float4*>(cbuf + 2 * ((r0 + 1) * CP + cx0)) = make_float4(c[2], dd[2], c[3], dd[3]);
      }
    }
    // The x stencil and the row stores read only this warp's rows of the
    // coefficient tile: a warp barrier orders them.  With one stage buffer,
    // FP32 reloads the buffer whose rows the warp above still reads (nxt0 /
    // nxt1): a CTA barrier then.  (The x-stencil results that the y stencil
    // reads across warps are written after the previous plane pair's last CTA
    // barrier and read after this one's.)
    if constexpr (BF && STAGES == 1) __syncthreads();
    else __syncwarp();

    if (STAGES == 1 && t < t_end) issue(t + 1);  // every thread is done with the stage buffer

    // ---- coefficients of this warp's owned rows (RS), from the shared tile
    if constexpr (RS) {
      if (wy && (own_c || own_f)) {
#pragma unroll
        for (int k = 0; k < RPW; ++k) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int r = 2 * (warp * RPW + k) + h;
            const bool orow = h == 0 ? owy0[k] : owy1[k];
            const int yr = h == 0 ? yr0[k] : yr1[k];
            // {coarse plane, fine plane} pairs of the interleaved tile
            const float2 v0 = *reinterpret_cast<const float2*>(cbuf + 2 * (r * CP + rsl0));
            const float2 v1 = *reinterpret_cast<const float2*>(cbuf + 2 * (r * CP + rsl1));
            if (orow && own_c) {
              if (rs0) LVL_Y(yzc + yr + ro0, TD(v0.x));
              if (rs1) LVL_Y(yzc + yr + ro1, TD(v1.x));
            }
            if (orow && own_f) {
              if (rs0) LVL_Y(yzf + yr + ro0, TD(v0.y));
              if (rs1) LVL_Y(yzf + yr + ro1, TD(v1.y));
            }
          }
        }
      }
    }

    // ---- x stencil on every row of this warp (both planes)
    if constexpr (BF) {
      // FP32, both planes at once: {coarse, fine} pairs in the interleaved
      // tiles, paired FMAs (the results equal two scalar FMA chains)
      if (kxo && kx_generic) {
        // every row's five taps from two 16-byte loads and one 8-byte load
#pragma unroll
        for (int k = 0; k < RPW; ++k) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int r = 2 * (warp * RPW + k) + h;
            const float* row = cbuf + 2 * (r * CP + dx - 2);
            const float4 t01 = *reinterpret_cast<const float4*>(row);
            const float4 t23 = *reinterpret_cast<const float4*>(row + 4);
            const float2 t4 = *reinterpret_cast<const float2*>(row + 8);
            float2 g = __fmul2_rn(make_float2(kx(0), kx(0)), make_float2(t01.x, t01.y));
            g = __ffma2_rn(make_float2(kx(1), kx(1)), make_float2(t01.z, t01.w), g);
            g = __ffma2_rn(make_float2(kx(2), kx(2)), make_float2(t23.x, t23.y), g);
            g = __ffma2_rn(make_float2(kx(3), kx(3)), make_float2(t23.z, t23.w), g);
            g = __ffma2_rn(make_float2(kx(4), kx(4)), t4, g);
            *reinterpret_cast<float2*>(gxb + 2 * (r * GP + lane)) = g;
          }
        }
      } else if (kxo) {
        // boundary columns: clamped slots, weight 0 outside the grid
#pragma unroll
        for (int k = 0; k < RPW; ++k) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int r = 2 * (warp * RPW + k) + h;
            float2 g = make_float2(0.f, 0.f);
#pragma unroll
            for (int o = 0; o < 5; ++o) {
              const int j = min(max(dx - 2 + o, 0), RC - 1);  // weight 0 where clamped
              g = __ffma2_rn(make_float2(kx(o), kx(o)), *reinterpret_cast<const float2*>(cbuf + 2 * (r * CP + j)), g);
            }
            *reinterpret_cast<float2*>(gxb + 2 * (r * GP + lane)) = g;
          }
        }
      }
    } else if (kxo) {
#pragma unroll
      for (int k = 0; k < RPW; ++k) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = 2 * (warp * RPW + k) + h;
          // rows coarse in y (of the coarse-z plane): c vanishes on coarse columns
          const bool zero_row = (h == 0 || !fy1[k]) && !afine;
          TS g, gf = TS(0);
          if (kx_generic) {
            const TS* row = cc + r * CP + dx - 2;
            const TS2 a01 = *reinterpret_cast<const TS2*>(row);
            const TS2 a23 = *reinterpret_cast<const TS2*>(row + 2);
            if (zero_row) {
              g = kx(1) * a01.y + kx(3) * a23.y;
            } else {
              g = kx(0) * a01.x + kx(1) * a01.y + kx(2) * a23.x + kx(3) * a23.y + kx(4) * row[4];
            }
            if (hf) {
              const TS* rf = cf + r * CP + dx - 2;
              const TS2 b01 = *reinterpret_cast<const TS2*>(rf);
              const TS2 b23 = *reinterpret_cast<const TS2*>(rf + 2);
              gf = kx(0) * b01.x + kx(1) * b01.y + kx(2) * b23.x + kx(3) * b23.y + kx(4) * rf[4];
            }
          } else {
            g = TS(0);
#pragma unroll
            for (int o = 0; o < 5; ++o)
              if (kxm & (1u << o)) {
                g += kx(o) * cc[r * CP + dx - 2 + o];
                if (hf) gf += kx(o) * cf[r * CP + dx - 2 + o];
              }
          }
          gxb[r * GP + lane] = g;
          if (hf) gxb[RR * GP + r * GP + lane] = gf;
        }
      }
    }
    __syncthreads();

    // ---- y stencil and z accumulation for this thread's outputs
    // z weights of the two planes for coarse planes t-1, t, t+1 (plane table)
    TS wzc[3], wzf[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) wzc[i] = pwt[8 * te + i];
#pragma unroll
    for (int i = 0; i < 2; ++i) wzf[i] = pwt[8 * te + 3 + i];
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
      const int j = warp * RPW + k;
      if constexpr (BF) {
        // both planes at once ({coarse, fine} pairs, paired FMAs), five taps;
        // rows clamped into the tile (weight 0 where clamped); computed on
        // every lane of a row slot with outputs (j < nby: uniform across the
        // row group), stored only where the output exists
        if (j < nby) {
          const float* gcol = gxb + 2 * lane;
          float2 g;
          if (kym[k] == 31u) {
            const float* g0 = gcol + 2 * (dyo[k] - 2) * GP;
            g = __fmul2_rn(make_float2(ky(k, 0), ky(k, 0)), *reinterpret_cast<const float2*>(g0));
#pragma unroll
            for (int o = 1; o < 5; ++o)
              g = __ffma2_rn(make_float2(ky(k, o), ky(k, o)), *reinterpret_cast<const float2*>(g0 + 2 * o * GP), g);
          } else {
            g = make_float2(0.f, 0.f);
#pragma unroll
            for (int o = 0; o < 5; ++o) {
              const int rr = min(max(dyo[k] + o - 2, 0), RR - 1);
              g = __ffma2_rn(make_float2(ky(k, o), ky(k, o)), *reinterpret_cast<const float2*>(gcol + 2 * rr * GP), g);
            }
          }
          const TS gc = g.x, gf = g.y;
          acc0[k] += wzc[0] * gc;
          acc1[k] += wzc[1] * gc;
          acc2[k] += wzc[2] * gc;
          acc0[k] += wzf[0] * gf;
          acc1[k] += wzf[1] * gf;
          if (kxo && t - 1 >= qz0 && t - 1 < qz1)
            LVL_F(int64_t(t - 1) * a.c_sz + int64_t(qy0 + j) * a.c_sy + qxo, fout(acc0[k]));
        }
      } else if (j < nby && kxo) {
        TS gc = TS(0), gf = TS(0);
        const TS* gcol = gxb + (dyo[k] - 2) * GP + lane;
        if (kym[k] == 31u) {  // interior row: all five taps inside the grid
          gc = ky(k, 0) * gcol[0] + ky(k, 1) * gcol[GP] + ky(k, 2) * gcol[2 * GP] + ky(k, 3) * gcol[3 * GP] +
               ky(k, 4) * gcol[4 * GP];
          if (hf) {
            const TS* fcol = gcol + RR * GP;
            gf = ky(k, 0) * fcol[0] + ky(k, 1) * fcol[GP] + ky(k, 2) * fcol[2 * GP] + ky(k, 3) * fcol[3 * GP] +
                 ky(k, 4) * fcol[4 * GP];
          }
        } else {
#pragma unroll
          for (int o = 0; o < 5; ++o) {
            if (kym[k] & (1u << o)) {
              gc += ky(k, o) * gxb[(dyo[k] + o - 2) * GP + lane];
              if (hf) gf += ky(k, o) * gxb[RR * GP + (dyo[k] + o - 2) * GP + lane];
            }
          }
        }
        acc0[k] += wzc[0] * gc;
        acc1[k] += wzc[1] * gc;
        acc2[k] += wzc[2] * gc;
        if (hf) {
          acc0[k] += wzf[0] * gf;
          acc1[k] += wzf[1] * gf;
        }
        if (t - 1 >= qz0 && t - 1 < qz1)
          LVL_F(int64_t(t - 1) * a.c_sz + int64_t(qy0 + j) * a.c_sy + qxo, fout(acc0[k]));
      }
      acc0[k] = acc1[k];
      acc1[k] = acc2[k];
      acc2[k] = TS(0);
#pragma unroll
      for (int e = 0; e < 4; ++e) Ip[k][e] = In[k][e];
    }
  }
  if (t_end == mz - 1 && qz1 == mz) {
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
      const int j = warp * RPW + k;
      if (j < nby && kxo) LVL_F(int64_t(mz - 1) * a.c_sz + int64_t(qy0 + j) * a.c_sy + qxo, fout(acc0[k]));
    }
  }
}

#undef LVL_CP
#undef LVL_CPZ
#undef LVL_Y
#undef LVL_YP
#undef LVL_W
#undef LVL_F

template <int MODE, int NW, int RPW, int STAGES, typename TI, typename TD, typename TS, typename TW, bool PK, bool QZ>
__global__ void __launch_bounds__(NW * 32, level_ctas_per_sm(NW)) k_level(const LevelArgs<TS, TW> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  level_body<MODE, NW, RPW, STAGES, TI, TD, TS, TW, PK, QZ>(a, blockIdx.x, blockIdx.y, blockIdx.z + a.bz0, smem_raw);
}

// ---------------------------------------------------------------------------
// Recomposition interpolation (Sec. II.A, recomposition): level-l values
// v = c + (P_z x P_y x P_x) v_coarse.  A CTA owns LX x (NW*32/LX*RPW) coarse
// (x, y) nodes (LX = 32, or 16 in half-warp row groups) and a chunk of
// coarse z planes; lane l / row k of a row group own the
// fine block {p(q), p(q)+1} x {p(q), p(q)+1} of their coarse node (the second
// node only when a fine node lies between q and q+1).  The coarse plane tile
// (one extra row and column for the right / lower neighbours) is staged in
// shared memory; the xy interpolants of each coarse plane stay in registers
// for the fine plane between it and the next one.
// ---------------------------------------------------------------------------
template <typename TS, typename TW>
struct InterpArgs {
  const void* c;  // coefficients: nodal (full grid) or this level's packed class; null = all zero
  int64_t y_sz, y_sy;
  const TW* w;    // coarse values (compact m grid)
  int64_t c_sz, c_sy;
  void* out;      // level-l values: full grid (out_full) or compact n grid
  int64_t o_sz, o_sy;
  int out_full;
  int n[3], m[3];
  int64_t s[3], N[3];
  const TS* wa[3];
  const TS* wb[3];
  int qz_chunk;
  int bz0;    // first z chunk of this launch (a launch may cover a subset of the chunks)
  double qs;  // QZ: bin width of the level's class
};

// Row groups of LX lanes (a warp, or half of one for fields with short coarse
// rows): a CTA of NW warps owns LX x (NW * 32 / LX * RPW) coarse nodes.
template <int NW, int RPW, typename TD, typename TW, int LX = 32>
constexpr size_t interp_table_offset() {
  constexpr int BY = NW * 32 / LX * RPW, TC = LX == 32 ? 33 : 24;
  return (sizeof(TD) * 2 * 2 * (2 * BY) * (2 * LX) + sizeof(TW) * 2 * (BY + 1) * TC + 15) / 16 * 16;
}
// plane table: per plane pair six offsets (int64), two weights, a flag
template <int NW, int RPW, typename TD, typename TS, typename TW, int LX = 32>
constexpr size_t interp_smem_bytes() {
  return interp_table_offset<NW, RPW, TD, TW, LX>() + kLevelPlanes * (6 * sizeof(int64_t) + 2 * sizeof(TS) + sizeof(int));
}

// PK: `c` is the class-packed class of this level (y_sz = n1*n2, y_sy = n2).
// QZ (with PK): `c` holds int32 codes (TD = int), coefficient = code * qs.
template <int NW, int RPW, typename TD, typename TO, typename TS, typename TW, bool PK = false, bool QZ = false,
          int LX = 32>
__device__ __forceinline__ void interp_body(const InterpArgs<TS, TW>& a, int bx, int by, int bz,
                                            unsigned char* smem_raw) {
  static_assert(LX == 32 || LX == 16, "row groups of a warp or half a warp");
  // coarse tile pitch: LX + 1 columns, padded for half-warp groups so that
  // the two halves of a warp (RPW rows apart) read different banks
  constexpr int BY = NW * 32 / LX * RPW, TR = BY + 1, TC = LX == 32 ? 33 : 24, RR = 2 * BY, RC = 2 * LX;
  using TD2 = typename Pair<TD>::type;
  TD* stage = reinterpret_cast<TD*>(smem_raw);                                  // [2][2][RR][RC]
  TW* tile = reinterpret_cast<TW*>(smem_raw + sizeof(TD) * 2 * 2 * RR * RC);  // [2][TR][TC]
  const int lane = threadIdx.x % LX, warp = threadIdx.x / LX;  // lane in the row group, row group
  const int nz = a.n[0], ny = a.n[1], nx = a.n[2];
  const int mz = a.m[0], my = a.m[1], mx = a.m[2];
  const int qx0 = bx * LX, qy0 = by * BY;
  const int qz0 = bz * a.qz_chunk, qz1 = min(qz0 + a.qz_chunk, mz);
  const int t_end = min(qz1, mz - 1);
  const int tcols = min(LX + 1, mx - qx0), trows = min(TR, my - qy0);
  const TD* __restrict__ cin = static_cast<const TD*>(a.c);
  const bool cz = cin == nullptr;  // coefficients of a dropped class: zero
  const TS qs = QZ ? TS(a.qs) : TS(1);
  // coefficient v plus interpolant b (QZ: code * q + b in one FMA)
  auto cadd = [&](TD v, TS b) -> TS {
    if constexpr (QZ) return fma(code_value<TS>(int(v)), qs, b);
    else return TS(v) + b;
  };
  TO* __restrict__ out = static_cast<TO*>(a.out);
  // bounds-checking builds: extents of the buffers; the ITP_* statements
  // check against them (other builds run the plain statements)
#ifdef MGR_DEBUG_BOUNDS
  const long long n_ci = PK ? (long long)nz * a.y_sz - (long long)mz * a.c_sz : (long long)a.N[0] * a.y_sz;
  const long long n_w = (long long)mz * a.c_sz;
  const long long n_o = (long long)(a.out_full ? a.N[0] : nz) * a.o_sz;
  constexpr long long n_stage = 2LL * 2 * RR * RC;
#endif
#define ITP_CP(dst, src) \
  MGR_GUARD(MGR_PIN(src, cin, n_ci, kDbgInterpC) && MGR_PIN(dst, stage, n_stage, kDbgInterpStage), \
            cp_async(dst, src, int(sizeof(TD))))
#define ITP_LP(dst, s0, s1, v0, v1, contig)                                                                          \
  MGR_GUARD((!(v0) || MGR_PIN(s0, cin, n_ci, kDbgInterpC)) && (!(v1) || MGR_PIN(s1, cin, n_ci, kDbgInterpC)) && \
                MGR_PIN((dst) + 1, stage, n_stage, kDbgInterpStage),                                              \
            load_pair(dst, s0, s1, v0, v1, contig))
#define ITP_OP(p0, p1, a0, a1, w0, w1, contig)                                                                          \
  MGR_GUARD((!(w0) || MGR_PIN(p0, out, n_o, kDbgInterpOut)) && (!(w1) || MGR_PIN(p1, out, n_o, kDbgInterpOut)), \
            store_pair<TO>(p0, p1, a0, a1, w0, w1, contig))

  // column block of this lane: fine nodes p(qx) and, when a fine node lies
  // between qx and qx+1, p(qx)+1
  const int qx = qx0 + lane;
  const bool ax = qx < mx;
  const int gx0 = pidx(min(qx, mx - 1), nx);
  const bool ox1 = ax && qx + 1 < mx && pidx(qx + 1, nx) - gx0 == 2;
  const TS wax1 = ox1 ? a.wa[2][gx0 + 1] : TS(0), wbx1 = ox1 ? a.wb[2][gx0 + 1] : TS(0);
  const int gx1 = min(gx0 + 1, nx - 1);
  const int cc0 = PK ? gx0 : int(fmap(gx0, a.s[2], a.N[2])), cc1 = PK ? gx1 : int(fmap(gx1, a.s[2], a.N[2]));
  const bool ccontig = cc1 == cc0 + 1;
  const int pcx1 = gx1 - cidx(gx1);  // packed column of gx1 in a row coarse in y and z
  const int oc0 = a.out_full ? cc0 : gx0, oc1 = a.out_full ? cc1 : gx1;
  const bool ocontig = oc1 == oc0 + 1;
  // row blocks
  bool ay[RPW], oy1[RPW];
  TS way1[RPW], wby1[RPW];
  int cr0[RPW], cr1[RPW], crc0[RPW], crc1[RPW];
  int64_t or0[RPW], or1[RPW];
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const int qy = qy0 + warp * RPW + k;
    ay[k] = qy < my;
    const int g0 = pidx(min(qy, my - 1), ny);
    oy1[k] = ay[k] && qy + 1 < my && pidx(qy + 1, ny) - g0 == 2;
    way1[k] = oy1[k] ? a.wa[1][g0 + 1] : TS(0);
    wby1[k] = oy1[k] ? a.wb[1][g0 + 1] : TS(0);
    const int g1 = min(g0 + 1, ny - 1);
    cr0[k] = PK ? g0 * nx : int(fmap(g0, a.s[1], a.N[1]) * a.y_sy);
    cr1[k] = PK ? g1 * nx : int(fmap(g1, a.s[1], a.N[1]) * a.y_sy);
    // packed rows of a coarse plane
    crc0[k] = g0 * nx - cidx(g0) * mx;
    crc1[k] = g1 * nx - cidx(g1) * mx;
    or0[k] = (a.out_full ? fmap(g0, a.s[1], a.N[1]) : int64_t(g0)) * a.o_sy;
    or1[k] = (a.out_full ? fmap(g1, a.s[1], a.N[1]) : int64_t(g1)) * a.o_sy;
  }

  // ---- plane table, computed once by the CTA (instead of by every warp on
  // every plane pair): entry t - qz0 holds the offsets of plane pair t's
  // coefficient planes (coarse p(t), and the fine plane before it when there
  // is one), of its output planes, of the coarse values' plane t, and the
  // fine plane's z interpolation weights
  int64_t* itab = reinterpret_cast<int64_t*>(smem_raw + interp_table_offset<NW, RPW, TD, TW, LX>());
  TS* iwt = reinterpret_cast<TS*>(itab + 6 * kLevelPlanes);
  int* ifl = reinterpret_cast<int*>(iwt + 2 * kLevelPlanes);
  auto cplane = [&](int g) -> int64_t {
    return PK ? int64_t(g) * a.y_sz - int64_t(cidx(g)) * a.c_sz : fmap(g, a.s[0], a.N[0]) * a.y_sz;
  };
  auto oplane = [&](int g) -> int64_t { return (a.out_full ? fmap(g, a.s[0], a.N[0]) : int64_t(g)) * a.o_sz; };
  (void)MGR_IN(t_end - qz0, kLevelPlanes, kDbgInterpStage);
  for (int e = threadIdx.x; e <= t_end - qz0 && e < kLevelPlanes; e += NW * 32) {
    const int t = qz0 + e, Pc = pidx(t, nz), Pf = Pc - 1;
    const bool hf = t > qz0 && Pc - pidx(t - 1, nz) == 2;
    itab[6 * e + 0] = cplane(Pc);
    itab[6 * e + 1] = hf ? cplane(Pf) : 0;
    itab[6 * e + 2] = oplane(Pc);
    itab[6 * e + 3] = oplane(max(Pf, 0));
    itab[6 * e + 4] = int64_t(t) * a.c_sz;
    iwt[2 * e + 0] = hf ? a.wa[0][Pf] : TS(0);
    iwt[2 * e + 1] = hf ? a.wb[0][Pf] : TS(0);
    ifl[e] = hf ? 1 : 0;
  }
  // this thread's copies of the coarse tile: offsets in the coarse plane
  // (-1: none) and slots
  constexpr int KT = (TR * TC + NW * 32 - 1) / (NW * 32);
  int tgo[KT], tso[KT];
#pragma unroll
  for (int i = 0; i < KT; ++i) {
    const int e = threadIdx.x + i * NW * 32;
    const int r = e / TC, cix = e - r * TC;
    tgo[i] = (e < trows * TC && cix < tcols) ? int(int64_t(r) * a.c_sy + cix) : -1;
    tso[i] = r * TC + cix;
  }
  const int64_t wtile0 = int64_t(qy0) * a.c_sy + qx0;
  __syncthreads();  // plane table staged

  // coefficient plane at offset poff of `cin`; zc: a coarse plane
  auto load_c = [&](TD* sb, int64_t poff, bool zc) {
    if (cz) return;
    if constexpr (PK) {
      const TD* base = cin + poff;
#pragma unroll
      for (int k = 0; k < RPW; ++k) {
        const int r0 = 2 * (warp * RPW + k);
        if (!ay[k]) continue;
        if (zc) {
          // the coarse row g0 of a coarse plane holds its fine column only
          if (ox1) ITP_CP(sb + r0 * RC + 2 * lane + 1, base + crc0[k] + pcx1);
          if (oy1[k])
            ITP_LP(sb + (r0 + 1) * RC + 2 * lane, base + crc1[k] + cc0, base + crc1[k] + cc1, ax, ox1, true);
        } else {
          ITP_LP(sb + r0 * RC + 2 * lane, base + cr0[k] + cc0, base + cr0[k] + cc1, ax, ox1, true);
          if (oy1[k])
            ITP_LP(sb + (r0 + 1) * RC + 2 * lane, base + cr1[k] + cc0, base + cr1[k] + cc1, ax, ox1, true);
        }
      }
      return;
    }
    const TD* base = cin + poff;
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
      const int r0 = 2 * (warp * RPW + k);
      if (ay[k]) {
        ITP_LP(sb + r0 * RC + 2 * lane, base + cr0[k] + cc0, base + cr0[k] + cc1, ax, ox1, ccontig);
        if (oy1[k]) ITP_LP(sb + (r0 + 1) * RC + 2 * lane, base + cr1[k] + cc0, base + cr1[k] + cc1, ax, ox1, ccontig);
      }
    }
  };
  auto issue = [&](int t) {
    const int e = t - qz0, st = e & 1;
    TW* tb = tile + st * TR * TC;
    const TW* src = a.w + itab[6 * e + 4] + wtile0;
#pragma unroll
    for (int i = 0; i < KT; ++i)
      if (tgo[i] >= 0)
        MGR_GUARD(MGR_PIN(src + tgo[i], a.w, n_w, kDbgInterpW), cp_async(tb + tso[i], src + tgo[i], int(sizeof(TW))));
    TD* sb = stage + st * 2 * RR * RC;
    if (t < qz1) load_c(sb, itab[6 * e + 0], true);
    if (ifl[e]) load_c(sb + RR * RC, itab[6 * e + 1], false);
    cp_commit();
  };

  auto ldc = [&](const TD* p) -> TD2 {
    TD2 v;
    if (cz) {
      v.x = v.y = TD(0);
    } else {
      v = *reinterpret_cast<const TD2*>(p);
    }
    return v;
  };

  TS Ip[RPW][4], In[RPW][4];
#pragma unroll
  for (int k = 0; k < RPW; ++k)
#pragma unroll
    for (int e = 0; e < 4; ++e) Ip[k][e] = In[k][e] = TS(0);

  issue(qz0);
  for (int t = qz0; t <= t_end; ++t) {
    if (t < t_end) {
      issue(t + 1);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    const int st = (t - qz0) & 1;
    const TW* tb = tile + st * TR * TC;
    const TD* sc = stage + st * 2 * RR * RC;
    const TD* sf = sc + RR * RC;
    const int te = t - qz0;
    const bool own_c = t < qz1;
    const bool hf = ifl[te] != 0;
    TO* ozc = out + itab[6 * te + 2];
    TO* ozf = out + itab[6 * te + 3];
    const TS za = iwt[2 * te + 0], zb = iwt[2 * te + 1];
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
      const int r = warp * RPW + k;
      const int r0 = 2 * r;
      const bool act = ax && ay[k];
      // coarse neighbours (clamped reads stay inside the staged tile)
      const int rr1 = min(r + 1, trows - 1), cl1 = min(lane + 1, tcols - 1);
      const int rr0 = min(r, trows - 1), cl0 = min(lane, tcols - 1);
      const TW w00r = tb[rr0 * TC + cl0];
      const TS w00 = TS(w00r), w01 = TS(tb[rr0 * TC + cl1]);
      const TS w10 = TS(tb[rr1 * TC + cl0]), w11 = TS(tb[rr1 * TC + cl1]);
      In[k][0] = w00;
      In[k][1] = ox1 ? wax1 * w00 + wbx1 * w01 : TS(0);
      In[k][2] = oy1[k] ? way1[k] * w00 + wby1[k] * w10 : TS(0);
      if (ox1 && oy1[k]) {
        const TS i21 = wax1 * w10 + wbx1 * w11;
        In[k][3] = way1[k] * In[k][1] + wby1[k] * i21;
      } else {
        In[k][3] = TS(0);
      }
      if (act && own_c) {
        const TD2 c0 = ldc(sc + r0 * RC + 2 * lane);
        ITP_OP(ozc + or0[k] + oc0, ozc + or0[k] + oc1, TO(w00r), TO(cadd(c0.y, In[k][1])), true, ox1, ocontig);
        if (oy1[k]) {
          const TD2 c1 = ldc(sc + (r0 + 1) * RC + 2 * lane);
          ITP_OP(ozc + or1[k] + oc0, ozc + or1[k] + oc1, TO(cadd(c1.x, In[k][2])), TO(cadd(c1.y, In[k][3])),
                         true, ox1, ocontig);
        }
      }
      if (act && hf) {
        const TD2 c0 = ldc(sf + r0 * RC + 2 * lane);
        ITP_OP(ozf + or0[k] + oc0, ozf + or0[k] + oc1, TO(QZ ? cadd(c0.x, za * Ip[k][0] + zb * In[k][0]) : TS(c0.x) + za * Ip[k][0] + zb * In[k][0]),
                       TO(QZ ? cadd(c0.y, za * Ip[k][1] + zb * In[k][1]) : TS(c0.y) + za * Ip[k][1] + zb * In[k][1]), true, ox1, ocontig);
        if (oy1[k]) {
          const TD2 c1 = ldc(sf + (r0 + 1) * RC + 2 * lane);
          ITP_OP(ozf + or1[k] + oc0, ozf + or1[k] + oc1, TO(QZ ? cadd(c1.x, za * Ip[k][2] + zb * In[k][2]) : TS(c1.x) + za * Ip[k][2] + zb * In[k][2]),
                         TO(QZ ? cadd(c1.y, za * Ip[k][3] + zb * In[k][3]) : TS(c1.y) + za * Ip[k][3] + zb * In[k][3]), true, ox1, ocontig);
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) Ip[k][e] = In[k][e];
    }
    __syncthreads();  // both stage buffers are reloaded two iterations later
  }
}

#undef ITP_CP
#undef ITP_LP
#undef ITP_OP

template <int NW, int RPW, typename TD, typename TO, typename TS, typename TW, bool PK, bool QZ>
__global__ void __launch_bounds__(NW * 32, level_ctas_per_sm(NW)) k_interp(const InterpArgs<TS, TW> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  interp_body<NW, RPW, TD, TO, TS, TW, PK, QZ>(a, blockIdx.x, blockIdx.y, blockIdx.z + a.bz0, smem_raw);
}
