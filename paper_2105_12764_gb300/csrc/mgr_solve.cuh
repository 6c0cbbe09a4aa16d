// mgr_solve.cuh -- Thomas solves of the coarse mass matrix along one axis
// (arXiv 2105.12764, Sec. III.A.3) and the coarsest-grid copy, as per-CTA
// bodies (used by the single-field kernels below and by the batched ones).
//
// The LU of the coarse mass matrix is scaled so each step is one FMA (the
// diagonal 1/u_q is folded into the mass-transfer stencil):
//   forward   y_q = f'_q - ta_q * y_{q-1}
//   backward  z_q = y_q  - tb_q * z_{q+1}
// The last axis of a level applies the correction (Eq. (1)) into the coarse
// workspace: w += z (decompose) or w -= z (recompose).
#pragma once

enum { SOLVE_INPLACE = 0, SOLVE_ADD = 1, SOLVE_SUB = 2 };

template <typename TW>
__device__ __forceinline__ void apply_op(TW* f, TW* w, int64_t g, TW v, int op) {
  if (op == SOLVE_INPLACE) f[g] = v;
  else if (op == SOLVE_ADD) w[g] = w[g] + v;
  else w[g] = w[g] - v;
}

// Lines along a strided axis, one thread per line: element q of line
// (o, i) sits at o*ostride + i + q*lstride; consecutive threads take
// consecutive i, so every step is a coalesced access.  `line` is this
// thread's line index in [0, inner*outer).  U elements of the line are
// loaded before the recurrence runs through them (loads in flight per thread).
template <typename TW, int U = 8>
__device__ __forceinline__ void solve_strided_line(TW* __restrict__ f, TW* __restrict__ w, int mline, int64_t lstride,
                                                   int inner, int64_t ostride, const TW* __restrict__ ta,
                                                   const TW* __restrict__ tb, int op, int64_t line,
                                                   long long ext = 0) {
  (void)ext;  // elements of f and w (the coarse grid): checked in bounds-checking builds
  const int i = int(line % inner);
  const int64_t o = line / inner;
  // the line's elements are o*ostride + i + q*lstride, q = 0..mline-1: its ends bound them all
  if (!MGR_IN(o * ostride + i, ext, kDbgSolveF) || !MGR_IN(o * ostride + i + int64_t(mline - 1) * lstride, ext, kDbgSolveF))
    return;
  TW* fl = f + o * ostride + i;
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
    if (op != SOLVE_INPLACE) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (q1 - u >= 0) wv[u] = wl[int64_t(q1 - u) * lstride];
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (q1 - u >= 0) {
        const int q = q1 - u;
        next = buf[u] - tb[q] * next;
        if (op == SOLVE_INPLACE) fl[int64_t(q) * lstride] = next;
        else if (op == SOLVE_ADD) wl[int64_t(q) * lstride] = wv[u] + next;
        else wl[int64_t(q) * lstride] = wv[u] - next;
      }
  }
}

#ifndef MGR_SOLVE_U32
#define MGR_SOLVE_U32 16
#endif
#ifndef MGR_SOLVE_U64
#define MGR_SOLVE_U64 8
#endif
template <typename TW>
__global__ void __launch_bounds__(128) k_solve_strided(TW* __restrict__ f, TW* __restrict__ w, int mline,
                                                       int64_t lstride, int inner, int64_t outer, int64_t ostride,
                                                       const TW* __restrict__ ta, const TW* __restrict__ tb, int op) {
  const int64_t id = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (id >= int64_t(inner) * outer) return;
  // loads in flight per thread and sweep (build-time knobs; sixteen FP64
  // elements cost occupancy and were slower than eight)
  solve_strided_line<TW, sizeof(TW) == 4 ? MGR_SOLVE_U32 : MGR_SOLVE_U64>(f, w, mline, lstride, inner, ostride, ta, tb, op, id,
                                                   max(int64_t(mline) * lstride, outer * ostride));
}

// Lines along a strided axis, 32 per CTA, staged whole in shared memory: the
// CTA's lines (consecutive line indices, so each step q is one or two
// contiguous row segments) are copied in with asynchronous copies all in
// flight, one warp runs the 32 recurrences on the staged lines, and the CTA
// writes them back (or applies the correction).  Each element crosses HBM
// once each way instead of twice, and all of a CTA's loads are in flight at
// once: the form for coarse levels, whose few lines leave the one-thread-per-
// line kernel latency-bound.  With many lines the single computing warp per
// CTA bounds it, and the one-thread-per-line kernel is faster.
constexpr int kStagedLines = 32;

template <typename TW>
size_t solve_staged_smem(int mline) {
  return sizeof(TW) * (size_t(mline) * kStagedLines + 2 * size_t(mline)) + sizeof(int64_t) * kStagedLines;
}

// Lines l0 .. l0+31 of the axis (the body of k_solve_staged and of the batched
// staged solves).
template <typename TW>
__device__ __forceinline__ void solve_staged_lines(TW* __restrict__ f, TW* __restrict__ w, int mline,
                                                   int64_t lstride, int inner, int64_t outer, int64_t ostride,
                                                   const TW* __restrict__ ta, const TW* __restrict__ tb, int op,
                                                   int64_t l0, unsigned char* smem_raw) {
  constexpr int NL = kStagedLines;
  TW* s = reinterpret_cast<TW*>(smem_raw);  // [mline][NL]
  TW* sa = s + int64_t(mline) * NL;           // [mline]
  TW* sb = sa + mline;                        // [mline]
  int64_t* off = reinterpret_cast<int64_t*>(sb + mline);  // [NL] offset of each line's first element
  const int64_t lines = int64_t(inner) * outer;
  const int nl = int(lines - l0 < NL ? lines - l0 : NL);
  if (threadIdx.x < NL) {
    const int64_t line = l0 + (threadIdx.x < nl ? threadIdx.x : 0);
    const int64_t o = line / inner;
    const int64_t first = o * ostride + (line - o * inner);
#ifdef MGR_DEBUG_BOUNDS
    // a line's elements are first + q*lstride: its ends bound them all (out of
    // bounds: recorded, and the line is pointed at element 0 to stay inside)
    const long long ext = max(int64_t(mline) * lstride, outer * ostride);
    const bool ok = MGR_IN(first, ext, kDbgSolveF) && MGR_IN(first + int64_t(mline - 1) * lstride, ext, kDbgSolveF);
    off[threadIdx.x] = ok ? first : 0;
#else
    off[threadIdx.x] = first;
#endif
  }
  for (int q = threadIdx.x; q < mline; q += blockDim.x) {
    sa[q] = ta[q];
    sb[q] = tb[q];
  }
  __syncthreads();
  const int total = mline * NL;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int q = e / NL, j = e - q * NL;
    if (j < nl) cp_async(s + e, f + off[j] + int64_t(q) * lstride, int(sizeof(TW)));
  }
  cp_commit();
  cp_wait<0>();
  __syncthreads();
  if (threadIdx.x < nl) {
    const int j = threadIdx.x;
    constexpr int U = 8;
    TW prev = TW(0);
    for (int q0 = 0; q0 < mline; q0 += U) {
      TW v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = (q0 + u < mline) ? s[(q0 + u) * NL + j] : TW(0);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        prev = v[u] - sa[min(q0 + u, mline - 1)] * prev;
        v[u] = prev;
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (q0 + u < mline) s[(q0 + u) * NL + j] = v[u];
    }
    TW next = TW(0);
    for (int q1 = mline - 1; q1 >= 0; q1 -= U) {
      TW v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = (q1 - u >= 0) ? s[(q1 - u) * NL + j] : TW(0);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        next = v[u] - sb[max(q1 - u, 0)] * next;
        v[u] = next;
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (q1 - u >= 0) s[(q1 - u) * NL + j] = v[u];
    }
  }
  __syncthreads();
  constexpr int W = 8;
  for (int e0 = threadIdx.x; e0 < total; e0 += W * blockDim.x) {
    int64_t g[W];
    TW sv[W], wv[W];
    bool ok[W];
#pragma unroll
    for (int u = 0; u < W; ++u) {
      const int e = e0 + u * blockDim.x;
      const int ee = e < total ? e : 0;
      const int q = ee / NL, j = ee - q * NL;
      ok[u] = e < total && j < nl;
      g[u] = off[j] + int64_t(q) * lstride;
      sv[u] = s[ee];
      wv[u] = (op != SOLVE_INPLACE && ok[u]) ? w[g[u]] : TW(0);
    }
#pragma unroll
    for (int u = 0; u < W; ++u) {
      if (!ok[u]) continue;
      if (op == SOLVE_INPLACE) f[g[u]] = sv[u];
      else if (op == SOLVE_ADD) w[g[u]] = wv[u] + sv[u];
      else w[g[u]] = wv[u] - sv[u];
    }
  }
}

template <typename TW>
__global__ void __launch_bounds__(128) k_solve_staged(TW* __restrict__ f, TW* __restrict__ w, int mline,
                                                      int64_t lstride, int inner, int64_t outer, int64_t ostride,
                                                      const TW* __restrict__ ta, const TW* __restrict__ tb,
                                                      int op) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  solve_staged_lines<TW>(f, w, mline, lstride, inner, outer, ostride, ta, tb, op, int64_t(blockIdx.x) * kStagedLines,
                         smem_raw);
}

// Lines along the contiguous axis: R rows of length mline (row pitch
// row_pitch) starting at row r0 are staged in shared memory with coalesced
// asynchronous copies by all threads; thread r < R then runs its row's
// recurrences through 16-byte vectors of the staged row (one shared load,
// E = 16 / sizeof(TW) dependent FMAs and one shared store per vector), and
// all threads write the rows back.  The recurrence coefficients are staged
// once, zero-padded to the pitch.
//
// Shared row pitch: a whole, odd number of 16-byte vectors.  A 16-byte shared
// access is served eight threads at a time, and rows whose starts differ by
// an odd number of vectors put those eight in different bank groups.
template <typename TW>
constexpr int contig_pitch(int mline) {
  constexpr int E = 16 / int(sizeof(TW));
  const int v = (mline + E - 1) / E;
  return ((v & 1) ? v : v + 1) * E;
}
template <typename TW>
constexpr size_t solve_contig_smem(int mline, int R) {
  return sizeof(TW) * (size_t(R) + 2) * size_t(contig_pitch<TW>(mline));
}
template <typename TW>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
};
template <>
struct Vec16<double> {
  using type = double2;
};

template <typename TW>
__device__ __forceinline__ void solve_contig_rows(TW* __restrict__ f, TW* __restrict__ w, int mline, int64_t rows,
                                                  int64_t row_pitch, int R, const TW* __restrict__ ta,
                                                  const TW* __restrict__ tb, int op, int64_t r0,
                                                  unsigned char* smem_raw) {
  const int pitch = contig_pitch<TW>(mline);
  TW* s = reinterpret_cast<TW*>(smem_raw);  // [R][pitch]
  TW* sa = s + R * pitch;                   // [pitch], zero past mline
  TW* sb = sa + pitch;                      // [pitch], zero past mline
  const int nr = int(rows - r0 < int64_t(R) ? rows - r0 : int64_t(R));
  // rows r0 .. r0+nr-1 of mline elements at pitch row_pitch
  if (!MGR_IN((r0 + nr - 1) * row_pitch + mline - 1, rows * row_pitch, kDbgSolveF)) return;
  // the rows go to shared memory as element-wise asynchronous copies, all in
  // flight at once (the staging, not the recurrences, bounds this kernel);
  // a warp takes whole rows, its lanes consecutive elements
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = wid; r < nr; r += nw) {
    const TW* src = f + (r0 + r) * row_pitch;
    TW* dst = s + r * pitch;
    for (int c = lane; c < mline; c += 32) cp_async(dst + c, src + c, int(sizeof(TW)));
  }
  cp_commit();
  for (int q = threadIdx.x; q < pitch; q += blockDim.x) {
    sa[q] = q < mline ? ta[q] : TW(0);
    sb[q] = q < mline ? tb[q] : TW(0);
  }
  cp_wait<0>();
  __syncthreads();
  if (threadIdx.x < nr) {
    using V = typename Vec16<TW>::type;
    constexpr int E = 16 / int(sizeof(TW));
    V* l = reinterpret_cast<V*>(s + threadIdx.x * pitch);
    const V* av = reinterpret_cast<const V*>(sa);
    const V* bv = reinterpret_cast<const V*>(sb);
    const int nv = (mline + E - 1) / E;  // vectors holding the row's elements
    // forward: the elements past mline in the last vector follow every real
    // one, so computing on them (the padding) changes nothing that is kept
    TW prev = TW(0);
#pragma unroll 2
    for (int i = 0; i < nv; ++i) {
      alignas(16) TW x[E];
      alignas(16) TW a[E];
      *reinterpret_cast<V*>(x) = l[i];
      *reinterpret_cast<V*>(a) = av[i];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        prev = x[e] - a[e] * prev;
        x[e] = prev;
      }
      l[i] = *reinterpret_cast<const V*>(x);
    }
    // backward from element mline-1: in the last vector the elements past
    // mline are skipped
    TW next = TW(0);
    {
      const int i = nv - 1;
      alignas(16) TW x[E];
      alignas(16) TW b[E];
      *reinterpret_cast<V*>(x) = l[i];
      *reinterpret_cast<V*>(b) = bv[i];
#pragma unroll
      for (int e = E - 1; e >= 0; --e)
        if (i * E + e < mline) {
          next = x[e] - b[e] * next;
          x[e] = next;
        }
      l[i] = *reinterpret_cast<const V*>(x);
    }
#pragma unroll 2
    for (int i = nv - 2; i >= 0; --i) {
      alignas(16) TW x[E];
      alignas(16) TW b[E];
      *reinterpret_cast<V*>(x) = l[i];
      *reinterpret_cast<V*>(b) = bv[i];
#pragma unroll
      for (int e = E - 1; e >= 0; --e) {
        next = x[e] - b[e] * next;
        x[e] = next;
      }
      l[i] = *reinterpret_cast<const V*>(x);
    }
  }
  __syncthreads();
  // write back (or apply the correction to w), a warp per row, W elements
  // per lane per round with their loads of w issued together
  constexpr int W = 8;
  for (int r = wid; r < nr; r += nw) {
    const TW* srow = s + r * pitch;
    const int64_t g0 = (r0 + r) * row_pitch;
    for (int c0 = lane; c0 < mline; c0 += 32 * W) {
      TW sv[W], wv[W];
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const int c = c0 + 32 * u;
        sv[u] = c < mline ? srow[c] : TW(0);
        wv[u] = (op != SOLVE_INPLACE && c < mline) ? w[g0 + c] : TW(0);
      }
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const int c = c0 + 32 * u;
        if (c >= mline) break;
        if (op == SOLVE_INPLACE) f[g0 + c] = sv[u];
        else if (op == SOLVE_ADD) w[g0 + c] = wv[u] + sv[u];
        else w[g0 + c] = wv[u] - sv[u];
      }
    }
  }
}

template <typename TW>
__global__ void __launch_bounds__(128) k_solve_contig(TW* __restrict__ f, TW* __restrict__ w, int mline, int64_t rows,
                                                      int64_t row_pitch, int R, const TW* __restrict__ ta,
                                                      const TW* __restrict__ tb, int op) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  solve_contig_rows<TW>(f, w, mline, rows, row_pitch, R, ta, tb, op, blockIdx.x * int64_t(R), smem_raw);
}

// Lines along the contiguous axis, 32 per warp (lane = line): the warp moves
// its lines through a 32 x 32 shared-memory tile (row segments loaded and
// stored coalesced, transposed in the tile), each lane runs its line's
// recurrence through the tile's columns.  The forward sweep writes y back to
// f, the backward sweep reads it again; no whole line is held on chip, so
// many warps (hence many independent recurrences) fit on an SM.
constexpr int kRowsWarps = 4;

template <typename TW>
__global__ void __launch_bounds__(kRowsWarps * 32) k_solve_rows(TW* __restrict__ f, TW* __restrict__ w, int mline,
                                                                int64_t rows, int64_t row_pitch,
                                                                const TW* __restrict__ ta, const TW* __restrict__ tb,
                                                                int op) {
  // loads of a tile are issued in batches of B before their shared-memory
  // stores (128 bytes of loads in flight per thread)
  constexpr int B = 128 / sizeof(TW);
  __shared__ TW tiles[kRowsWarps][32][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r0 = (int64_t(blockIdx.x) * kRowsWarps + warp) * 32;
  if (r0 >= rows) return;
  const int nr = int(rows - r0 < 32 ? rows - r0 : 32);
  // rows r0 .. r0+nr-1 of mline elements at pitch row_pitch
  if (!MGR_IN((r0 + nr - 1) * row_pitch + mline - 1, rows * row_pitch, kDbgSolveF)) return;
  TW(*tile)[33] = tiles[warp];
  TW* base = f + r0 * row_pitch;
  TW* wb = w + r0 * row_pitch;
  const bool act = lane < nr;
  auto load_tile = [&](int c0) {
#pragma unroll
    for (int i0 = 0; i0 < 32; i0 += B) {
      TW v[B];
#pragma unroll
      for (int u = 0; u < B; ++u) v[u] = (i0 + u < nr) ? base[int64_t(i0 + u) * row_pitch + c0 + lane] : TW(0);
#pragma unroll
      for (int u = 0; u < B; ++u) tile[lane][i0 + u] = v[u];
    }
  };
  TW prev = TW(0);
  for (int c0 = 0; c0 < mline; c0 += 32) {
    const int nc = min(32, mline - c0);
    if (lane < nc) load_tile(c0);
    __syncwarp();
    if (act) {
      for (int c = 0; c < nc; ++c) {
        prev = tile[c][lane] - ta[c0 + c] * prev;
        tile[c][lane] = prev;
      }
    }
    __syncwarp();
    if (lane < nc) {
#pragma unroll 8
      for (int i = 0; i < nr; ++i) base[int64_t(i) * row_pitch + c0 + lane] = tile[lane][i];
    }
    __syncwarp();
  }
  TW next = TW(0);
  for (int c0 = ((mline - 1) / 32) * 32; c0 >= 0; c0 -= 32) {
    const int nc = min(32, mline - c0);
    if (lane < nc) load_tile(c0);
    __syncwarp();
    if (act) {
      for (int c = nc - 1; c >= 0; --c) {
        next = tile[c][lane] - tb[c0 + c] * next;
        tile[c][lane] = next;
      }
    }
    __syncwarp();
    if (lane < nc) {
      if (op == SOLVE_INPLACE) {
#pragma unroll 8
        for (int i = 0; i < nr; ++i) base[int64_t(i) * row_pitch + c0 + lane] = tile[lane][i];
      } else {
        const TW sg = op == SOLVE_ADD ? TW(1) : TW(-1);
#pragma unroll
        for (int i0 = 0; i0 < 32; i0 += B) {
          TW v[B];
#pragma unroll
          for (int u = 0; u < B; ++u) v[u] = (i0 + u < nr) ? wb[int64_t(i0 + u) * row_pitch + c0 + lane] : TW(0);
#pragma unroll
          for (int u = 0; u < B; ++u)
            if (i0 + u < nr) wb[int64_t(i0 + u) * row_pitch + c0 + lane] = v[u] + sg * tile[lane][i0 + u];
        }
      }
    }
    __syncwarp();
  }
}

// Coarsest grid <-> nodal positions (dir 0: gather nodal -> compact; 1: scatter)
template <typename TD, typename TW>
__device__ __forceinline__ void coarsest_copy(TD* y, int64_t y_sz, int64_t y_sy, TW* w, int3 n, longlong3 s,
                                              longlong3 N, int dir, int64_t e0, int64_t estep) {
  const int64_t total = int64_t(n.x) * n.y * n.z;
  for (int64_t e = e0; e < total; e += estep) {
    const int gx = int(e % n.z);
    const int64_t rest = e / n.z;
    const int gy = int(rest % n.y), gz = int(rest / n.y);
    const int64_t yo = fmap(gz, s.x, N.x) * y_sz + fmap(gy, s.y, N.y) * y_sy + fmap(gx, s.z, N.z);
    if (!MGR_IN(yo, N.x * y_sz, kDbgCoarsestY)) continue;
    if (dir == 0) w[e] = TW(y[yo]);
    else y[yo] = TD(w[e]);
  }
}

template <typename TD, typename TW>
__global__ void k_coarsest(TD* y, int64_t y_sz, int64_t y_sy, TW* w, int3 n, longlong3 s, longlong3 N, int dir) {
  coarsest_copy<TD, TW>(y, y_sz, y_sy, w, n, s, N, dir, blockIdx.x * int64_t(blockDim.x) + threadIdx.x,
                        int64_t(gridDim.x) * blockDim.x);
}
