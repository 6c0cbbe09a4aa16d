// mgr_small.cuh -- the coarse end of the hierarchy in one CTA.
//
// Once a level grid fits in shared memory (a few thousand nodes), the tiled
// level pass, the line solves and the interpolation are each latency-bound
// launches that use a handful of SMs.  k_small_dec / k_small_rec run all of
// those levels in a single CTA: the level values, coefficients, the
// intermediate stencil results, the load vector and the coarse values live in
// shared memory, and every step of Sec. II.A is one parallel loop over its
// grid followed by a barrier:
//
//   decompose, level l (n -> m nodes per axis):
//     W = v on the coarse nodes; c = v - (P_0 x P_1 x P_2) W, 0 on coarse nodes
//     (written to the nodal output); f = K_z K_y K_x c (three 5-tap passes);
//     Thomas solves along x, y, z (scaled LU, one FMA per step); W += z.
//   recompose, level l: c from the nodal input, f and z as above, W -= z,
//     v = c + (P_0 x P_1 x P_2) W.
//
// Stencils use the stencil type TS, solves and coarse values the solve type TW
// (the same split as the tiled kernels).  Included inside an anonymous
// namespace after mgr_device.cuh.
#pragma once

constexpr int kSmallMaxLevels = 16;
constexpr int kSmallThreads = 1024;

template <typename TS, typename TW>
struct SmallArgs {
  int levels;  // the small levels are levels..1
  int n[kSmallMaxLevels + 1][3], m[kSmallMaxLevels + 1][3];
  int active[kSmallMaxLevels + 1][3];
  int64_t s[kSmallMaxLevels + 1][3];  // full-grid stride of a level-l node
  int64_t N[3];                       // full-grid lengths
  int64_t s0[3];                      // stride of the coarsest grid
  int n0[3];                          // coarsest grid sizes
  const TS* wa[kSmallMaxLevels + 1][3];
  const TS* wb[kSmallMaxLevels + 1][3];
  const TS* k[kSmallMaxLevels + 1][3];
  const TW* ta[kSmallMaxLevels + 1][3];
  const TW* tb[kSmallMaxLevels + 1][3];
  const void* vin;  // decompose: level-`levels` values (compact TW, or the field when vin_full)
  int vin_full;
  void* vout;       // recompose: level-`levels` values (compact TW, or the field when vout_full)
  int vout_full;
  const void* cin;  // recompose: nodal coefficients
  void* out;        // decompose: nodal output
  int64_t sz, sy;   // full-grid strides (elements) of the nodal arrays
};

template <typename TS, typename TW>
constexpr size_t small_smem_bytes(int n0, int n1, int n2, int m0, int m1, int m2) {
  return sizeof(TW) * (size_t(n0) * n1 * n2 + 2 * size_t(m0) * m1 * m2) +
         sizeof(TS) * (size_t(n0) * n1 * m2 + size_t(n0) * m1 * m2) + 64;
}

// Index arithmetic of the element loops: n / d and n % d for 0 <= n < 2^22 and a
// divisor d >= 1 fixed for the loop, from the single-precision reciprocal of d
// taken once.  float(n) is exact, and fl(n * fl(1/d)) is within a relative
// 2^-23 of n/d, so below 2^22 its truncation q0 is floor(n/d) or one off;
// the remainder n - q0*d says which way and one step corrects it.  (A runtime
// integer division is a long instruction sequence; these loops do a few per
// element.)
struct SmallDiv {
  int d;
  float rd;
  __device__ explicit SmallDiv(int divisor) : d(divisor), rd(1.0f / float(divisor)) {}
  __device__ __forceinline__ int quo(int n) const {
    int q = int(float(n) * rd);
    const int r = n - q * d;
    return q + (r >= d ? 1 : 0) - (r < 0 ? 1 : 0);
  }
  // (q, r) with n = q*d + r, 0 <= r < d
  __device__ __forceinline__ int quo_rem(int n, int& r) const {
    const int q = quo(n);
    r = n - q * d;
    return q;
  }
};

__device__ __forceinline__ int64_t small_full(const int64_t* s, const int64_t* N, int i0, int i1, int i2, int64_t sz,
                                               int64_t sy) {
  return fmap(i0, s[0], N[0]) * sz + fmap(i1, s[1], N[1]) * sy + fmap(i2, s[2], N[2]);
}

// Full-grid element i of a field (N[0] * sz elements): read, and write, checked
// in bounds-checking builds.
template <typename T>
__device__ __forceinline__ T small_ld(const T* p, int64_t i, const int64_t* N, int64_t sz) {
  (void)N;
  (void)sz;
  return MGR_IN(i, N[0] * sz, kDbgSmallIn) ? p[i] : T(0);
}
template <typename T>
__device__ __forceinline__ void small_st(T* p, int64_t i, T v, const int64_t* N, int64_t sz) {
  (void)N;
  (void)sz;
  if (MGR_IN(i, N[0] * sz, kDbgSmallOut)) p[i] = v;
}

// (P_0 x P_1 x P_2) W one axis at a time.  small_interp_rows: A = P_2 W on
// the coarse (q0, q1) rows of the level (m0 x m1 x n2 values, in scratch; the
// caller synchronizes); small_interp_at: the y and then z interpolation of A
// at level node (i0, i1, i2) (a coarse index takes its coarse value, a fine one
// the weighted pair around it).  About 2.6 FMAs a node on average instead of
// up to 16 for the eight-neighbour tensor-product sum.
template <typename TS, typename TW>
__device__ __forceinline__ void small_interp_rows(const TW* W, TS* A, const int* n, const int* m, const TS* wa2,
                                                  const TS* wb2) {
  const int n2 = n[2], m2 = m[2];
  const SmallDiv dn2(n2);
  for (int e = threadIdx.x; e < m[0] * m[1] * n2; e += blockDim.x) {
    int i2;
    const int q01 = dn2.quo_rem(e, i2);
    const TW* row = W + int64_t(q01) * m2;
    A[e] = is_coarse(i2, n2) ? TS(row[cidx(i2)])
                             : wa2[i2] * TS(row[cidx(i2 - 1)]) + wb2[i2] * TS(row[cidx(i2 + 1)]);
  }
}
template <typename TS>
__device__ __forceinline__ TS small_interp_at(const TS* A, const int* n, const int* m, const TS* const* wa,
                                              const TS* const* wb, int i0, int i1, int i2) {
  const int n2 = n[2], m1 = m[1];
  // the y interpolant on coarse plane q0
  auto plane = [&](int q0) -> TS {
    const TS* a = A + int64_t(q0) * m1 * n2 + i2;
    if (is_coarse(i1, n[1])) return a[int64_t(cidx(i1)) * n2];
    return wa[1][i1] * a[int64_t(cidx(i1 - 1)) * n2] + wb[1][i1] * a[int64_t(cidx(i1 + 1)) * n2];
  };
  if (is_coarse(i0, n[0])) return plane(cidx(i0));
  return wa[0][i0] * plane(cidx(i0 - 1)) + wb[0][i0] * plane(cidx(i0 + 1));
}

// f = K_0 K_1 K_2 c on the level's grids: c (n0 n1 n2, TW) -> t1 (n0 n1 m2)
// -> t2 (n0 m1 m2) -> f (m0 m1 m2, TW).
template <typename TS, typename TW>
__device__ __forceinline__ void small_load_vector(const TW* c, TS* t1, TS* t2, TW* f, const int* n, const int* m,
                                                  const TS* const* K) {
  const int n0 = n[0], n1 = n[1], n2 = n[2], m0 = m[0], m1 = m[1], m2 = m[2];
  const SmallDiv dm2(m2), dm1(m1), dm12(m1 * m2);
  for (int e = threadIdx.x; e < n0 * n1 * m2; e += blockDim.x) {
    int q;
    const int r = dm2.quo_rem(e, q);
    const int p = pidx(q, n2);
    TS acc = TS(0);
    for (int o = 0; o < 5; ++o) {
      const int j = p + o - 2;
      if (j >= 0 && j < n2) acc += K[2][5 * q + o] * TS(c[int64_t(r) * n2 + j]);
    }
    t1[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n0 * m1 * m2; e += blockDim.x) {
    int x, q;
    const int i0 = dm1.quo_rem(dm2.quo_rem(e, x), q);
    const int p = pidx(q, n1);
    TS acc = TS(0);
    for (int o = 0; o < 5; ++o) {
      const int j = p + o - 2;
      if (j >= 0 && j < n1) acc += K[1][5 * q + o] * t1[(int64_t(i0) * n1 + j) * m2 + x];
    }
    t2[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m0 * m1 * m2; e += blockDim.x) {
    int yx;
    const int q = dm12.quo_rem(e, yx);
    const int p = pidx(q, n0);
    TS acc = TS(0);
    for (int o = 0; o < 5; ++o) {
      const int j = p + o - 2;
      if (j >= 0 && j < n0) acc += K[0][5 * q + o] * t2[int64_t(j) * m1 * m2 + yx];
    }
    f[e] = TW(acc);
  }
  __syncthreads();
}

// Thomas solves of (x_k M_k) z = f in place along every active axis (x, y, z).
template <typename TW>
__device__ __forceinline__ void small_solves(TW* f, const int* m, const int* active, const TW* const* ta,
                                             const TW* const* tb) {
  const int m0 = m[0], m1 = m[1], m2 = m[2];
  for (int axis = 2; axis >= 0; --axis) {
    if (!active[axis]) continue;
    const int len = m[axis];
    const int lines = m0 * m1 * m2 / len;
    const int stride = axis == 2 ? 1 : (axis == 1 ? m2 : m1 * m2);
    const SmallDiv dm2(m2);
    for (int li = threadIdx.x; li < lines; li += blockDim.x) {
      int base;
      if (axis == 2) {
        base = li * m2;
      } else if (axis == 1) {
        int x;
        base = dm2.quo_rem(li, x) * m1 * m2 + x;
      } else {
        base = li;
      }
      TW prev = TW(0);
      for (int q = 0; q < len; ++q) {
        prev = f[base + q * stride] - ta[axis][q] * prev;
        f[base + q * stride] = prev;
      }
      TW next = TW(0);
      for (int q = len - 1; q >= 0; --q) {
        next = f[base + q * stride] - tb[axis][q] * next;
        f[base + q * stride] = next;
      }
    }
    __syncthreads();
  }
}

// One field's coarse levels, decomposition: the body of k_small_dec and of
// the batched one-CTA phase (smem_raw: small_smem_bytes of level a.levels).
template <typename TD, typename TS, typename TW>
__device__ __forceinline__ void small_dec_body(const SmallArgs<TS, TW>& a, unsigned char* smem_raw) {
  const int ls = a.levels;
  const int64_t nv = int64_t(a.n[ls][0]) * a.n[ls][1] * a.n[ls][2];
  const int64_t mv = int64_t(a.m[ls][0]) * a.m[ls][1] * a.m[ls][2];
  TW* V = reinterpret_cast<TW*>(smem_raw);
  TW* W = V + nv;
  TW* F = W + mv;
  TS* T1 = reinterpret_cast<TS*>(F + mv);
  TS* T2 = T1 + int64_t(a.n[ls][0]) * a.n[ls][1] * a.m[ls][2];
  TD* out = static_cast<TD*>(a.out);
  // level-ls values
  {
    const SmallDiv dn1(a.n[ls][1]), dn2(a.n[ls][2]);
    for (int e = threadIdx.x; e < int(nv); e += blockDim.x) {
      if (a.vin_full) {
        int i1, i2;
        const int i0 = dn1.quo_rem(dn2.quo_rem(e, i2), i1);
        V[e] = TW(small_ld(static_cast<const TD*>(a.vin), small_full(a.s[ls], a.N, i0, i1, i2, a.sz, a.sy), a.N, a.sz));
      } else {
        V[e] = static_cast<const TW*>(a.vin)[e];
      }
    }
  }
  __syncthreads();
  for (int l = ls; l >= 1; --l) {
    const int* n = a.n[l];
    const int* m = a.m[l];
    const int ln = n[0] * n[1] * n[2], lm = m[0] * m[1] * m[2];
    const SmallDiv dn1(n[1]), dn2(n[2]), dm1(m[1]), dm2(m[2]);
    // coarse values
    for (int e = threadIdx.x; e < lm; e += blockDim.x) {
      int q1, q2;
      const int q0 = dm1.quo_rem(dm2.quo_rem(e, q2), q1);
      W[e] = V[(int64_t(pidx(q0, n[0])) * n[1] + pidx(q1, n[1])) * n[2] + pidx(q2, n[2])];
    }
    __syncthreads();
    // x interpolants of the coarse rows (scratch: the stencil buffers T1, T2,
    // free until the load vector; m0 m1 n2 <= n0 m2 (n1 + m1) values fit)
    small_interp_rows<TS, TW>(W, T1, n, m, a.wa[l][2], a.wb[l][2]);
    __syncthreads();
    // coefficients (in place), written to their nodal positions
    for (int e = threadIdx.x; e < ln; e += blockDim.x) {
      int i1, i2;
      const int i0 = dn1.quo_rem(dn2.quo_rem(e, i2), i1);
      if (is_coarse(i0, n[0]) && is_coarse(i1, n[1]) && is_coarse(i2, n[2])) {
        V[e] = TW(0);
        continue;
      }
      const TS c = TS(V[e]) - small_interp_at<TS>(T1, n, m, a.wa[l], a.wb[l], i0, i1, i2);
      V[e] = TW(c);
      small_st(out, small_full(a.s[l], a.N, i0, i1, i2, a.sz, a.sy), TD(c), a.N, a.sz);
    }
    __syncthreads();
    small_load_vector<TS, TW>(V, T1, T2, F, n, m, a.k[l]);
    small_solves<TW>(F, m, a.active[l], a.ta[l], a.tb[l]);
    // correction (Eq. (1)), and the corrected coarse values become the next level
    for (int e = threadIdx.x; e < lm; e += blockDim.x) V[e] = W[e] + F[e];
    __syncthreads();
  }
  // coarsest values
  const int c0 = a.n0[0], c1 = a.n0[1], c2 = a.n0[2];
  const SmallDiv dc1(c1), dc2(c2);
  for (int e = threadIdx.x; e < c0 * c1 * c2; e += blockDim.x) {
    int i1, i2;
    const int i0 = dc1.quo_rem(dc2.quo_rem(e, i2), i1);
    small_st(out, small_full(a.s0, a.N, i0, i1, i2, a.sz, a.sy), TD(V[e]), a.N, a.sz);
  }
}

template <typename TD, typename TS, typename TW>
__global__ void __launch_bounds__(kSmallThreads, 1) k_small_dec(const SmallArgs<TS, TW> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  small_dec_body<TD, TS, TW>(a, smem_raw);
}

// One field's coarse levels, recomposition (see small_dec_body).
template <typename TD, typename TS, typename TW>
__device__ __forceinline__ void small_rec_body(const SmallArgs<TS, TW>& a, unsigned char* smem_raw) {
  const int ls = a.levels;
  const int64_t nv = int64_t(a.n[ls][0]) * a.n[ls][1] * a.n[ls][2];
  const int64_t mv = int64_t(a.m[ls][0]) * a.m[ls][1] * a.m[ls][2];
  TW* V = reinterpret_cast<TW*>(smem_raw);
  TW* W = V + nv;
  TW* F = W + mv;
  TS* T1 = reinterpret_cast<TS*>(F + mv);
  TS* T2 = T1 + int64_t(a.n[ls][0]) * a.n[ls][1] * a.m[ls][2];
  const TD* cin = static_cast<const TD*>(a.cin);
  // coarsest values
  {
    const int c0 = a.n0[0], c1 = a.n0[1], c2 = a.n0[2];
    const SmallDiv dc1(c1), dc2(c2);
    for (int e = threadIdx.x; e < c0 * c1 * c2; e += blockDim.x) {
      int i1, i2;
      const int i0 = dc1.quo_rem(dc2.quo_rem(e, i2), i1);
      W[e] = TW(small_ld(cin, small_full(a.s0, a.N, i0, i1, i2, a.sz, a.sy), a.N, a.sz));
    }
  }
  __syncthreads();
  for (int l = 1; l <= ls; ++l) {
    const int* n = a.n[l];
    const int* m = a.m[l];
    const int ln = n[0] * n[1] * n[2], lm = m[0] * m[1] * m[2];
    const SmallDiv dn1(n[1]), dn2(n[2]);
    // this level's coefficients (0 on the coarse nodes)
    for (int e = threadIdx.x; e < ln; e += blockDim.x) {
      int i1, i2;
      const int i0 = dn1.quo_rem(dn2.quo_rem(e, i2), i1);
      const bool coarse = is_coarse(i0, n[0]) && is_coarse(i1, n[1]) && is_coarse(i2, n[2]);
      V[e] = coarse ? TW(0) : TW(small_ld(cin, small_full(a.s[l], a.N, i0, i1, i2, a.sz, a.sy), a.N, a.sz));
    }
    __syncthreads();
    small_load_vector<TS, TW>(V, T1, T2, F, n, m, a.k[l]);
    small_solves<TW>(F, m, a.active[l], a.ta[l], a.tb[l]);
    for (int e = threadIdx.x; e < lm; e += blockDim.x) W[e] -= F[e];
    __syncthreads();
    // level values: coefficients plus the interpolant of the coarse values
    // (x interpolants of the coarse rows first, in the stencil buffers)
    small_interp_rows<TS, TW>(W, T1, n, m, a.wa[l][2], a.wb[l][2]);
    __syncthreads();
    for (int e = threadIdx.x; e < ln; e += blockDim.x) {
      int i1, i2;
      const int i0 = dn1.quo_rem(dn2.quo_rem(e, i2), i1);
      if (is_coarse(i0, n[0]) && is_coarse(i1, n[1]) && is_coarse(i2, n[2])) {
        V[e] = W[(int64_t(cidx(i0)) * m[1] + cidx(i1)) * m[2] + cidx(i2)];
      } else {
        V[e] = TW(TS(V[e]) + small_interp_at<TS>(T1, n, m, a.wa[l], a.wb[l], i0, i1, i2));
      }
    }
    __syncthreads();
    if (l < ls) {
      for (int e = threadIdx.x; e < ln; e += blockDim.x) W[e] = V[e];
      __syncthreads();
    }
  }
  // level-ls values
  const SmallDiv dn1(a.n[ls][1]), dn2(a.n[ls][2]);
  for (int e = threadIdx.x; e < int(nv); e += blockDim.x) {
    if (a.vout_full) {
      int i1, i2;
      const int i0 = dn1.quo_rem(dn2.quo_rem(e, i2), i1);
      small_st(static_cast<TD*>(a.vout), small_full(a.s[ls], a.N, i0, i1, i2, a.sz, a.sy), TD(V[e]), a.N, a.sz);
    } else {
      static_cast<TW*>(a.vout)[e] = V[e];
    }
  }
}

template <typename TD, typename TS, typename TW>
__global__ void __launch_bounds__(kSmallThreads, 1) k_small_rec(const SmallArgs<TS, TW> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  small_rec_body<TD, TS, TW>(a, smem_raw);
}
