// mgr_plan.cpp -- host-side plan construction (FP64).
//
// For every level l = L..1 and every axis this builds, from the axis
// coordinates (arXiv 2105.12764, Sec. III.A.2 "r_i = h_i/(h_i+h_{i+1})"):
//   * the interpolation weights of the fine nodes (Sec. II.A.1, Fig.
//     example-1d; the FMA form of Table "fma" uses the right-neighbour weight
//     r, we keep both weights so no 1-r cancellation happens on stretched grids);
//   * the mass-transfer stencil K = P^T M (Sec. III.A.2; the paper prints K
//     with a garbled diagonal entry, so K is formed here as the product P^T M
//     of the interpolation and the P1 mass matrix, five taps per coarse node);
//   * the LU factors of the coarse mass matrix M_{l-1} for the Thomas solves
//     (Sec. III.A.3; Table "fma" rows "Solv. Corr.": precomputed diag/subdiag).
// The diagonal of U is folded into K (row q scaled by 1/u_q), so each solve
// step on the device is one fused multiply-add:
//     forward   y_q = f'_q - ta_q * y_{q-1},   ta_q = e_{q-1} / u_q
//     backward  z_q = y_q  - tb_q * z_{q+1},   tb_q = e_q / u_q
// where e_q = h_q / 6 is the off-diagonal of M_{l-1}.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "mgr_internal.h"

namespace mgr {
namespace {

int64_t coarse_len(int64_t n) { return n / 2 + 1; }  // even positions plus the last one

int levels_until(int64_t n, int64_t stop) {
  int L = 0;
  while (n > stop) {
    n = coarse_len(n);
    ++L;
  }
  return L;
}

}  // namespace

int resolve_levels(const mgr_desc* d, int* levels, int* max_levels, int* default_levels) {
  if (!d || d->ndim < 1 || d->ndim > 4) return MGR_EINVAL;
  int mx = 1 << 30, df = 1 << 30;
  for (int k = 0; k < d->ndim; ++k) {
    if (d->shape[k] < 2 || d->shape[k] > (int64_t(1) << 30)) return MGR_EINVAL;
    mx = std::min(mx, levels_until(d->shape[k], 2));
    df = std::min(df, levels_until(d->shape[k], 3));
  }
  // the kernels address within a plane of the two fastest axes (and, for 4D,
  // within a time slice) with 32-bit offsets
  const int64_t plane = d->ndim >= 2 ? d->shape[d->ndim - 1] * d->shape[d->ndim - 2] : d->shape[0];
  if (plane >= (int64_t(1) << 31)) return MGR_EINVAL;
  if (d->ndim == 4 && d->shape[1] * plane >= (int64_t(1) << 31)) return MGR_EINVAL;
  if (max_levels) *max_levels = mx;
  if (default_levels) *default_levels = df;
  if (levels) {
    int L = d->levels < 0 ? df : d->levels;
    if (L > mx || L > kMaxLevels) return MGR_EINVAL;
    *levels = L;
  }
  return MGR_OK;
}

int build_plan_tables(mgr_plan* p) {
  const mgr_desc& d = p->desc;
  const int L = p->levels;
  // full-grid coordinates per internal axis (axis kAxes-1 = fastest); entry
  // kAxes is the time axis of a 4D field (desc axis 0)
  const bool st = d.ndim == 4;
  const int nsp = st ? 3 : d.ndim;  // spatial dimensions
  const int lead = kAxes - nsp;
  std::vector<double> xs[kAxes + 1];
  auto load_axis = [&](int k, std::vector<double>& x) {
    const int64_t N = d.shape[k];
    x.resize(N);
    for (int64_t i = 0; i < N; ++i) x[i] = d.coords[k] ? d.coords[k][i] : double(i);
    for (int64_t i = 1; i < N; ++i)
      if (!(x[i] > x[i - 1]) || !std::isfinite(x[i])) return false;
    return std::isfinite(x[0]);
  };
  for (int a = 0; a < kAxes; ++a) {
    if (a < lead) {
      p->full[a] = 1;
      xs[a].assign(1, 0.0);
      continue;
    }
    const int k = a - lead + (st ? 1 : 0);
    p->full[a] = d.shape[k];
    if (!load_axis(k, xs[a])) return MGR_EINVAL;
  }
  p->full_t = st ? d.shape[0] : 1;
  if (st) {
    if (!load_axis(0, xs[kAxes])) return MGR_EINVAL;
  } else {
    xs[kAxes].assign(1, 0.0);
  }
  std::vector<double>& T = p->tables.host;
  T.clear();
  p->geom.assign(L + 1, LevelGeom{});
  auto axref = [&](int l, int a) -> AxisLevel& { return a < kAxes ? p->geom[l].ax[a] : p->geom[l].tax; };
  // level sizes per axis: n_L = N, n_{l-1} = n_l/2 + 1
  for (int a = 0; a <= kAxes; ++a) {
    const int64_t full = a < kAxes ? p->full[a] : p->full_t;
    const bool inactive = a < kAxes ? a < lead : !st;
    int64_t n = full;
    for (int l = L; l >= 1; --l) {
      AxisLevel& ax = axref(l, a);
      ax.N = full;
      ax.s = int64_t(1) << (L - l);
      ax.n = int(n);
      if (inactive) {
        ax.m = 1;
        ax.active = false;
      } else {
        ax.m = int(coarse_len(n));
        ax.active = true;
        n = ax.m;
      }
    }
    if (a < kAxes) p->coarsest[a] = n;
    else p->coarsest_t = n;
  }
  // class sizes: the coarsest grid, then |N_l| - |N_{l-1}| per level
  p->class_off.assign(L + 2, 0);
  p->class_off[1] = p->coarsest[0] * p->coarsest[1] * p->coarsest[2] * p->coarsest_t;
  for (int l = 1; l <= L; ++l)
    p->class_off[l + 1] = p->class_off[l] + p->geom[l].fine_count() - p->geom[l].coarse_count();
  auto push = [&](size_t count) {
    int64_t off = int64_t(T.size());
    // keep every table 16-byte aligned in both FP64 and FP32 copies
    size_t padded = (count + 3) & ~size_t(3);
    T.resize(T.size() + padded, 0.0);
    return off;
  };
  for (int l = L; l >= 1; --l) {
    for (int a = 0; a <= kAxes; ++a) {
      AxisLevel& ax = axref(l, a);
      const int n = ax.n, m = ax.m;
      ax.o_wa = push(n);
      ax.o_wb = push(n);
      ax.o_k = push(size_t(5) * m);
      ax.o_ta = push(m);
      ax.o_tb = push(m);
      if (!ax.active) {
        // identity stencil, no solve
        T[ax.o_k + 2] = 1.0;
        continue;
      }
      // level-l coordinates
      std::vector<double> x(n);
      for (int i = 0; i < n; ++i) x[i] = xs[a][std::min<int64_t>(int64_t(i) * ax.s, ax.N - 1)];
      auto pidx = [&](int q) { return std::min(2 * q, n - 1); };
      auto coarse = [&](int i) { return (i % 2 == 0) || (i == n - 1); };
      // interpolation weights of fine nodes (neighbours i-1 and i+1 are coarse)
      for (int i = 0; i < n; ++i) {
        if (coarse(i)) continue;
        const double xa = x[i - 1], xb = x[i + 1], xj = x[i];
        T[ax.o_wa + i] = (xb - xj) / (xb - xa);
        T[ax.o_wb + i] = (xj - xa) / (xb - xa);
      }
      // P1 mass matrix on level l: sub ml, diag md, super mu
      std::vector<double> ml(n), md(n), mu(n);
      for (int j = 0; j < n; ++j) {
        const double hl = j > 0 ? x[j] - x[j - 1] : 0.0;
        const double hr = j < n - 1 ? x[j + 1] - x[j] : 0.0;
        md[j] = (hl + hr) / 3.0;
        ml[j] = hl / 6.0;
        mu[j] = hr / 6.0;
      }
      // K = P^T M, row q stored at taps (j - pidx(q) + 2)
      std::vector<double> K(size_t(5) * m, 0.0);
      auto addK = [&](int q, int j, double v) {
        const int t = j - pidx(q) + 2;
        if (t < 0 || t > 4) return false;
        K[size_t(5) * q + t] += v;
        return true;
      };
      for (int i = 0; i < n; ++i) {
        int qs[2];
        double ws[2];
        int cnt;
        if (coarse(i)) {
          qs[0] = (i + 1) / 2;
          ws[0] = 1.0;
          cnt = 1;
        } else {
          qs[0] = (i - 1) / 2;  // coarse index of i-1 (even)
          ws[0] = T[ax.o_wa + i];
          qs[1] = (i + 1) / 2;  // coarse index of i+1 (even, at most n-1)
          ws[1] = T[ax.o_wb + i];
          cnt = 2;
        }
        for (int c = 0; c < cnt; ++c) {
          if (i > 0 && !addK(qs[c], i - 1, ws[c] * ml[i])) return MGR_EINVAL;
          if (!addK(qs[c], i, ws[c] * md[i])) return MGR_EINVAL;
          if (i < n - 1 && !addK(qs[c], i + 1, ws[c] * mu[i])) return MGR_EINVAL;
        }
      }
      // coarse mass matrix M_{l-1} and its LU factors
      std::vector<double> xc(m), cd(m), ce(m), u(m);
      for (int q = 0; q < m; ++q) xc[q] = x[pidx(q)];
      for (int q = 0; q < m; ++q) {
        const double hl = q > 0 ? xc[q] - xc[q - 1] : 0.0;
        const double hr = q < m - 1 ? xc[q + 1] - xc[q] : 0.0;
        cd[q] = (hl + hr) / 3.0;
        ce[q] = hr / 6.0;
      }
      u[0] = cd[0];
      for (int q = 1; q < m; ++q) u[q] = cd[q] - (ce[q - 1] / u[q - 1]) * ce[q - 1];
      for (int q = 0; q < m; ++q) {
        const double inv = 1.0 / u[q];
        for (int t = 0; t < 5; ++t) T[ax.o_k + 5 * q + t] = K[size_t(5) * q + t] * inv;
        T[ax.o_ta + q] = q > 0 ? ce[q - 1] * inv : 0.0;
        T[ax.o_tb + q] = q < m - 1 ? ce[q] * inv : 0.0;
      }
    }
  }
  return MGR_OK;
}

}  // namespace mgr

// ---------------------------------------------------------------------------
// Algorithmic work per launch (reported by mgr_profile).
//
// Flop counts are those of the minimal arithmetic of each step, counting a
// fused multiply-add as 2 flops:
//   coefficients / interpolant, separable form: a node whose slowest fine axis
//     is k costs 3 FMA (interpolate along k, keep that value for the slower
//     axes, subtract) or 2 FMA when k is the slowest active axis;
//   mass-transfer along x: 5 taps per coarse output, 2 on lines whose other
//     coordinates are all coarse (the coefficients vanish on coarse nodes);
//   along y and z: 5 taps per output; solves: 2 FMA per coarse node and axis.
// Bytes are the compulsory traffic of each launch's inputs and outputs.
// ---------------------------------------------------------------------------
namespace mgr {
namespace {

double coef_fma(const LevelGeom& g) {
  int slowest = -1;
  for (int k = 0; k < kAxes; ++k)
    if (g.ax[k].active) { slowest = k; break; }
  double total = 0;
  for (int k = 0; k < kAxes; ++k) {
    if (!g.ax[k].active) continue;
    // nodes whose slowest fine axis is k: coarse on slower axes (j < k),
    // fine on k, anything on faster axes (j > k)
    double cnt = double(g.ax[k].n - g.ax[k].m);
    for (int j = 0; j < k; ++j) cnt *= g.ax[j].m;
    for (int j = k + 1; j < kAxes; ++j) cnt *= g.ax[j].n;
    total += cnt * (k == slowest ? 2.0 : 3.0);
  }
  return total;
}

double stencil_fma(const LevelGeom& g) {
  const AxisLevel &z = g.ax[0], &y = g.ax[1], &x = g.ax[2];
  double t = 0;
  if (x.active) {
    const double lines_coarse = double(z.m) * y.m;
    const double lines_all = double(z.n) * y.n;
    t += x.m * (2.0 * lines_coarse + 5.0 * (lines_all - lines_coarse));
  }
  if (y.active) t += 5.0 * double(z.n) * y.m * x.m;
  if (z.active) t += 5.0 * double(z.m) * y.m * x.m;
  return t;
}

}  // namespace

Work work_level_load(const mgr_plan* p, int l, bool decompose) {
  const LevelGeom& g = p->geom[l];
  const double n = double(g.fine_count()), m = double(g.coarse_count());
  const double sd = double(p->elem), sw = double(p->welem);
  Work w;
  if (decompose) {
    const double sin = (l == p->levels) ? sd : sw;
    w.bytes = n * sin + (n - m) * sd + 2.0 * m * sw;
    w.flops = 2.0 * (coef_fma(g) + stencil_fma(g));
  } else {
    w.bytes = n * sd + m * sw;
    w.flops = 2.0 * stencil_fma(g);
  }
  return w;
}

Work work_solve(const mgr_plan* p, int l, int axis, bool final_op) {
  (void)axis;
  const double m = double(p->geom[l].coarse_count());
  const double sw = double(p->welem);
  Work w;
  w.bytes = 2.0 * m * sw + (final_op ? 2.0 * m * sw : 0.0);
  w.flops = 4.0 * m + (final_op ? m : 0.0);
  return w;
}

// ---------------------------------------------------------------------------
// Quantization bins (the quantization stage around the refactoring, Sec. V).
// A perturbation d_l of the level-l coefficients reaches the recomposed field
// through e_l = d_l + P_l (e_{l-1} - Z_l d_l), Z_l = (x_k M_{l-1,k})^-1 (x_k K_k),
// |P_l|_inf = 1, so |e_L|_inf <= |d_0| + sum_l (1 + |Z_l|_inf) |d_l|; with
// rounding, |d_l| <= q_l/2, and tau split evenly over the L+1 classes:
// q_0 = 2 tau/(L+1), q_l = 2 tau/((L+1)(1 + |Z_l|_inf)).  |Z_l|_inf is the
// product over axes of the 1D norms, each evaluated exactly, column by
// column, with this plan's scaled K rows and Thomas recurrences.
// ---------------------------------------------------------------------------
namespace {

double correction_norm(const mgr_plan* p, int l, int a) {
  const AxisLevel& ax = p->geom[l].ax[a];
  if (!ax.active) return 1.0;
  const int n = ax.n, m = ax.m;
  const double* T = p->tables.host.data();
  const double* K = T + ax.o_k;
  const double* ta = T + ax.o_ta;
  const double* tb = T + ax.o_tb;
  std::vector<double> z(m), rows(m, 0.0);
  for (int j = 0; j < n; ++j) {
    std::fill(z.begin(), z.end(), 0.0);
    for (int q = std::max(0, j / 2 - 2); q <= std::min(m - 1, j / 2 + 2); ++q) {
      const int t = j - std::min(2 * q, n - 1) + 2;
      if (t >= 0 && t <= 4) z[q] = K[5 * q + t];
    }
    for (int q = 1; q < m; ++q) z[q] -= ta[q] * z[q - 1];
    for (int q = m - 2; q >= 0; --q) z[q] -= tb[q] * z[q + 1];
    for (int q = 0; q < m; ++q) rows[q] += std::fabs(z[q]);
  }
  return *std::max_element(rows.begin(), rows.end());
}

}  // namespace

int quant_bins(mgr_plan* p, double tau, std::vector<double>& bins) {
  if (!(tau > 0.0) || !std::isfinite(tau)) return MGR_EINVAL;
  const int L = p->levels;
  {
    std::lock_guard<std::mutex> lk(p->quant_mu);
    if (int(p->znorm.size()) != L + 1) {
      std::vector<double> zn(L + 1, 0.0);
      for (int l = 1; l <= L; ++l) {
        double v = 1.0;
        for (int a = 0; a < kAxes; ++a) v *= correction_norm(p, l, a);
        zn[l] = v;
      }
      p->znorm = zn;
    }
  }
  bins.assign(L + 1, 0.0);
  bins[0] = 2.0 * tau / (L + 1);
  for (int l = 1; l <= L; ++l) bins[l] = 2.0 * tau / ((L + 1) * (1.0 + p->znorm[l]));
  return MGR_OK;
}

Work work_interp(const mgr_plan* p, int l) {
  const LevelGeom& g = p->geom[l];
  const double n = double(g.fine_count()), m = double(g.coarse_count());
  const double sd = double(p->elem), sw = double(p->welem);
  Work w;
  w.bytes = n * sd + m * sw + n * (l == p->levels ? sd : sw);
  w.flops = 2.0 * coef_fma(g);
  return w;
}

}  // namespace mgr
