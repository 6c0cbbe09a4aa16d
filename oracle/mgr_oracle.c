/*
 * mgr_oracle.c -- plain, slow, FP64 CPU oracle for multigrid hierarchical
 * decomposition and recomposition of a structured-grid field
 * (arXiv 2105.12764, Section II.A "Theory of multigrid-based hierarchical
 * data refactoring", Eq. (1) and Eq. (2)).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library (the CUDA path, its
 * C ABI or its Python binding) may include, link, import or call this file.
 * It is used by the tests, by __graft_entry__.smoke() and by the CPU
 * baseline leg of bench.py.  It shares no code, header, table or constant
 * with the GPU path.
 *
 * What it computes, step by step, in the order of Section II.A:
 *
 *   Hierarchy (per dimension k).  The finest level list is 0..n_k-1.  The next
 *   coarser list keeps every other entry of the current list starting at the
 *   first one, plus the last entry if it was skipped (the paper's dyadic
 *   2^L+1 hierarchy when n_k = 2^L+1; Section IV.A mentions other sizes only
 *   as a pre/post-processing step, so this keep-last nesting is our reading).
 *   The default depth (levels = -1) stops when the smallest dimension reaches
 *   3 nodes; an explicit depth may go on until it reaches 2 nodes, as in the
 *   two-level 5-node example of Fig. example-1d.
 *
 *   Decompose, for l = L..1 (Section II.A.1, II.A.2, Eq. (1)):
 *     v   := nodal values of Q_l u on N_l (v = u at l = L)
 *     c   := v - (P_0 x ... x P_{d-1}) v|N_{l-1}     coefficients, Sec. II.A.1;
 *                                                 exactly 0 on N_{l-1}
 *     f   := (K_0 x ... x K_{d-1}) c,  K_k = P_k^T M_k   load vector, Sec. II.A.2
 *            (the paper's f_{l-1} = R_l M_l vec(C_l) with R_l = P^T)
 *     z   := solve (M^c_0 x ... x M^c_{d-1}) z = f   Thomas algorithm along
 *            each dimension (Sec. III.A.3), dimensions processed last-first
 *            ("rows then columns", Sec. II.A)
 *     v   := v|N_{l-1} + z                        Eq. (1): Q_{l-1}u
 *   The coefficients of level l are stored at the nodes of N_l \ N_{l-1}
 *   (nodal layout: same shape as the input); at the end the coarsest nodal
 *   values are stored at the nodes of N_0.
 *
 *   Recompose, for l = 1..L: the same traversal in reverse (Sec. II.A,
 *   "Overall decomposition/recomposition process"): z from the level-l
 *   coefficients as above, v|N_{l-1} := v - z, then
 *   v := c + (P_0 x ... x P_{d-1}) v|N_{l-1}.
 *
 * Building blocks (1D, on the coordinates x_0 < ... < x_{n-1} of one level):
 *   P (n x m)  piecewise-linear interpolation from the coarse nodes: a coarse
 *              node copies its value; a fine node j between coarse a < j < b
 *              takes (x_b-x_j)/(x_b-x_a) of a and (x_j-x_a)/(x_b-x_a) of b.
 *   M (n x n)  P1 mass matrix (Gram matrix of the hat functions):
 *              M_jj = (h_{j-1}+h_j)/3, M_{j,j+1} = h_j/6, h_j = x_{j+1}-x_j,
 *              missing spacings at the two ends count as 0.  (The paper prints
 *              six times this matrix with shifted indices, Sec. III.A.2; a
 *              common scale cancels between M_l and M_{l-1}.)
 *   K (m x n)  K = P^T M, formed numerically (Sec. III.A.2 "mass-trans").
 *   M^c        the mass matrix built the same way on the coarse coordinates.
 *
 *   Coefficient classes (Sec. I): class 0 = nodal values on N_0, class l =
 *   coefficients on N_l \ N_{l-1}; the class-packed layout concatenates them,
 *   coarsest first, each in row-major order of its level grid.  Recomposing
 *   from a prefix of the classes treats the dropped classes as zero.
 *
 * Pins (checked by the -m "not gpu" tests): the worked 1D example of
 * Fig. example-1d; dense L2 projection Q_l u = (Phi^T G Phi)^-1 ... solved
 * densely with exact quadrature on tiny 1D/2D/3D grids; closed-form mass
 * entries; the uniform K row; zero coefficients for multilinear fields; the
 * quadratic closed form; linearity; separability; round trip.
 *
 * Error returns: 0 on success, -1 on invalid arguments, -2 when memory
 * cannot be allocated.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAXDIM 4

/* ------------------------------------------------------------------ */
/* Hierarchy: level index lists (keep-last rule)                        */
/* ------------------------------------------------------------------ */

/* Is position i of a level list of length n kept in the next coarser list? */
static int is_coarse(int64_t i, int64_t n) { return (i % 2 == 0) || (i == n - 1); }

static int64_t coarse_count(int64_t n) {
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i)
    if (is_coarse(i, n)) ++m;
  return m;
}

/* Number of coarsenings of a list of n nodes until it has `stop` nodes. */
static int levels_until(int64_t n, int64_t stop) {
  int L = 0;
  while (n > stop) {
    n = coarse_count(n);
    ++L;
  }
  return L;
}

int oracle_max_levels_1d(int64_t n) { return levels_until(n, 2); }
int oracle_default_levels_1d(int64_t n) { return levels_until(n, 3); }

static int min_over_dims(int ndim, const int64_t* shape, int64_t stop) {
  if (ndim < 1 || ndim > ORACLE_MAXDIM) return -1;
  int L = 1 << 30;
  for (int k = 0; k < ndim; ++k) {
    if (shape[k] < 2) return -1;
    int lk = levels_until(shape[k], stop);
    if (lk < L) L = lk;
  }
  return L;
}

/* Deepest hierarchy allowed: the smallest dimension reaches 2 nodes (the
   two-node coarsest grid of Fig. example-1d). */
int oracle_max_levels(int ndim, const int64_t* shape) { return min_over_dims(ndim, shape, 2); }

/* Default depth (levels = -1): the smallest dimension reaches 3 nodes. */
int oracle_default_levels(int ndim, const int64_t* shape) { return min_over_dims(ndim, shape, 3); }

/* ------------------------------------------------------------------ */
/* 1D operators on one level                                            */
/* ------------------------------------------------------------------ */

typedef struct {
  int64_t n, m;       /* fine (level l) and coarse (level l-1) sizes          */
  double* x;          /* level-l coordinates, length n                        */
  double* xc;         /* level-(l-1) coordinates, length m                    */
  int64_t* cidx;      /* for a coarse position i: its index in the coarse list;
                         -1 for a fine position                               */
  /* interpolation P: row i has (p0, w0) and optionally (p1, w1)             */
  int64_t* p0; int64_t* p1; double* w0; double* w1; int* nnz;
  /* K = P^T M stored dense (m x n) plus the nonzero column band of each row */
  double* K; int64_t* klo; int64_t* khi;
  /* coarse mass matrix M^c: sub, diag, super (length m)                     */
  double* ma; double* mb; double* mc;
} level1d;

static void level1d_free(level1d* o) {
  free(o->x); free(o->xc); free(o->cidx); free(o->p0); free(o->p1); free(o->w0); free(o->w1);
  free(o->nnz); free(o->K); free(o->klo); free(o->khi); free(o->ma); free(o->mb); free(o->mc);
  memset(o, 0, sizeof(*o));
}

/* P1 mass matrix on coordinates x[0..n): sub a, diag b, super c. */
static void mass_matrix(int64_t n, const double* x, double* a, double* b, double* c) {
  for (int64_t j = 0; j < n; ++j) {
    double hl = (j > 0) ? x[j] - x[j - 1] : 0.0;
    double hr = (j < n - 1) ? x[j + 1] - x[j] : 0.0;
    b[j] = (hl + hr) / 3.0;
    a[j] = hl / 6.0;
    c[j] = hr / 6.0;
  }
}

void oracle_mass_1d(int64_t n, const double* x, double* sub, double* diag, double* super) {
  mass_matrix(n, x, sub, diag, super);
}

static int level1d_build(level1d* o, int64_t n, const double* x) {
  memset(o, 0, sizeof(*o));
  o->n = n;
  o->m = coarse_count(n);
  int64_t m = o->m;
  o->x = (double*)malloc(sizeof(double) * n);
  o->xc = (double*)malloc(sizeof(double) * m);
  o->cidx = (int64_t*)malloc(sizeof(int64_t) * n);
  o->p0 = (int64_t*)malloc(sizeof(int64_t) * n);
  o->p1 = (int64_t*)malloc(sizeof(int64_t) * n);
  o->w0 = (double*)malloc(sizeof(double) * n);
  o->w1 = (double*)malloc(sizeof(double) * n);
  o->nnz = (int*)malloc(sizeof(int) * n);
  o->K = (double*)calloc((size_t)(m * n), sizeof(double));
  o->klo = (int64_t*)malloc(sizeof(int64_t) * m);
  o->khi = (int64_t*)malloc(sizeof(int64_t) * m);
  o->ma = (double*)malloc(sizeof(double) * m);
  o->mb = (double*)malloc(sizeof(double) * m);
  o->mc = (double*)malloc(sizeof(double) * m);
  if (!o->x || !o->xc || !o->cidx || !o->p0 || !o->p1 || !o->w0 || !o->w1 || !o->nnz || !o->K ||
      !o->klo || !o->khi || !o->ma || !o->mb || !o->mc) {
    level1d_free(o);
    return -2;
  }
  memcpy(o->x, x, sizeof(double) * n);
  int64_t q = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (is_coarse(i, n)) {
      o->cidx[i] = q;
      o->xc[q] = x[i];
      ++q;
    } else {
      o->cidx[i] = -1;
    }
  }
  /* P: coarse rows copy, fine rows interpolate linearly between i-1 and i+1
     (both neighbours of a fine position are coarse under the keep-last rule) */
  for (int64_t i = 0; i < n; ++i) {
    if (o->cidx[i] >= 0) {
      o->nnz[i] = 1; o->p0[i] = o->cidx[i]; o->w0[i] = 1.0; o->p1[i] = 0; o->w1[i] = 0.0;
    } else {
      double xa = x[i - 1], xb = x[i + 1], xj = x[i];
      o->nnz[i] = 2;
      o->p0[i] = o->cidx[i - 1]; o->w0[i] = (xb - xj) / (xb - xa);
      o->p1[i] = o->cidx[i + 1]; o->w1[i] = (xj - xa) / (xb - xa);
    }
  }
  /* K = P^T M : K[q][j] = sum_i P[i][q] M[i][j] */
  double* a = (double*)malloc(sizeof(double) * n);
  double* b = (double*)malloc(sizeof(double) * n);
  double* c = (double*)malloc(sizeof(double) * n);
  if (!a || !b || !c) { free(a); free(b); free(c); level1d_free(o); return -2; }
  mass_matrix(n, x, a, b, c);
  for (int64_t i = 0; i < n; ++i) {
    for (int t = 0; t < o->nnz[i]; ++t) {
      int64_t qq = (t == 0) ? o->p0[i] : o->p1[i];
      double w = (t == 0) ? o->w0[i] : o->w1[i];
      if (i > 0) o->K[qq * n + (i - 1)] += w * a[i];
      o->K[qq * n + i] += w * b[i];
      if (i < n - 1) o->K[qq * n + (i + 1)] += w * c[i];
    }
  }
  free(a); free(b); free(c);
  for (int64_t r = 0; r < m; ++r) {
    int64_t lo = n, hi = -1;
    for (int64_t j = 0; j < n; ++j)
      if (o->K[r * n + j] != 0.0) { if (j < lo) lo = j; if (j > hi) hi = j; }
    if (hi < 0) { lo = 0; hi = -1; }
    o->klo[r] = lo; o->khi[r] = hi;
  }
  /* coarse mass matrix on the coarse coordinates */
  mass_matrix(m, o->xc, o->ma, o->mb, o->mc);
  return 0;
}

/* K of one level, dense m x n, for the pins.  Returns m (or <0 on error). */
int64_t oracle_transfer_1d(int64_t n, const double* x, double* K_out /* m*n, may be NULL */) {
  level1d o;
  if (n < 2) return -1;
  if (level1d_build(&o, n, x) != 0) return -2;
  int64_t m = o.m;
  if (K_out) memcpy(K_out, o.K, sizeof(double) * (size_t)(m * n));
  level1d_free(&o);
  return m;
}

/* Interpolation P of one level, dense n x m, for the pins. */
int64_t oracle_interp_1d(int64_t n, const double* x, double* P_out /* n*m, may be NULL */) {
  level1d o;
  if (n < 2) return -1;
  if (level1d_build(&o, n, x) != 0) return -2;
  int64_t m = o.m;
  if (P_out) {
    memset(P_out, 0, sizeof(double) * (size_t)(n * m));
    for (int64_t i = 0; i < n; ++i) {
      P_out[i * m + o.p0[i]] += o.w0[i];
      if (o.nnz[i] == 2) P_out[i * m + o.p1[i]] += o.w1[i];
    }
  }
  level1d_free(&o);
  return m;
}

/* ------------------------------------------------------------------ */
/* 1D line operations                                                   */
/* ------------------------------------------------------------------ */

/* out[0..n) = P in[0..m) */
static void line_interp(const level1d* o, const double* in, double* out) {
  for (int64_t i = 0; i < o->n; ++i) {
    if (o->nnz[i] == 1)
      out[i] = in[o->p0[i]];
    else
      out[i] = o->w0[i] * in[o->p0[i]] + o->w1[i] * in[o->p1[i]];
  }
}

/* out[0..m) = K in[0..n) */
static void line_transfer(const level1d* o, const double* in, double* out) {
  for (int64_t r = 0; r < o->m; ++r) {
    double s = 0.0;
    for (int64_t j = o->klo[r]; j <= o->khi[r]; ++j) s += o->K[r * o->n + j] * in[j];
    out[r] = s;
  }
}

/* Thomas algorithm for M^c z = d, in place on d[0..m).  work: 2m doubles. */
static void line_thomas(const level1d* o, double* d, double* work) {
  int64_t m = o->m;
  double* cp = work;
  double* dp = work + m;
  cp[0] = o->mc[0] / o->mb[0];
  dp[0] = d[0] / o->mb[0];
  for (int64_t i = 1; i < m; ++i) {
    double den = o->mb[i] - o->ma[i] * cp[i - 1];
    cp[i] = o->mc[i] / den;
    dp[i] = (d[i] - o->ma[i] * dp[i - 1]) / den;
  }
  d[m - 1] = dp[m - 1];
  for (int64_t i = m - 2; i >= 0; --i) d[i] = dp[i] - cp[i] * d[i + 1];
}

/* ------------------------------------------------------------------ */
/* Apply a 1D operation along one axis of a row-major array             */
/* ------------------------------------------------------------------ */

enum { OP_INTERP = 0, OP_TRANSFER = 1, OP_SOLVE = 2 };

/* in has shape `shape` (ndim dims); out has the same shape except along
   `axis` where its length is nout.  Returns 0 or -2. */
static int apply_axis(int ndim, const int64_t* shape, int axis, const level1d* o, int op,
                      const double* in, double* out) {
  int64_t nin = shape[axis];
  int64_t nout = (op == OP_INTERP) ? o->n : (op == OP_TRANSFER ? o->m : o->m);
  int64_t inner = 1, outer = 1;
  for (int k = axis + 1; k < ndim; ++k) inner *= shape[k];
  for (int k = 0; k < axis; ++k) outer *= shape[k];
  int64_t maxlen = (nin > nout ? nin : nout);
  double* lin = (double*)malloc(sizeof(double) * maxlen);
  double* lout = (double*)malloc(sizeof(double) * maxlen);
  double* work = (double*)malloc(sizeof(double) * 2 * maxlen);
  if (!lin || !lout || !work) { free(lin); free(lout); free(work); return -2; }
  for (int64_t a = 0; a < outer; ++a) {
    for (int64_t b = 0; b < inner; ++b) {
      for (int64_t i = 0; i < nin; ++i) lin[i] = in[(a * nin + i) * inner + b];
      if (op == OP_INTERP) {
        line_interp(o, lin, lout);
      } else if (op == OP_TRANSFER) {
        line_transfer(o, lin, lout);
      } else {
        for (int64_t i = 0; i < nin; ++i) lout[i] = lin[i];
        line_thomas(o, lout, work);
      }
      for (int64_t i = 0; i < nout; ++i) out[(a * nout + i) * inner + b] = lout[i];
    }
  }
  free(lin); free(lout); free(work);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Multi-dimensional helpers                                            */
/* ------------------------------------------------------------------ */

static int64_t prod(int ndim, const int64_t* s) {
  int64_t p = 1;
  for (int k = 0; k < ndim; ++k) p *= s[k];
  return p;
}

/* Unravel flat index f of shape s into idx. */
static void unravel(int ndim, const int64_t* s, int64_t f, int64_t* idx) {
  for (int k = ndim - 1; k >= 0; --k) {
    idx[k] = f % s[k];
    f /= s[k];
  }
}

typedef struct {
  int ndim;
  int L;
  int64_t full[ORACLE_MAXDIM];
  /* lists[l][k]: full-grid indices of the level-l list along dim k, l = 0..L */
  int64_t* lists[64][ORACLE_MAXDIM];
  int64_t len[64][ORACLE_MAXDIM];
  double* coord[ORACLE_MAXDIM]; /* full-grid coordinates */
} hierarchy;

static void hierarchy_free(hierarchy* h) {
  for (int l = 0; l <= h->L; ++l)
    for (int k = 0; k < h->ndim; ++k) free(h->lists[l][k]);
  for (int k = 0; k < h->ndim; ++k) free(h->coord[k]);
  memset(h, 0, sizeof(*h));
}

static int hierarchy_build(hierarchy* h, int ndim, const int64_t* shape, const double* const* coords,
                           int levels) {
  memset(h, 0, sizeof(*h));
  int maxL = oracle_max_levels(ndim, shape);
  if (maxL < 0) return -1;
  if (levels < 0) levels = oracle_default_levels(ndim, shape);
  if (levels > maxL || levels > 62) return -1;
  h->ndim = ndim;
  h->L = levels;
  for (int k = 0; k < ndim; ++k) {
    h->full[k] = shape[k];
    h->coord[k] = (double*)malloc(sizeof(double) * shape[k]);
    if (!h->coord[k]) { hierarchy_free(h); return -2; }
    for (int64_t i = 0; i < shape[k]; ++i) h->coord[k][i] = (coords && coords[k]) ? coords[k][i] : (double)i;
    for (int64_t i = 1; i < shape[k]; ++i)
      if (!(h->coord[k][i] > h->coord[k][i - 1])) { hierarchy_free(h); return -1; }
  }
  for (int k = 0; k < ndim; ++k) {
    h->len[levels][k] = shape[k];
    h->lists[levels][k] = (int64_t*)malloc(sizeof(int64_t) * shape[k]);
    if (!h->lists[levels][k]) { hierarchy_free(h); return -2; }
    for (int64_t i = 0; i < shape[k]; ++i) h->lists[levels][k][i] = i;
    for (int l = levels; l >= 1; --l) {
      int64_t n = h->len[l][k];
      int64_t m = coarse_count(n);
      h->len[l - 1][k] = m;
      h->lists[l - 1][k] = (int64_t*)malloc(sizeof(int64_t) * m);
      if (!h->lists[l - 1][k]) { hierarchy_free(h); return -2; }
      int64_t q = 0;
      for (int64_t i = 0; i < n; ++i)
        if (is_coarse(i, n)) h->lists[l - 1][k][q++] = h->lists[l][k][i];
    }
  }
  return 0;
}

/* Build the 1D operators of level l for every dimension. */
static int build_level_ops(const hierarchy* h, int l, level1d* ops) {
  for (int k = 0; k < h->ndim; ++k) {
    int64_t n = h->len[l][k];
    double* x = (double*)malloc(sizeof(double) * n);
    if (!x) return -2;
    for (int64_t i = 0; i < n; ++i) x[i] = h->coord[k][h->lists[l][k][i]];
    int rc = level1d_build(&ops[k], n, x);
    free(x);
    if (rc != 0) {
      for (int j = 0; j < k; ++j) level1d_free(&ops[j]);
      return rc;
    }
  }
  return 0;
}

/* Flat offset in the full grid of the level-l node with level indices idx. */
static int64_t full_offset(const hierarchy* h, int l, const int64_t* idx) {
  int64_t off = 0;
  for (int k = 0; k < h->ndim; ++k) off = off * h->full[k] + h->lists[l][k][idx[k]];
  return off;
}

/* z := (x_k M^c_k)^-1 (x_k K_k) c  for the level-l coefficient array c (shape n). */
static int correction(int ndim, const level1d* ops, const double* c, double** z_out) {
  int64_t shape[ORACLE_MAXDIM];
  for (int k = 0; k < ndim; ++k) shape[k] = ops[k].n;
  double* cur = (double*)malloc(sizeof(double) * prod(ndim, shape));
  if (!cur) return -2;
  memcpy(cur, c, sizeof(double) * prod(ndim, shape));
  /* load vector: K along each dimension, last dimension first */
  for (int k = ndim - 1; k >= 0; --k) {
    int64_t s2[ORACLE_MAXDIM];
    memcpy(s2, shape, sizeof(s2));
    s2[k] = ops[k].m;
    double* nxt = (double*)malloc(sizeof(double) * prod(ndim, s2));
    if (!nxt) { free(cur); return -2; }
    if (apply_axis(ndim, shape, k, &ops[k], OP_TRANSFER, cur, nxt) != 0) { free(cur); free(nxt); return -2; }
    free(cur);
    cur = nxt;
    shape[k] = ops[k].m;
  }
  /* tridiagonal solves on the coarse grid, last dimension first */
  for (int k = ndim - 1; k >= 0; --k) {
    double* nxt = (double*)malloc(sizeof(double) * prod(ndim, shape));
    if (!nxt) { free(cur); return -2; }
    if (apply_axis(ndim, shape, k, &ops[k], OP_SOLVE, cur, nxt) != 0) { free(cur); free(nxt); return -2; }
    free(cur);
    cur = nxt;
  }
  *z_out = cur;
  return 0;
}

/* I := (x_k P_k) vc, vc of coarse shape m, I of fine shape n. */
static int interpolate(int ndim, const level1d* ops, const double* vc, double** I_out) {
  int64_t shape[ORACLE_MAXDIM];
  for (int k = 0; k < ndim; ++k) shape[k] = ops[k].m;
  double* cur = (double*)malloc(sizeof(double) * prod(ndim, shape));
  if (!cur) return -2;
  memcpy(cur, vc, sizeof(double) * prod(ndim, shape));
  for (int k = ndim - 1; k >= 0; --k) {
    int64_t s2[ORACLE_MAXDIM];
    memcpy(s2, shape, sizeof(s2));
    s2[k] = ops[k].n;
    double* nxt = (double*)malloc(sizeof(double) * prod(ndim, s2));
    if (!nxt) { free(cur); return -2; }
    if (apply_axis(ndim, shape, k, &ops[k], OP_INTERP, cur, nxt) != 0) { free(cur); free(nxt); return -2; }
    free(cur);
    cur = nxt;
    shape[k] = ops[k].n;
  }
  *I_out = cur;
  return 0;
}

/* Is the level-l node idx in N_{l-1}?  Returns its coarse flat index or -1. */
static int64_t coarse_flat(int ndim, const level1d* ops, const int64_t* idx) {
  int64_t f = 0;
  for (int k = 0; k < ndim; ++k) {
    int64_t ci = ops[k].cidx[idx[k]];
    if (ci < 0) return -1;
    f = f * ops[k].m + ci;
  }
  return f;
}

/* ------------------------------------------------------------------ */
/* Public entry points                                                  */
/* ------------------------------------------------------------------ */

int oracle_decompose(int ndim, const int64_t* shape, const double* const* coords, int levels,
                     const double* in, double* out) {
  hierarchy h;
  int rc = hierarchy_build(&h, ndim, shape, coords, levels);
  if (rc != 0) return rc;
  int64_t N = prod(ndim, shape);
  double* v = (double*)malloc(sizeof(double) * N);
  double* tmp = (double*)malloc(sizeof(double) * N);
  if (!v || !tmp) { free(v); free(tmp); hierarchy_free(&h); return -2; }
  memcpy(v, in, sizeof(double) * N);
  memcpy(tmp, in, sizeof(double) * N);
  for (int l = h.L; l >= 1; --l) {
    level1d ops[ORACLE_MAXDIM];
    if ((rc = build_level_ops(&h, l, ops)) != 0) break;
    int64_t n[ORACLE_MAXDIM], m[ORACLE_MAXDIM];
    for (int k = 0; k < ndim; ++k) { n[k] = ops[k].n; m[k] = ops[k].m; }
    int64_t nn = prod(ndim, n), mm = prod(ndim, m);
    /* v restricted to N_{l-1} */
    double* vc = (double*)malloc(sizeof(double) * mm);
    double* c = (double*)malloc(sizeof(double) * nn);
    if (!vc || !c) { free(vc); free(c); rc = -2; }
    int64_t idx[ORACLE_MAXDIM];
    if (rc == 0) {
      for (int64_t f = 0; f < nn; ++f) {
        unravel(ndim, n, f, idx);
        int64_t cf = coarse_flat(ndim, ops, idx);
        if (cf >= 0) vc[cf] = v[f];
      }
    }
    /* coefficients: c = v - interpolant of v|N_{l-1}; exactly zero on N_{l-1} */
    double* I = NULL;
    if (rc == 0) rc = interpolate(ndim, ops, vc, &I);
    if (rc == 0) {
      for (int64_t f = 0; f < nn; ++f) {
        unravel(ndim, n, f, idx);
        if (coarse_flat(ndim, ops, idx) >= 0) {
          c[f] = 0.0;
        } else {
          c[f] = v[f] - I[f];
          tmp[full_offset(&h, l, idx)] = c[f];
        }
      }
    }
    free(I);
    /* correction z = Q_{l-1}(coefficients), then v := v|N_{l-1} + z */
    double* z = NULL;
    if (rc == 0) rc = correction(ndim, ops, c, &z);
    if (rc == 0) {
      for (int64_t f = 0; f < mm; ++f) vc[f] += z[f];
      free(v);
      v = vc;
      vc = NULL;
    }
    free(z); free(vc); free(c);
    for (int k = 0; k < ndim; ++k) level1d_free(&ops[k]);
    if (rc != 0) break;
  }
  if (rc == 0) {
    int64_t n0[ORACLE_MAXDIM];
    for (int k = 0; k < ndim; ++k) n0[k] = h.len[0][k];
    int64_t idx[ORACLE_MAXDIM];
    for (int64_t f = 0; f < prod(ndim, n0); ++f) {
      unravel(ndim, n0, f, idx);
      tmp[full_offset(&h, 0, idx)] = v[f];
    }
    memcpy(out, tmp, sizeof(double) * N);
  }
  free(v); free(tmp);
  hierarchy_free(&h);
  return rc;
}

int oracle_recompose(int ndim, const int64_t* shape, const double* const* coords, int levels,
                     const double* in, double* out) {
  hierarchy h;
  int rc = hierarchy_build(&h, ndim, shape, coords, levels);
  if (rc != 0) return rc;
  int64_t N = prod(ndim, shape);
  int64_t n0[ORACLE_MAXDIM];
  for (int k = 0; k < ndim; ++k) n0[k] = h.len[0][k];
  int64_t idx[ORACLE_MAXDIM];
  double* v = (double*)malloc(sizeof(double) * prod(ndim, n0));
  if (!v) { hierarchy_free(&h); return -2; }
  for (int64_t f = 0; f < prod(ndim, n0); ++f) {
    unravel(ndim, n0, f, idx);
    v[f] = in[full_offset(&h, 0, idx)];
  }
  for (int l = 1; l <= h.L; ++l) {
    level1d ops[ORACLE_MAXDIM];
    if ((rc = build_level_ops(&h, l, ops)) != 0) break;
    int64_t n[ORACLE_MAXDIM];
    for (int k = 0; k < ndim; ++k) n[k] = ops[k].n;
    int64_t nn = prod(ndim, n);
    double* c = (double*)malloc(sizeof(double) * nn);
    if (!c) rc = -2;
    if (rc == 0) {
      for (int64_t f = 0; f < nn; ++f) {
        unravel(ndim, n, f, idx);
        c[f] = (coarse_flat(ndim, ops, idx) >= 0) ? 0.0 : in[full_offset(&h, l, idx)];
      }
    }
    double* z = NULL;
    if (rc == 0) rc = correction(ndim, ops, c, &z);
    double* I = NULL;
    if (rc == 0) {
      int64_t mm = 1;
      for (int k = 0; k < ndim; ++k) mm *= ops[k].m;
      for (int64_t f = 0; f < mm; ++f) v[f] -= z[f];
      rc = interpolate(ndim, ops, v, &I);
    }
    if (rc == 0) {
      for (int64_t f = 0; f < nn; ++f) I[f] += c[f];
      free(v);
      v = I;
      I = NULL;
    }
    free(I); free(z); free(c);
    for (int k = 0; k < ndim; ++k) level1d_free(&ops[k]);
    if (rc != 0) break;
  }
  if (rc == 0) memcpy(out, v, sizeof(double) * N);
  free(v);
  hierarchy_free(&h);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Coefficient classes (Sec. I: the data are modelled by hierarchically */
/* organised coefficient classes; reconstructing from a prefix of them   */
/* gives an approximation of chosen fidelity)                            */
/* ------------------------------------------------------------------ */
/*
 * Class 0 holds the nodal values on the coarsest grid N_0; class l (1..L)
 * holds the coefficients on N_l \ N_{l-1}.  The class-packed layout stores
 * the classes one after another, coarsest first, each in row-major order of
 * its level grid (nodes of N_{l-1} skipped).  With the nodal layout every
 * entry already sits at its own full-grid position, so packing is a pure
 * reordering: it is written here directly from that definition, visiting the
 * level grids node by node.
 */

/* Is the level-l node idx in N_{l-1} (coarse along every dimension)? */
static int in_coarser(const hierarchy* h, int l, const int64_t* idx) {
  for (int k = 0; k < h->ndim; ++k)
    if (!is_coarse(idx[k], h->len[l][k])) return 0;
  return 1;
}

/* offsets[c] = first packed position of class c, c = 0..L; offsets[L+1] = N.
   Returns the number of classes L+1, or a negative error. */
int oracle_class_offsets(int ndim, const int64_t* shape, int levels, int64_t* offsets) {
  hierarchy h;
  int rc = hierarchy_build(&h, ndim, shape, NULL, levels);
  if (rc != 0) return rc;
  int64_t pos = 0;
  for (int l = 0; l <= h.L; ++l) {
    offsets[l] = pos;
    int64_t n = 1, mm = 1;
    for (int k = 0; k < ndim; ++k) n *= h.len[l][k];
    if (l > 0)
      for (int k = 0; k < ndim; ++k) mm *= h.len[l - 1][k];
    pos += (l == 0) ? n : n - mm;
  }
  offsets[h.L + 1] = pos;
  int ncls = h.L + 1;
  hierarchy_free(&h);
  return ncls;
}

/* Visit every entry of the packed layout in order, calling
   fn(packed position, nodal offset, class). */
static int for_each_class_entry(int ndim, const int64_t* shape, int levels,
                                void (*fn)(void*, int64_t, int64_t, int), void* arg) {
  hierarchy h;
  int rc = hierarchy_build(&h, ndim, shape, NULL, levels);
  if (rc != 0) return rc;
  int64_t pos = 0, idx[ORACLE_MAXDIM];
  for (int l = 0; l <= h.L; ++l) {
    int64_t n[ORACLE_MAXDIM];
    for (int k = 0; k < ndim; ++k) n[k] = h.len[l][k];
    for (int64_t f = 0; f < prod(ndim, n); ++f) {
      unravel(ndim, n, f, idx);
      if (l > 0 && in_coarser(&h, l, idx)) continue;
      fn(arg, pos++, full_offset(&h, l, idx), l);
    }
  }
  hierarchy_free(&h);
  return 0;
}

typedef struct {
  const double* src;
  double* dst;
  int nclasses;
} copy_args;

static void pack_one(void* a, int64_t pos, int64_t off, int cls) {
  copy_args* c = (copy_args*)a;
  (void)cls;
  c->dst[pos] = c->src[off];
}

static void unpack_one(void* a, int64_t pos, int64_t off, int cls) {
  copy_args* c = (copy_args*)a;
  c->dst[off] = (cls < c->nclasses) ? c->src[pos] : 0.0;
}

/* nodal layout -> class-packed layout (a permutation of the N entries). */
int oracle_pack_classes(int ndim, const int64_t* shape, int levels, const double* nodal, double* packed) {
  copy_args a = {nodal, packed, 0};
  return for_each_class_entry(ndim, shape, levels, pack_one, &a);
}

/* class-packed layout -> nodal layout, keeping classes 0..nclasses-1; the
   positions of the dropped classes are set to 0 (a dropped class is a zero
   coefficient class).  `packed` needs only its first offsets[nclasses]
   entries. */
int oracle_unpack_classes(int ndim, const int64_t* shape, int levels, int nclasses, const double* packed,
                          double* nodal) {
  if (nclasses < 1) return -1;
  copy_args a = {packed, nodal, nclasses};
  return for_each_class_entry(ndim, shape, levels, unpack_one, &a);
}

/* ------------------------------------------------------------------ */
/* Linear quantization bins with an L-infinity guarantee                */
/* (the quantization stage that follows refactoring in the lossy        */
/* compression workflow of Sec. V "Lossy compression")                  */
/* ------------------------------------------------------------------ */
/*
 * The paper moves quantization and dequantization to the GPU but does not
 * state the quantizer.  Reading adopted: uniform (linear) quantization of
 * each coefficient class with its own bin width q_l, codes k = round(c / q_l),
 * dequantized values k * q_l, and widths chosen so that the recomposed field
 * is within tau of the original in the maximum norm.
 *
 * Bound.  Recomposition maps coefficient perturbations d_0 (coarsest values)
 * and d_l (level l) to a field perturbation e with e_0 = d_0 and
 * e_l = d_l + P_l (e_{l-1} - Z_l d_l), where Z_l = (x_k M^c_k)^-1 (x_k K_k) is
 * the correction operator of level l and P_l the interpolation (rows are
 * convex weights, so |P_l|_inf = 1).  Hence
 *   |e_L|_inf <= |d_0|_inf + sum_l (1 + |Z_l|_inf) |d_l|_inf,
 * and |Z_l|_inf is the product over dimensions of the 1D norms (the infinity
 * norm of a Kronecker product is the product of the norms).  Rounding gives
 * |d_l|_inf <= q_l / 2; splitting tau equally over the L+1 classes gives
 *   q_0 = 2 tau / (L+1),   q_l = 2 tau / ((L+1) (1 + |Z_l|_inf)).
 */

/* |Z|_inf of one dimension at one level: Z = (M^c)^-1 K, column by column. */
static int correction_norm_1d(const level1d* o, double* norm) {
  int64_t n = o->n, m = o->m;
  double* col = (double*)malloc(sizeof(double) * m);
  double* work = (double*)malloc(sizeof(double) * 2 * m);
  double* rows = (double*)calloc((size_t)m, sizeof(double));
  if (!col || !work || !rows) { free(col); free(work); free(rows); return -2; }
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t r = 0; r < m; ++r) col[r] = o->K[r * n + j];
    line_thomas(o, col, work);
    for (int64_t r = 0; r < m; ++r) rows[r] += col[r] < 0 ? -col[r] : col[r];
  }
  double best = 0.0;
  for (int64_t r = 0; r < m; ++r)
    if (rows[r] > best) best = rows[r];
  *norm = best;
  free(col); free(work); free(rows);
  return 0;
}

/* bins[c] = bin width of class c (c = 0..L) for the L-infinity tolerance tau.
   Returns L+1, or a negative error. */
int oracle_quant_bins(int ndim, const int64_t* shape, const double* const* coords, int levels, double tau,
                      double* bins) {
  if (!(tau > 0.0)) return -1;
  hierarchy h;
  int rc = hierarchy_build(&h, ndim, shape, coords, levels);
  if (rc != 0) return rc;
  int L = h.L;
  bins[0] = 2.0 * tau / (L + 1);
  for (int l = 1; l <= L && rc == 0; ++l) {
    level1d ops[ORACLE_MAXDIM];
    if ((rc = build_level_ops(&h, l, ops)) != 0) break;
    double znorm = 1.0;
    for (int k = 0; k < ndim && rc == 0; ++k) {
      double nk = 0.0;
      rc = correction_norm_1d(&ops[k], &nk);
      znorm *= nk;
    }
    bins[l] = 2.0 * tau / ((L + 1) * (1.0 + znorm));
    for (int k = 0; k < ndim; ++k) level1d_free(&ops[k]);
  }
  hierarchy_free(&h);
  return rc == 0 ? L + 1 : rc;
}
