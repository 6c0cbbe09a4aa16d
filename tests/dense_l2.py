"""Dense L2-projection reference for tiny grids (independent of ``oracle/``).

This is the definition of the multilevel decomposition written out with
dense linear algebra, used to pin the oracle (arXiv 2105.12764, Sec. II.A,
Eq. (1) and Eq. (2): the coarse values after each level are the L2
projection Q_l u, and the level-l coefficients are (I - Pi_{l-1}) Q_l u).

Nothing here reuses the oracle's building blocks:
  * level node lists come from a literal slicing of the previous list;
  * hat functions are evaluated with ``numpy.interp`` on unit vectors;
  * Gram matrices are integrated with Simpson's rule on every finest element,
    which is exact for products of two piecewise-linear functions;
  * projections are dense solves ``numpy.linalg.solve(G, B)``.
"""
import numpy as np


def level_lists(n, levels):
    """Full-grid index lists of levels 0..levels (index by level)."""
    lists = [list(range(n))]
    for _ in range(levels):
        cur = lists[-1]
        nxt = cur[::2]
        if (len(cur) - 1) % 2 == 1:
            nxt = nxt + [cur[-1]]
        lists.append(nxt)
    return lists[::-1]


def hats(x_nodes, x_eval):
    """Matrix H[p, i] = value of the hat function of node i (nodes x_nodes) at x_eval[p]."""
    m = len(x_nodes)
    H = np.empty((len(x_eval), m))
    for i in range(m):
        e = np.zeros(m)
        e[i] = 1.0
        H[:, i] = np.interp(x_eval, x_nodes, e)
    return H


def _simpson_points(x):
    """Nodes, midpoints and Simpson weights on every element of the finest grid."""
    h = np.diff(x)
    mid = 0.5 * (x[:-1] + x[1:])
    return h, mid


def gram(x_full, xa, xb):
    """G[i, j] = integral of hat_i(level a) * hat_j(level b) over the finest grid."""
    h, mid = _simpson_points(x_full)
    A0, A1, Am = hats(xa, x_full[:-1]), hats(xa, x_full[1:]), hats(xa, mid)
    B0, B1, Bm = hats(xb, x_full[:-1]), hats(xb, x_full[1:]), hats(xb, mid)
    w = h / 6.0
    return (A0 * w[:, None]).T @ B0 + 4.0 * (Am * w[:, None]).T @ Bm + (A1 * w[:, None]).T @ B1


def _apply_axis(mat, arr, axis):
    return np.moveaxis(np.tensordot(mat, arr, axes=([1], [axis])), 0, axis)


def projection_operators(x_full, lst_full, lst_level):
    """1D operator taking finest nodal values to the nodal values of Q_level u."""
    xf = x_full[lst_full]
    xl = x_full[lst_level]
    G = gram(x_full, xl, xl)
    B = gram(x_full, xl, xf)
    return np.linalg.solve(G, B)


def interpolation(x_full, lst_fine, lst_coarse):
    """1D piecewise-linear interpolation from level lst_coarse to level lst_fine nodes."""
    return hats(x_full[lst_coarse], x_full[lst_fine])


def dense_decompose(u, coords=None, levels=None):
    """Nodal-layout decomposition of ``u`` by dense projections."""
    u = np.asarray(u, dtype=np.float64)
    d = u.ndim
    xs = [np.arange(u.shape[k], dtype=np.float64) if coords is None or coords[k] is None
          else np.asarray(coords[k], dtype=np.float64) for k in range(d)]
    lists = [level_lists(u.shape[k], levels) for k in range(d)]
    L = levels
    out = np.array(u, copy=True)
    # Q_l u for every level l (l = L is u itself)
    Q = {}
    for l in range(0, L + 1):
        a = u
        for k in range(d):
            Pk = projection_operators(xs[k], lists[k][L], lists[k][l])
            a = _apply_axis(Pk, a, k)
        Q[l] = a
    # coarsest values
    idx0 = np.ix_(*[np.array(lists[k][0]) for k in range(d)])
    out[idx0] = Q[0]
    # coefficients of level l: (I - Pi_{l-1}) Q_l u at N_l \ N_{l-1}
    for l in range(1, L + 1):
        interp = Q[l]
        # restrict Q_l u to N_{l-1} (positions of lists[l-1] inside lists[l])
        sel = []
        for k in range(d):
            pos = {g: i for i, g in enumerate(lists[k][l])}
            sel.append(np.array([pos[g] for g in lists[k][l - 1]]))
        coarse_vals = Q[l][np.ix_(*sel)]
        Pi = coarse_vals
        for k in range(d):
            Ik = interpolation(xs[k], lists[k][l], lists[k][l - 1])
            Pi = _apply_axis(Ik, Pi, k)
        coef = interp - Pi
        # write at N_l \ N_{l-1}
        fine_mask = np.zeros(Q[l].shape, dtype=bool)
        grids = np.meshgrid(*[np.isin(np.arange(len(lists[k][l])), sel[k]) for k in range(d)], indexing="ij")
        all_coarse = np.logical_and.reduce(grids) if d > 1 else grids[0]
        fine_mask = ~all_coarse
        full_idx = np.ix_(*[np.array(lists[k][l]) for k in range(d)])
        block = out[full_idx]
        block[fine_mask] = coef[fine_mask]
        out[full_idx] = block
    return out
