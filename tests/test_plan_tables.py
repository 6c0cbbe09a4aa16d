"""Pins of the CUDA library's plan tables (no GPU: mgr_plan_tables_host builds
them on the host), against quantities built independently of the library:

* interpolation weights = the hat functions of the coarse nodes evaluated at
  the fine nodes (numpy.interp, tests/dense_l2.py);
* the scaled mass-transfer taps times the LU pivots = K = P^T M with the
  Simpson-exact Gram matrix M (dense_l2) and = the oracle's transfer_1d;
* the whole table set of an axis -- taps, then the forward and backward
  recurrences -- applied to every fine unit vector = M_coarse^-1 K from a
  dense solve with the coarse Gram matrix (Sec. III.A.2 / III.A.3);
* the pivots u_q = the diagonal of the LU factors of the dense coarse Gram
  matrix, and ta, tb their off-diagonal ratios;
on uniform, geometrically stretched and random coordinates, sizes that are
2^k+1 and sizes that are not, every level of the hierarchy, and each axis of
multi-dimensional descriptions (each with its own coordinates).
"""
import numpy as np
import pytest

import oracle
import paper_2105_12764_gb300 as mgr
from dense_l2 import gram, hats, level_lists


def coords_of(kind, n, rng):
    if kind == "uniform":
        return np.arange(n, dtype=np.float64)
    if kind == "stretched":
        return np.concatenate([[0.0], np.cumsum(1.01 ** np.arange(n - 1))])
    return np.concatenate([[0.0], np.cumsum(rng.uniform(0.2, 3.0, n - 1))])


def dense_operators(x_full, L, l):
    lists = level_lists(len(x_full), L)
    xl = x_full[lists[l]]
    xc = x_full[lists[l - 1]]
    P = hats(xc, xl)                 # n x m
    M = gram(xl, xl, xl)             # level-l Gram matrix
    Mc = gram(xc, xc, xc)            # coarse Gram matrix
    return xl, xc, P, M, Mc


def check_axis(t, x_full, L, l):
    xl, xc, P, M, Mc = dense_operators(x_full, L, l)
    n, m = len(xl), len(xc)
    assert (t["n"], t["m"]) == (n, m)
    scale = np.abs(M).max()
    # interpolation weights of the fine nodes
    for i in range(n):
        if i % 2 == 0 or i == n - 1:
            assert t["wa"][i] == 0.0 and t["wb"][i] == 0.0
            continue
        np.testing.assert_allclose([t["wa"][i], t["wb"][i]], [P[i, (i - 1) // 2], P[i, (i + 1) // 2]],
                                   rtol=1e-14, atol=1e-15)
    # scaled taps as a dense m x n matrix
    Ks = np.zeros((m, n))
    for q in range(m):
        p = min(2 * q, n - 1)
        for o in range(5):
            j = p + o - 2
            if 0 <= j < n:
                Ks[q, j] = t["k"][q, o]
            else:
                assert t["k"][q, o] == 0.0
    # the recurrences applied to every fine unit vector: M_coarse^-1 K
    Z = Ks.copy()
    for q in range(1, m):
        Z[q] -= t["ta"][q] * Z[q - 1]
    for q in range(m - 2, -1, -1):
        Z[q] -= t["tb"][q] * Z[q + 1]
    K = P.T @ M
    want = np.linalg.solve(Mc, K)
    np.testing.assert_allclose(Z, want, rtol=0, atol=1e-13 * np.abs(want).max())
    # pivots of the coarse Gram matrix (LU without pivoting, SPD tridiagonal)
    u = np.empty(m)
    u[0] = Mc[0, 0]
    for q in range(1, m):
        u[q] = Mc[q, q] - Mc[q, q - 1] * Mc[q - 1, q] / u[q - 1]
    np.testing.assert_allclose(Ks * u[:, None], K, rtol=0, atol=1e-13 * scale)
    np.testing.assert_allclose(Ks * u[:, None], oracle.transfer_1d(xl), rtol=0, atol=1e-13 * scale)
    for q in range(m):
        if q > 0:
            assert t["ta"][q] == pytest.approx(Mc[q, q - 1] / u[q], rel=1e-13)
        else:
            assert t["ta"][q] == 0.0
        if q < m - 1:
            assert t["tb"][q] == pytest.approx(Mc[q, q + 1] / u[q], rel=1e-13)
        else:
            assert t["tb"][q] == 0.0


@pytest.mark.parametrize("kind", ["uniform", "stretched", "random"])
@pytest.mark.parametrize("n", [2, 3, 4, 5, 9, 12, 17, 23, 33, 65])
def test_1d_tables_every_level(kind, n):
    rng = np.random.default_rng(n)
    x = coords_of(kind, n, rng)
    L = oracle.max_levels((n,))
    for l in range(1, L + 1):
        t = mgr.plan_tables_host((n,), [x], L, l, 0)
        check_axis(t, x, L, l)


def test_3d_axes_use_their_own_coordinates():
    rng = np.random.default_rng(11)
    shape = (17, 30, 41)
    xs = [coords_of("random", shape[0], rng), coords_of("stretched", shape[1], rng), coords_of("random", shape[2], rng)]
    L = oracle.default_levels(shape)
    for l in range(1, L + 1):
        for axis in range(3):
            t = mgr.plan_tables_host(shape, xs, -1, l, axis)
            check_axis(t, xs[axis], L, l)


def test_4d_time_axis_and_space_axes():
    rng = np.random.default_rng(12)
    shape = (9, 11, 13, 17)
    xs = [coords_of("random", s, rng) for s in shape]
    L = oracle.default_levels(shape)
    for l in range(1, L + 1):
        for axis in range(4):
            check_axis(mgr.plan_tables_host(shape, xs, -1, l, axis), xs[axis], L, l)


def test_argument_errors():
    with pytest.raises(mgr.MgrError):
        mgr.plan_tables_host((17, 17), None, -1, 0, 0)  # level 0 has no tables
    with pytest.raises(mgr.MgrError):
        mgr.plan_tables_host((17, 17), None, -1, 1, 2)  # axis out of range
    with pytest.raises(mgr.MgrError):
        mgr.plan_tables_host((17, 17), None, -1, 9, 0)  # deeper than the hierarchy
    bad = np.array([0.0, 1.0, 1.0, 2.0, 3.0])
    with pytest.raises(mgr.MgrError):
        mgr.plan_tables_host((5,), [bad], -1, 1, 0)  # coordinates not increasing
