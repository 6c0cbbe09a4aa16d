"""Pins of the oracle's coefficient-class layout and progressive recomposition.

arXiv 2105.12764, Sec. I: the refactored data are hierarchically organised
coefficient classes, and an approximation of chosen fidelity is rebuilt from
the first few of them.  Class 0 is the coarsest grid N_0, class l the
coefficients on N_l \\ N_{l-1}; the packed layout stores them coarsest first,
each in row-major order of its level grid.  Checked against:

* the worked example of Fig. example-1d (hand-derived golden fixture);
* the class sizes |N_l| - |N_{l-1}| from independently built level lists;
* the packed order rebuilt with numpy index arithmetic;
* the dense L2 projection: the field rebuilt from classes 0..k is Q_k u,
  interpolated to the finest grid (Eq. (1)), on tiny 1D/2D/3D grids;
* the projection property: the M-norm error ||u - Q_k u|| does not grow as
  classes are added, and the error of class k+1's omission is orthogonal to
  the level-k space.
"""
import os

import numpy as np
import pytest

import dense_l2
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel_linf(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def stretched(n, ratio=1.1):
    return np.concatenate([[0.0], np.cumsum(ratio ** np.arange(n - 1))])


def packed_order(shape, L):
    """Nodal flat offsets in packed order, from dense_l2's level lists."""
    d = len(shape)
    lists = [dense_l2.level_lists(shape[k], L) for k in range(d)]
    strides = [int(np.prod(shape[k + 1:])) for k in range(d)]
    order = []
    for l in range(L + 1):
        full = [np.array(lists[k][l]) for k in range(d)]
        grids = np.meshgrid(*full, indexing="ij")
        offs = sum(g * s for g, s in zip(grids, strides)).ravel()
        if l == 0:
            keep = np.ones(offs.shape, dtype=bool)
        else:
            coarse = [np.isin(full[k], lists[k][l - 1]) for k in range(d)]
            cg = np.meshgrid(*coarse, indexing="ij")
            keep = ~np.logical_and.reduce(cg).ravel() if d > 1 else ~cg[0].ravel()
        order.append(offs[keep])
    return np.concatenate(order)


SHAPES = [(2,), (5,), (17,), (24,), (33,), (5, 5), (9, 6), (7, 12), (5, 5, 5), (9, 6, 7), (11, 8, 5)]


def test_worked_example_classes():
    rows = np.loadtxt(os.path.join(GOLDEN, "worked_example_1d_classes.txt"))
    u = np.arange(5.0) ** 2 - 5 * np.arange(5.0) + 6
    np.testing.assert_array_equal(rows[3], u)
    packed = oracle.pack_classes(oracle.decompose(u, levels=2), levels=2)
    np.testing.assert_allclose(packed, rows[0], rtol=0, atol=1e-15)
    np.testing.assert_array_equal(oracle.class_offsets((5,), 2), [0, 2, 3, 5])
    for k in range(3):
        np.testing.assert_allclose(oracle.recompose_classes(packed, (5,), k + 1, levels=2), rows[k + 1],
                                   rtol=0, atol=1e-14)


@pytest.mark.parametrize("shape", SHAPES)
def test_class_sizes(shape):
    d = len(shape)
    for L in range(0, oracle.max_levels(shape) + 1):
        lists = [dense_l2.level_lists(shape[k], L) for k in range(d)]
        size = [int(np.prod([len(lists[k][l]) for k in range(d)])) for l in range(L + 1)]
        expect = np.cumsum([0, size[0]] + [size[l] - size[l - 1] for l in range(1, L + 1)])
        np.testing.assert_array_equal(oracle.class_offsets(shape, L), expect)
        assert expect[-1] == int(np.prod(shape))


@pytest.mark.parametrize("shape", SHAPES)
def test_packed_order_and_inverse(shape):
    rng = np.random.default_rng(len(shape))
    for L in range(0, oracle.max_levels(shape) + 1):
        N = int(np.prod(shape))
        idx = np.arange(N, dtype=np.float64).reshape(shape)
        perm = oracle.pack_classes(idx, L)
        np.testing.assert_array_equal(perm, packed_order(shape, L).astype(np.float64))
        np.testing.assert_array_equal(np.sort(perm), np.arange(N, dtype=np.float64))
        x = rng.standard_normal(shape)
        np.testing.assert_array_equal(oracle.unpack_classes(oracle.pack_classes(x, L), shape, None, L), x)


@pytest.mark.parametrize("shape", SHAPES)
def test_unpack_prefix_zeroes_dropped_classes(shape):
    L = oracle.default_levels(shape)
    offs = oracle.class_offsets(shape, L)
    x = np.random.default_rng(1).standard_normal(shape) + 10.0  # no zero entries
    packed = oracle.pack_classes(x, L)
    order = packed_order(shape, L)
    for k in range(1, L + 2):
        y = oracle.unpack_classes(packed[: offs[k]], shape, k, L).ravel()
        kept = order[: offs[k]]
        dropped = order[offs[k]:]
        np.testing.assert_array_equal(y[kept], x.ravel()[kept])
        assert np.all(y[dropped] == 0.0)


def prefix_by_projection(u, coords, L, k):
    """Q_k u interpolated to the finest grid, by dense projection (dense_l2)."""
    d = u.ndim
    xs = [np.arange(u.shape[j], dtype=np.float64) if coords is None else coords[j] for j in range(d)]
    a = u
    for j in range(d):
        lists = dense_l2.level_lists(u.shape[j], L)
        Pj = dense_l2.projection_operators(xs[j], lists[L], lists[k])
        Ij = dense_l2.interpolation(xs[j], lists[L], lists[k])
        a = dense_l2._apply_axis(Ij @ Pj, a, j)
    return a


@pytest.mark.parametrize("shape,kind", [((17,), "uniform"), ((20,), "stretched"), ((9, 9), "uniform"),
                                        ((11, 8), "stretched"), ((9, 7, 6), "uniform"), ((7, 9, 10), "stretched")])
def test_prefix_is_projection(shape, kind):
    rng = np.random.default_rng(sum(shape))
    u = rng.standard_normal(shape)
    coords = None if kind == "uniform" else [stretched(n) for n in shape]
    L = oracle.max_levels(shape)
    packed = oracle.pack_classes(oracle.decompose(u, coords, L), L)
    for k in range(L + 1):
        got = oracle.recompose_classes(packed, shape, k + 1, coords, L)
        assert rel_linf(got, prefix_by_projection(u, coords, L, k)) <= 1e-12


def test_prefix_error_decreases_in_mass_norm():
    shape = (13, 10)
    coords = [stretched(13, 1.2), stretched(10, 0.9)]
    u = np.random.default_rng(5).standard_normal(shape)
    L = oracle.max_levels(shape)
    G = [dense_l2.gram(c, c, c) for c in coords]  # finest-grid mass matrices
    packed = oracle.pack_classes(oracle.decompose(u, coords, L), L)
    errs = []
    prev = None
    for k in range(L + 1):
        r = u - oracle.recompose_classes(packed, shape, k + 1, coords, L)
        errs.append(float(np.sum(r * (G[0] @ r @ G[1].T))))  # ||u - Q_k u||_M^2
        if prev is not None:
            # Q_k u - Q_{k-1} u lies in the level-k space, to which u - Q_k u is M-orthogonal
            inc = prev - r
            assert abs(np.sum(r * (G[0] @ inc @ G[1].T))) <= 1e-10 * max(1.0, errs[0])
        prev = r
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-12) for i in range(L))
    assert errs[-1] <= 1e-24


def test_invalid_class_arguments():
    with pytest.raises(ValueError):
        oracle.unpack_classes(np.zeros(5), (5,), 0, 2)
    with pytest.raises(ValueError):
        oracle.unpack_classes(np.zeros(2), (5,), 2, 2)  # classes 0, 1 need 3 entries
    with pytest.raises(ValueError):
        oracle.class_offsets((5,), 3)
