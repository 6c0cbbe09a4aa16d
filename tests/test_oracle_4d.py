"""Pins of the oracle in four dimensions: the (3+1)-D spatiotemporal form of
the decomposition (Sec. III.E: the method generalises to any number of
dimensions; time is one more tensor-product axis).

* dense L2-projection definition (dense_l2) on tiny 4D grids, uniform and
  random spacing, every depth;
* fields multilinear on the coarse 4D grid have zero coefficients;
* separable fields: coarsest values are the tensor product of the 1D ones;
* round trip.
"""
import numpy as np
import pytest

import dense_l2
import oracle


def rel_linf(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def random_coords(rng, n):
    return np.concatenate([[0.0], np.cumsum(rng.uniform(0.2, 3.0, n - 1))])


SHAPES_4D = [(5, 5, 5, 5), (3, 5, 4, 6), (6, 9, 5, 7), (9, 6, 7, 5), (5, 3, 9, 4), (9, 9, 9, 9)]


@pytest.mark.parametrize("shape", SHAPES_4D)
@pytest.mark.parametrize("kind", ["uniform", "random"])
def test_dense_projection_4d(shape, kind):
    rng = np.random.default_rng(sum(shape))
    u = rng.standard_normal(shape)
    coords = None if kind == "uniform" else [random_coords(rng, s) for s in shape]
    for L in range(0, oracle.max_levels(shape) + 1):
        a = oracle.decompose(u, coords, L)
        assert rel_linf(a, dense_l2.dense_decompose(u, coords, L)) <= 1e-13, (shape, kind, L)
        assert rel_linf(oracle.recompose(a, coords, L), u) <= 1e-13


def test_multilinear_4d_has_zero_coefficients():
    shape = (9, 5, 9, 6)
    rng = np.random.default_rng(4)
    coords = [random_coords(rng, s) for s in shape]
    # a multilinear function of the coordinates is reproduced by the coarse interpolant
    g = np.meshgrid(*coords, indexing="ij")
    u = 1.0 + 0.3 * g[0] - 0.2 * g[1] * g[2] + 0.05 * g[0] * g[1] * g[2] * g[3] + 0.7 * g[3]
    L = oracle.max_levels(shape)
    out = oracle.decompose(u, coords, L)
    mask = np.ones(shape, dtype=bool)
    lists = [dense_l2.level_lists(s, L) for s in shape]
    mask[np.ix_(*[np.array(lists[k][0]) for k in range(4)])] = False
    assert np.abs(out[mask]).max() <= 1e-12 * np.abs(u).max()


def test_separable_4d():
    shape = (5, 9, 6, 7)
    rng = np.random.default_rng(9)
    parts = [rng.standard_normal(s) for s in shape]
    u = np.einsum("a,b,c,d->abcd", *parts)
    L = oracle.default_levels(shape)
    out = oracle.decompose(u, None, L)
    lists = [dense_l2.level_lists(s, L) for s in shape]
    c1 = [oracle.decompose(p, None, L)[lists[k][0]] for k, p in enumerate(parts)]
    want = np.einsum("a,b,c,d->abcd", *c1)
    got = out[np.ix_(*[np.array(lists[k][0]) for k in range(4)])]
    assert rel_linf(got, want) <= 1e-13
