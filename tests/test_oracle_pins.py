"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

arXiv 2105.12764, Sec. II.A: the coarse values after each level are the L2
projection Q_l u (Eq. (1)); the correction is the orthogonal projection of the
coefficients (Eq. (2)); coefficients are interpolation residuals.  Each test
below checks the oracle against something other than itself:

* the worked example of Fig. example-1d (golden fixture, hand-derived);
* the dense L2-projection definition (``dense_l2.py``) on tiny grids;
* closed forms: P1 mass entries (exact Simpson quadrature), the uniform
  mass-transfer row h*[1/2, 3, 5, 3, 1/2]/6, the quadratic midpoint error;
* invariants: multilinear fields, linearity, separability, round trip,
  the Galerkin identity P^T M P = M_coarse.
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


def stretched(n, ratio=1.01):
    """x_0 = 0, x_{i+1} - x_i = ratio**i (geometric stretching)."""
    return np.concatenate([[0.0], np.cumsum(ratio ** np.arange(n - 1))])


def random_coords(rng, n):
    return np.concatenate([[0.0], np.cumsum(rng.uniform(0.2, 3.0, n - 1))])


# ---------------------------------------------------------------- golden ----

def test_worked_example_fig_example_1d():
    data = np.loadtxt(os.path.join(GOLDEN, "worked_example_1d.txt"))
    x, u, expect = data[:, 0], data[:, 1], data[:, 2]
    np.testing.assert_array_equal(u, x ** 2 - 5 * x + 6)
    out = oracle.decompose(u, levels=2)
    np.testing.assert_allclose(out, expect, rtol=0, atol=1e-15)
    np.testing.assert_allclose(oracle.recompose(out, levels=2), u, rtol=0, atol=1e-15)


# ------------------------------------------------------ dense projection ----

@pytest.mark.parametrize("n", list(range(2, 34)))
@pytest.mark.parametrize("kind", ["uniform", "stretched", "random"])
def test_dense_projection_1d(n, kind):
    rng = np.random.default_rng(n)
    u = rng.standard_normal(n)
    coords = None if kind == "uniform" else [stretched(n, 1.1) if kind == "stretched" else random_coords(rng, n)]
    for L in range(0, oracle.max_levels((n,)) + 1):
        a = oracle.decompose(u, coords, L)
        b = dense_l2.dense_decompose(u, coords, L)
        assert rel_linf(a, b) <= 1e-13, (n, kind, L)


SHAPES_ND = [(5, 5), (9, 7), (6, 11), (17, 9), (4, 13), (3, 2), (5, 6, 7), (9, 9, 5), (7, 4, 5), (17, 9, 7), (6, 6, 10)]


@pytest.mark.parametrize("shape", SHAPES_ND)
@pytest.mark.parametrize("kind", ["uniform", "random"])
def test_dense_projection_nd(shape, kind):
    rng = np.random.default_rng(sum(shape))
    u = rng.standard_normal(shape)
    coords = None if kind == "uniform" else [random_coords(rng, s) for s in shape]
    for L in range(0, oracle.max_levels(shape) + 1):
        a = oracle.decompose(u, coords, L)
        b = dense_l2.dense_decompose(u, coords, L)
        assert rel_linf(a, b) <= 1e-13, (shape, kind, L)


def test_dense_projection_stretched_3d():
    shape = (9, 8, 7)
    rng = np.random.default_rng(7)
    u = rng.standard_normal(shape)
    coords = [stretched(s, 1.3) for s in shape]
    for L in range(0, oracle.max_levels(shape) + 1):
        assert rel_linf(oracle.decompose(u, coords, L), dense_l2.dense_decompose(u, coords, L)) <= 1e-13


# ----------------------------------------------------------- closed forms ---

@pytest.mark.parametrize("kind", ["uniform", "random"])
def test_mass_matrix_closed_form_vs_quadrature(kind):
    rng = np.random.default_rng(3)
    n = 12
    x = np.arange(n, dtype=float) if kind == "uniform" else random_coords(rng, n)
    sub, diag, sup = oracle.mass_1d(x)
    M = np.diag(diag) + np.diag(sub[1:], -1) + np.diag(sup[:-1], 1)
    G = dense_l2.gram(x, x, x)  # exact Simpson quadrature of hat products
    np.testing.assert_allclose(M, G, rtol=1e-14, atol=1e-15)
    h = np.diff(x)
    np.testing.assert_allclose(diag[1:-1], (h[:-1] + h[1:]) / 3, rtol=1e-15)
    np.testing.assert_allclose(diag[[0, -1]], [h[0] / 3, h[-1] / 3], rtol=1e-15)
    np.testing.assert_allclose(sup[:-1], h / 6, rtol=1e-15)


@pytest.mark.parametrize("h", [1.0, 0.25, 3.0])
def test_uniform_mass_transfer_row(h):
    # Sec. III.A.2 "mass-trans" K = R M with R = P^T; on a uniform grid every
    # interior row is h * [1/2, 3, 5, 3, 1/2] / 6 (the printed diagonal entry
    # of the paper's K is garbled; this is the value of P^T M).
    n = 17
    x = h * np.arange(n, dtype=float)
    K = oracle.transfer_1d(x)
    assert K.shape == (9, 17)
    for q in range(1, 8):
        row = K[q, 2 * q - 2:2 * q + 3]
        np.testing.assert_allclose(row * 6 / h, [0.5, 3, 5, 3, 0.5], rtol=1e-15)
        assert np.count_nonzero(K[q]) == 5


@pytest.mark.parametrize("n", [5, 6, 9, 12, 17])
def test_transfer_equals_interp_transpose_times_mass(n):
    rng = np.random.default_rng(n)
    x = random_coords(rng, n)
    K = oracle.transfer_1d(x)
    G = dense_l2.gram(x, x, x)
    lst = dense_l2.level_lists(n, 1)
    P = dense_l2.interpolation(x, lst[1], lst[0])
    np.testing.assert_allclose(K, P.T @ G, rtol=1e-13, atol=1e-14 * np.abs(K).max())
    np.testing.assert_allclose(oracle.interp_1d(x), P, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("n", [5, 8, 13])
def test_galerkin_identity(n):
    rng = np.random.default_rng(n + 100)
    x = random_coords(rng, n)
    P = oracle.interp_1d(x)
    sub, diag, sup = oracle.mass_1d(x)
    M = np.diag(diag) + np.diag(sub[1:], -1) + np.diag(sup[:-1], 1)
    xc = x[dense_l2.level_lists(n, 1)[0]]
    s2, d2, u2 = oracle.mass_1d(xc)
    Mc = np.diag(d2) + np.diag(s2[1:], -1) + np.diag(u2[:-1], 1)
    np.testing.assert_allclose(P.T @ M @ P, Mc, rtol=1e-13, atol=1e-14 * np.abs(Mc).max())


@pytest.mark.parametrize("L", [1, 3, 5])
def test_quadratic_closed_form(L):
    # Every level-l coefficient of alpha x^2 + beta x + gamma on a uniform grid
    # is -alpha h_l^2 (midpoint interpolation error); the corrected coarse
    # values stay quadratic with the same alpha, so this holds at every level.
    n = 2 ** L + 1
    h = 0.5
    x = h * np.arange(n)
    alpha, beta, gamma = 1.7, -0.3, 2.0
    u = alpha * x ** 2 + beta * x + gamma
    out = oracle.decompose(u, [x], L)
    lists = dense_l2.level_lists(n, L)
    for l in range(1, L + 1):
        fine = sorted(set(lists[l]) - set(lists[l - 1]))
        hl = h * 2 ** (L - l)
        np.testing.assert_allclose(out[fine], -alpha * hl ** 2, rtol=1e-12)


# --------------------------------------------------------------- invariants -

@pytest.mark.parametrize("shape", [(9, 9, 9), (10, 7, 6), (17, 5)])
def test_multilinear_fields_have_zero_coefficients(shape):
    # A field that is multilinear on the coarsest grid is in V_0 and is
    # reproduced exactly by every interpolant: all coefficients vanish and the
    # coarsest values are its samples.
    rng = np.random.default_rng(11)
    coords = [random_coords(rng, s) for s in shape]
    L = oracle.default_levels(shape)
    lists = [dense_l2.level_lists(s, L) for s in shape]
    # hat functions of the coarsest grid, combined multilinearly
    vals = rng.standard_normal([len(lists[k][0]) for k in range(len(shape))])
    u = vals
    for k in range(len(shape)):
        H = dense_l2.hats(coords[k][lists[k][0]], coords[k])
        u = np.moveaxis(np.tensordot(H, u, axes=([1], [k])), 0, k)
    out = oracle.decompose(u, coords, L)
    idx0 = np.ix_(*[np.array(lists[k][0]) for k in range(len(shape))])
    coarse = out[idx0].copy()
    rest = out.copy()
    rest[idx0] = 0.0
    assert np.abs(rest).max() <= 1e-13 * np.abs(u).max()
    np.testing.assert_allclose(coarse, vals, rtol=0, atol=1e-13 * np.abs(u).max())


def test_integer_bilinear_uniform_is_exact():
    shape = (17, 9, 9)
    z, y, x = np.meshgrid(*[np.arange(s, dtype=float) for s in shape], indexing="ij")
    u = 3 + 2 * x - y + 4 * z + x * y - 2 * y * z + x * z + x * y * z
    out = oracle.decompose(u)
    L = oracle.default_levels(shape)
    lists = [dense_l2.level_lists(s, L) for s in shape]
    idx0 = np.ix_(*[np.array(l[0]) for l in lists])
    rest = out.copy()
    rest[idx0] = 0.0
    assert np.count_nonzero(rest) == 0
    np.testing.assert_array_equal(out[idx0], u[idx0])


def test_linearity():
    rng = np.random.default_rng(5)
    shape = (9, 10, 7)
    coords = [random_coords(rng, s) for s in shape]
    a, b = rng.standard_normal(shape), rng.standard_normal(shape)
    lhs = oracle.decompose(2.5 * a - 0.75 * b, coords)
    rhs = 2.5 * oracle.decompose(a, coords) - 0.75 * oracle.decompose(b, coords)
    assert rel_linf(lhs, rhs) <= 1e-14


def test_separable_field_coarsest_is_tensor_product():
    rng = np.random.default_rng(9)
    shape = (17, 12, 9)
    coords = [random_coords(rng, s) for s in shape]
    L = oracle.default_levels(shape)
    us = [rng.standard_normal(s) for s in shape]
    u = np.einsum("i,j,k->ijk", *us)
    out = oracle.decompose(u, coords, L)
    lists = [dense_l2.level_lists(s, L) for s in shape]
    c1 = [oracle.decompose(us[k], [coords[k]], L)[lists[k][0]] for k in range(3)]
    expect = np.einsum("i,j,k->ijk", *c1)
    got = out[np.ix_(*[np.array(l[0]) for l in lists])]
    assert rel_linf(got, expect) <= 1e-13


@pytest.mark.parametrize("shape", [(65,), (33, 17), (9, 9, 9), (20, 13, 11), (7, 30)])
@pytest.mark.parametrize("kind", ["uniform", "stretched"])
def test_round_trip(shape, kind):
    rng = np.random.default_rng(len(shape) * 31 + shape[0])
    u = rng.standard_normal(shape)
    coords = None if kind == "uniform" else [stretched(s, 1.01) for s in shape]
    for L in {0, 1, oracle.default_levels(shape), oracle.max_levels(shape)}:
        c = oracle.decompose(u, coords, L)
        assert rel_linf(oracle.recompose(c, coords, L), u) <= 1e-13


def test_levels_zero_is_identity():
    u = np.random.default_rng(0).standard_normal((6, 7))
    np.testing.assert_array_equal(oracle.decompose(u, levels=0), u)


def test_invalid_arguments():
    with pytest.raises(ValueError):
        oracle.decompose(np.zeros((1, 5)))
    with pytest.raises(ValueError):
        oracle.decompose(np.zeros(9), levels=4)
    with pytest.raises(ValueError):
        oracle.decompose(np.zeros(5), coords=[np.array([0, 1, 1, 2, 3.0])])


def test_hierarchy_depths():
    assert oracle.default_levels((65, 65, 65)) == 5
    assert oracle.default_levels((513, 513, 513)) == 8
    assert oracle.default_levels((1000, 700, 300)) == 8
    assert oracle.max_levels((5,)) == 2
    assert oracle.default_levels((5,)) == 1
    lists = [dense_l2.level_lists(s, 8) for s in (1000, 700, 300)]
    assert [len(l[0]) for l in lists] == [5, 4, 3]
