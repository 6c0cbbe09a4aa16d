"""Pins of the oracle's linear quantization stage (Sec. V, lossy compression:
quantization and dequantization around the refactoring).  The paper does not
state the quantizer; the reading is uniform per-class bins
q_0 = 2 tau/(L+1), q_l = 2 tau/((L+1)(1 + |Z_l|_inf)), Z_l the level-l
correction operator, which bounds the recomposed field's max-norm error by tau.

* the operator norms behind the bins, against Z_l built independently from
  dense Gram matrices (dense_l2) on tiny grids;
* the guarantee |u - recompose(dequantize(quantize(decompose(u))))|_inf <= tau
  on 1D/2D/3D, uniform and stretched, dyadic and not;
* round-half-to-even, saturation, and |c - k q| <= q/2.
"""
import numpy as np
import pytest

import dense_l2
import oracle


def stretched(n, ratio=1.1):
    return np.concatenate([[0.0], np.cumsum(ratio ** np.arange(n - 1))])


def bins_by_dense(shape, coords, L, tau):
    d = len(shape)
    xs = [np.arange(shape[k], dtype=np.float64) if coords is None else coords[k] for k in range(d)]
    lists = [dense_l2.level_lists(shape[k], L) for k in range(d)]
    q = [2 * tau / (L + 1)]
    for l in range(1, L + 1):
        z = 1.0
        for k in range(d):
            Z = dense_l2.projection_operators(xs[k], lists[k][l], lists[k][l - 1])
            z *= np.abs(Z).sum(axis=1).max()
        q.append(2 * tau / ((L + 1) * (1 + z)))
    return np.array(q)


@pytest.mark.parametrize("shape,kind", [((5,), "uniform"), ((17,), "uniform"), ((24,), "stretched"),
                                        ((9, 9), "uniform"), ((11, 8), "stretched"), ((9, 7, 6), "stretched")])
def test_bins_against_dense_operators(shape, kind):
    coords = None if kind == "uniform" else [stretched(n) for n in shape]
    for L in range(0, oracle.max_levels(shape) + 1):
        got = oracle.quant_bins(shape, 0.25, coords, L)
        np.testing.assert_allclose(got, bins_by_dense(shape, coords, L, 0.25), rtol=1e-12, atol=0)


def test_bins_scale_with_tau_and_level_count():
    b1 = oracle.quant_bins((33, 33), 1.0)
    np.testing.assert_allclose(oracle.quant_bins((33, 33), 1e-4), 1e-4 * b1, rtol=1e-14)
    assert b1[0] == pytest.approx(2.0 / len(b1))
    assert np.all(b1[1:] < b1[0])  # every correction operator has norm > 0


@pytest.mark.parametrize("shape,kind", [((65,), "uniform"), ((40,), "stretched"), ((33, 17), "uniform"),
                                        ((20, 31), "stretched"), ((17, 9, 13), "uniform"), ((12, 10, 9), "stretched")])
@pytest.mark.parametrize("tau", [1e-1, 1e-3])
def test_error_guarantee(shape, kind, tau):
    rng = np.random.default_rng(len(shape) * 7 + int(-np.log10(tau)))
    coords = None if kind == "uniform" else [stretched(n) for n in shape]
    u = rng.standard_normal(shape) * 3.0
    L = oracle.default_levels(shape)
    offs = oracle.class_offsets(shape, L)
    bins = oracle.quant_bins(shape, tau, coords, L)
    packed = oracle.pack_classes(oracle.decompose(u, coords, L), L)
    codes, sat = oracle.quantize(packed, bins, offs)
    assert sat == 0
    back = oracle.recompose_classes(oracle.dequantize(codes, bins, offs), shape, None, coords, L)
    err = np.abs(back - u).max()
    assert err <= tau * (1 + 1e-9)
    assert err >= 1e-3 * tau  # the bins are not vanishingly small


def test_rounding_and_saturation():
    bins = np.array([0.5, 0.25])
    offs = np.array([0, 4, 8])
    c = np.array([0.25, 0.75, -0.25, 1.25,      # class 0: c/q = 0.5, 1.5, -0.5, 2.5
                  1e12, -1e12, 0.3, -0.3])     # class 1: saturated, saturated, 1.2, -1.2
    codes, sat = oracle.quantize(c, bins, offs)
    assert codes.tolist() == [0, 2, 0, 2, 2147483647, -2147483647, 1, -1]
    assert sat == 2
    rng = np.random.default_rng(0)
    c = rng.standard_normal(8)
    codes, _ = oracle.quantize(c, bins, offs)
    deq = oracle.dequantize(codes, bins, offs)
    assert np.all(np.abs(deq[:4] - c[:4]) <= 0.25 + 1e-15)
    assert np.all(np.abs(deq[4:] - c[4:]) <= 0.125 + 1e-15)


def test_float32_decision_precision():
    """The rounding decision in FP32 uses c*(1/q) rounded to FP32, as a kernel
    computing in FP32 does."""
    q = 3.0
    c = np.float32(np.float32(1.5) * np.float32(3.0))  # c*(1/q) rounds to exactly 1.5 in FP32
    codes64, _ = oracle.quantize(np.array([c], dtype=np.float64), np.array([q]), np.array([0, 1]), np.float64)
    codes32, _ = oracle.quantize(np.array([c], dtype=np.float32), np.array([q]), np.array([0, 1]), np.float32)
    assert codes32[0] == 2  # half to even of 1.5 in FP32
    assert codes64[0] in (1, 2)
