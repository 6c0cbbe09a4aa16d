"""GPU parity of the fused linear quantization (Sec. V, the quantization stage
around the refactoring) against the FP64 oracle.

* bin widths (mgr_quant_bins, from the plan's own operators) = oracle bins  <= 1e-12
* codes of mgr_decompose_quantized = round-half-even(c * (1/q)) of the same
  coefficients, the decision in the kernel's precision: equal except at ties
* end to end: the codes equal the oracle's quantizer applied to the oracle's
  own class-packed decomposition, except where the oracle's rounding decision
  lies within the coefficients' GPU-vs-oracle error of a half-integer
* mgr_recompose_dequantized of given codes = oracle recompose of the
  dequantized classes                                                     <= 1e-12 (FP64), 1e-5 (FP32)
* the guarantee |u - recompose(codes)|_inf <= tau (+ rounding)
* saturation counting, invalid arguments, the zero-level hierarchy
"""
import numpy as np
import pytest

import oracle
import paper_2105_12764_gb300 as mgr
from gpu_util import np_dtype, rel_linf, torch_dtype

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def ctx():
    return mgr.Context(0)


def random_coords(rng, n):
    return np.concatenate([[0.0], np.cumsum(rng.uniform(0.2, 3.0, n - 1))])


class Q:
    def __init__(self, ctx, shape, coords=None, levels=-1, dtype=mgr.MGR_F64, prec=mgr.MGR_PREC_NATIVE):
        self.plan = mgr.Plan(ctx, shape, coords, levels, dtype, prec)
        self.shape = tuple(shape)
        self.td, self.nd = torch_dtype(dtype), np_dtype(dtype)
        n = int(np.prod(shape))
        self.ws = torch.empty(max(self.plan.workspace_bytes, 256), dtype=torch.uint8, device="cuda")
        self.x = torch.empty(self.shape, dtype=self.td, device="cuda")
        self.p = torch.empty(n, dtype=self.td, device="cuda")
        self.k = torch.empty(n, dtype=torch.int32, device="cuda")
        self.y = torch.empty(self.shape, dtype=self.td, device="cuda")
        self.sat = torch.zeros(1, dtype=torch.int64, device="cuda")

    def load(self, u):
        self.x.copy_(torch.from_numpy(np.ascontiguousarray(u, dtype=self.nd)))

    def coefficients(self):
        self.plan.decompose_packed(self.x, self.p, self.ws)
        torch.cuda.synchronize()
        return self.p.cpu().numpy()

    def quantize(self, tau):
        self.sat.zero_()
        self.plan.decompose_quantized(self.x, self.k, tau, self.ws, self.sat)
        torch.cuda.synchronize()
        return self.k.cpu().numpy().astype(np.int64), int(self.sat.item())

    def recompose(self, codes, k, tau):
        self.k.copy_(torch.from_numpy(np.asarray(codes, dtype=np.int32)))
        self.plan.recompose_dequantized(self.k, k, tau, self.y, self.ws)
        torch.cuda.synchronize()
        return self.y.cpu().numpy()

    def close(self):
        self.plan.close()


def ties(c, bins, offs, prec):
    """Positions whose rounding decision is within a few ulps of a half-integer."""
    out = np.zeros(c.shape, dtype=bool)
    eps = np.finfo(prec).eps
    for l in range(len(bins)):
        a, b = int(offs[l]), int(offs[l + 1])
        t = np.abs(c[a:b].astype(np.float64) / float(bins[l]))
        out[a:b] = np.abs(t - np.floor(t) - 0.5) <= 8 * eps * np.maximum(1.0, t)
    return out


def check_codes(r, codes, c, bins, offs, prec, class0_prec):
    want, _ = oracle.quantize(c, bins, offs, prec)
    w0, _ = oracle.quantize(c[: offs[1]], bins[:1], offs[:2], class0_prec)
    want[: offs[1]] = w0
    diff = codes != want
    amb = ties(c, bins, offs, prec)
    if class0_prec != prec:
        # class 0 is rounded from the solve-precision value, which the FP32
        # coefficient array only holds rounded: allow one code of difference
        amb[: offs[1]] |= np.abs(codes[: offs[1]] - want[: offs[1]]) <= 1
    assert not np.any(diff & ~amb), f"{int(np.sum(diff & ~amb))} codes differ away from ties"
    assert np.all(np.abs(codes - want) <= 1)


@pytest.mark.parametrize("shape,kind", [((257,), "uniform"), ((100,), "random"), ((65, 70), "random"),
                                        ((33, 33, 33), "uniform"), ((29, 28, 60), "random"),
                                        ((58, 60, 121), "uniform"), ((12, 29, 59), "random")])
def test_fp64(ctx, shape, kind):
    rng = np.random.default_rng(sum(shape))
    coords = None if kind == "uniform" else [random_coords(rng, s) for s in shape]
    u = rng.standard_normal(shape) * 2.0
    r = Q(ctx, shape, coords)
    try:
        L = r.plan.levels
        offs = r.plan.class_offsets()
        r.load(u)
        c = r.coefficients()
        for tau in (1e-2, 1e-5):
            bins = np.array(r.plan.quant_bins(tau))
            np.testing.assert_allclose(bins, oracle.quant_bins(shape, tau, coords, L), rtol=1e-12, atol=0)
            codes, sat = r.quantize(tau)
            assert sat == 0
            check_codes(r, codes, c, bins, offs, np.float64, np.float64)
            deq = oracle.dequantize(codes, bins, offs)
            for k in sorted({1, L, L + 1}):
                got = r.recompose(codes, k, tau)
                want = oracle.recompose_classes(deq, shape, k, coords, L)
                assert rel_linf(got, want) <= 1e-12
                if k == L + 1:
                    err = np.abs(got - u).max()
                    assert err <= tau * (1 + 1e-9) + 1e-12 * np.abs(u).max()
    finally:
        r.close()


@pytest.mark.parametrize("form", ["fp32", "mixed"])
@pytest.mark.parametrize("shape", [(65, 70), (33, 40, 71)])
def test_fp32_forms(ctx, form, shape):
    rng = np.random.default_rng(5)
    coords = [random_coords(rng, s) for s in shape]
    u = (rng.standard_normal(shape) * 2.0).astype(np.float32)
    prec = mgr.MGR_PREC_MIXED if form == "mixed" else mgr.MGR_PREC_NATIVE
    r = Q(ctx, shape, coords, -1, mgr.MGR_F32, prec)
    try:
        L = r.plan.levels
        offs = r.plan.class_offsets()
        r.load(u)
        c = r.coefficients()
        tau = 1e-2
        bins = np.array(r.plan.quant_bins(tau))
        np.testing.assert_allclose(bins, oracle.quant_bins(shape, tau, coords, L), rtol=1e-12, atol=0)
        codes, sat = r.quantize(tau)
        assert sat == 0
        check_codes(r, codes, c, bins, offs, np.float32, np.float64 if form == "mixed" else np.float32)
        deq = oracle.dequantize(codes, bins, offs)
        got = r.recompose(codes, L + 1, tau)
        assert rel_linf(got, oracle.recompose_classes(deq, shape, None, coords, L)) <= 1e-5
        u64 = u.astype(np.float64)
        assert np.abs(got - u64).max() <= tau * (1 + 1e-6) + 1e-5 * np.abs(u64).max()
    finally:
        r.close()


def near_half(c_ref, c_gpu, bins, offs, prec, slack0=0.0):
    """Mask of the codes whose rounding decision may legitimately differ: the
    oracle's value t = c_ref/q (taken in `prec`) lies within the per-class
    GPU-vs-oracle coefficient error (plus a few ulps of t) of a half-integer.
    slack0 widens class 0 by an absolute amount (the mixed form rounds class 0
    from an FP64 value the FP32 output holds only rounded)."""
    out = np.zeros(c_ref.shape, dtype=bool)
    eps = float(np.finfo(prec).eps)
    for l in range(len(bins)):
        a, b = int(offs[l]), int(offs[l + 1])
        if b <= a:
            continue
        q = float(bins[l])
        t = np.abs(c_ref[a:b] / q)
        err = (float(np.abs(c_gpu[a:b].astype(np.float64) - c_ref[a:b]).max()) + (slack0 if l == 0 else 0.0)) / q
        out[a:b] = np.abs(t - np.floor(t) - 0.5) <= err + 8 * eps * np.maximum(1.0, t)
    return out


@pytest.mark.parametrize("form", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("shape,kind", [((129, 100), "stretched"), ((45, 52, 61), "random"),
                                        ((65, 65, 65), "uniform"), ((31, 70, 129), "stretched")])
def test_codes_match_oracle_end_to_end(ctx, form, shape, kind):
    rng = np.random.default_rng(len(shape) * 100 + shape[-1])
    if kind == "uniform":
        coords = None
    elif kind == "random":
        coords = [random_coords(rng, s) for s in shape]
    else:
        coords = [np.concatenate([[0.0], np.cumsum(1.01 ** np.arange(s - 1))]) for s in shape]
    dtype = mgr.MGR_F64 if form == "fp64" else mgr.MGR_F32
    prec = mgr.MGR_PREC_MIXED if form == "mixed" else mgr.MGR_PREC_NATIVE
    u = rng.standard_normal(shape) * 2.0
    if dtype == mgr.MGR_F32:
        u = u.astype(np.float32)
    r = Q(ctx, shape, coords, -1, dtype, prec)
    try:
        L = r.plan.levels
        offs = r.plan.class_offsets()
        c_ref = oracle.pack_classes(oracle.decompose(u.astype(np.float64), coords, L), L)
        r.load(u)
        c_gpu = r.coefficients()
        tol = 1e-12 if form == "fp64" else 1e-5
        assert rel_linf(c_gpu, c_ref) <= tol
        span = float(u.max() - u.min())
        for rel in (1e-2, 1e-4):
            tau = rel * span
            bins = np.array(r.plan.quant_bins(tau))
            codes, sat = r.quantize(tau)
            assert sat == 0
            p = np.float64 if form == "fp64" else np.float32
            want, _ = oracle.quantize(c_ref, bins, offs, p)
            slack0 = 0.0
            if form != "fp32":
                w0, _ = oracle.quantize(c_ref[: offs[1]], bins[:1], offs[:2], np.float64)
                want[: offs[1]] = w0
                if form == "mixed":
                    slack0 = float(np.abs(c_ref[: offs[1]]).max()) * float(np.finfo(np.float32).eps)
            amb = near_half(c_ref, c_gpu, bins, offs, p, slack0)
            diff = codes != want
            assert not np.any(diff & ~amb), f"{int(np.sum(diff & ~amb))} codes differ away from a rounding tie"
            assert np.all(np.abs(codes - want) <= 1)
            # the mask stays a small part of the codes: within FP64 error of a tie is rare;
            # FP32 coefficients carry ~1e-7 relative error, a few percent of a bin at tau = 1e-4
            assert amb.mean() < (1e-3 if form == "fp64" else 0.1)
    finally:
        r.close()


def test_saturation_is_counted(ctx):
    shape = (33, 34, 35)
    r = Q(ctx, shape)
    try:
        u = np.random.default_rng(1).standard_normal(shape) * 1e9
        r.load(u)
        codes, sat = r.quantize(1e-3)
        assert sat > 0
        assert np.abs(codes).max() == 2147483647
        r.load(u * 1e-9)
        _, sat = r.quantize(1e-3)
        assert sat == 0
    finally:
        r.close()


def test_tolerance_is_part_of_the_replayed_graph(ctx):
    shape = (40, 41, 42)
    r = Q(ctx, shape)
    try:
        r.load(np.random.default_rng(2).standard_normal(shape))
        k1, _ = r.quantize(1e-2)
        k2, _ = r.quantize(1e-3)
        k1b, _ = r.quantize(1e-2)
        np.testing.assert_array_equal(k1, k1b)
        assert np.abs(k2).max() > 5 * np.abs(k1).max()
    finally:
        r.close()


def test_levels_zero(ctx):
    shape = (6, 7)
    r = Q(ctx, shape, None, 0)
    try:
        u = np.random.default_rng(3).standard_normal(shape)
        r.load(u)
        tau = 1e-3
        bins = r.plan.quant_bins(tau)
        assert bins == [2 * tau]
        codes, sat = r.quantize(tau)
        np.testing.assert_array_equal(codes, np.rint(u.ravel() * (1.0 / (2 * tau))).astype(np.int64))
        got = r.recompose(codes, 1, tau)
        assert np.abs(got - u).max() <= tau * (1 + 1e-12)
    finally:
        r.close()


def test_invalid_arguments(ctx):
    shape = (17, 18, 19)
    r = Q(ctx, shape)
    L = r.plan.levels
    try:
        for tau in (0.0, -1.0, float("nan")):
            with pytest.raises(mgr.MgrError) as ei:
                r.plan.decompose_quantized(r.x, r.k, tau, r.ws)
            assert ei.value.code == mgr.MGR_EINVAL
            with pytest.raises(mgr.MgrError) as ei:
                r.plan.quant_bins(tau)
            assert ei.value.code == mgr.MGR_EINVAL
        for k in (0, L + 2):
            with pytest.raises(mgr.MgrError) as ei:
                r.plan.recompose_dequantized(r.k, k, 1e-3, r.y, r.ws)
            assert ei.value.code == mgr.MGR_EINVAL
        # codes overlapping the field
        with pytest.raises(mgr.MgrError) as ei:
            r.plan.decompose_quantized(r.x, r.x, 1e-3, r.ws)
        assert ei.value.code == mgr.MGR_EINVAL
    finally:
        r.close()
