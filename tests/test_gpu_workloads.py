"""Full-size parity: the bench workloads through the C ABI vs the FP64 oracle.

513^3 k^-5/3 field, full hierarchy (8 levels), in the launch configuration
bench.py times (same plan, graph-replayed launches): FP64 vs oracle <= 1e-12,
round trip <= 1e-13; FP32 and mixed <= 1e-5.
1000 x 700 x 300 stretched (1.01 per cell): FP64 <= 1e-12 (round trip
<= 1e-13), FP32 and mixed <= 1e-5.
Fused quantization at 513^3: the codes equal the oracle's quantizer applied to
the oracle's own class-packed decomposition, except where the oracle's
rounding decision lies within the coefficients' error of a half-integer.
Every output element is compared (the oracle computes the whole field).
"""
import numpy as np
import pytest

import oracle
import paper_2105_12764_gb300 as mgr
from gpu_util import Runner, rel_linf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def ctx():
    return mgr.Context(0)


@pytest.fixture(scope="module")
def grf513_field():
    from paper_2105_12764_gb300 import synth

    return synth.workload("grf513")[0]


@pytest.fixture(scope="module")
def grf513_oracle(grf513_field):
    return oracle.decompose(grf513_field)


def test_grf513_fp64_full(ctx, grf513_field, grf513_oracle):
    r = Runner(ctx, grf513_field.shape, None, -1, mgr.MGR_F64)
    try:
        got = r.decompose(grf513_field)
        assert rel_linf(got, grf513_oracle) <= 1e-12
        back = r.recompose(got)
        assert rel_linf(back, grf513_field) <= 1e-13
    finally:
        r.close()


@pytest.mark.parametrize("prec", [mgr.MGR_PREC_NATIVE, mgr.MGR_PREC_MIXED])
def test_grf513_fp32_forms_full(ctx, grf513_field, prec):
    u32 = grf513_field.astype(np.float32)
    ref = oracle.decompose(u32.astype(np.float64))
    r = Runner(ctx, grf513_field.shape, None, -1, mgr.MGR_F32, prec)
    try:
        got = r.decompose(u32)
        err = rel_linf(got, ref)
        assert err <= 1e-5, err
        back = r.recompose(got)
        assert rel_linf(back, u32) <= 1e-5
    finally:
        r.close()


@pytest.fixture(scope="module")
def stretched_field():
    from paper_2105_12764_gb300 import synth

    return synth.workload("bumps_stretched_1000x700x300")


@pytest.fixture(scope="module")
def stretched_oracle32(stretched_field):
    u, coords = stretched_field
    return oracle.decompose(u.astype(np.float32).astype(np.float64), coords)


@pytest.mark.parametrize("prec", [mgr.MGR_PREC_MIXED, mgr.MGR_PREC_NATIVE])
def test_stretched_1000x700x300_fp32_forms_full(ctx, stretched_field, stretched_oracle32, prec):
    u, coords = stretched_field
    u32 = u.astype(np.float32)
    r = Runner(ctx, u32.shape, coords, -1, mgr.MGR_F32, prec)
    try:
        assert r.plan.levels == 8
        got = r.decompose(u32)
        err = rel_linf(got, stretched_oracle32)
        assert err <= 1e-5, err
        back = r.recompose(got)
        assert rel_linf(back, u32) <= 1e-5
    finally:
        r.close()


def test_stretched_1000x700x300_fp64_full(ctx, stretched_field):
    u, coords = stretched_field
    ref = oracle.decompose(u, coords)
    r = Runner(ctx, u.shape, coords, -1, mgr.MGR_F64)
    try:
        assert r.plan.levels == 8
        got = r.decompose(u)
        err = rel_linf(got, ref)
        assert err <= 1e-12, err
        del ref
        back = r.recompose(got)
        assert rel_linf(back, u) <= 1e-13
    finally:
        r.close()


def test_grf513_fp64_class_packed_and_progressive_full(ctx, grf513_field, grf513_oracle):
    """The class-packed form at the bench size: equal to the oracle's classes; every
    class recomposes the field; class 0 alone gives the coarsest interpolant."""
    shape = grf513_field.shape
    plan = mgr.Plan(ctx, shape, None, -1, mgr.MGR_F64)
    L = plan.levels
    x = torch.from_numpy(grf513_field).cuda()
    pk = torch.empty(x.numel(), dtype=x.dtype, device="cuda")
    y = torch.empty_like(x)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    try:
        plan.decompose_packed(x, pk, ws)
        torch.cuda.synchronize()
        want = oracle.pack_classes(grf513_oracle, L)
        assert rel_linf(pk.cpu().numpy(), want) <= 1e-12
        plan.recompose_packed(pk, L + 1, y, ws)
        torch.cuda.synchronize()
        assert rel_linf(y.cpu().numpy(), grf513_field) <= 1e-13
        # prefix of the first L classes (finest class dropped), against the oracle on
        # its own classes
        plan.recompose_packed(pk, L, y, ws)
        torch.cuda.synchronize()
        prog = oracle.recompose_classes(want, shape, L, None, L)
        assert rel_linf(y.cpu().numpy(), prog) <= 1e-12
    finally:
        plan.close()


def test_grf513_fp64_quantized_full(ctx, grf513_field):
    """Fused quantization at the bench size: the recomposed field is within tau."""
    plan = mgr.Plan(ctx, grf513_field.shape, None, -1, mgr.MGR_F64)
    x = torch.from_numpy(grf513_field).cuda()
    codes = torch.empty(x.numel(), dtype=torch.int32, device="cuda")
    y = torch.empty_like(x)
    sat = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    try:
        span = float(grf513_field.max() - grf513_field.min())
        for rel in (1e-2, 1e-5):
            tau = rel * span
            plan.decompose_quantized(x, codes, tau, ws, sat)
            plan.recompose_dequantized(codes, plan.levels + 1, tau, y, ws)
            torch.cuda.synchronize()
            assert int(sat.item()) == 0
            err = float((y - x).abs().max().item())
            assert err <= tau * (1 + 1e-9), (rel, err, tau)
    finally:
        plan.close()


def test_grf513_fp64_quantized_codes_match_oracle(ctx, grf513_field, grf513_oracle):
    """Codes at the bench size against the oracle end to end: the oracle's quantizer
    on the oracle's own class-packed coefficients.  A code may differ (by one) only
    where the oracle's value c/q lies within the coefficients' GPU-vs-oracle error
    of a half-integer; everywhere else the codes are equal."""
    shape = grf513_field.shape
    plan = mgr.Plan(ctx, shape, None, -1, mgr.MGR_F64)
    L = plan.levels
    offs = plan.class_offsets()
    x = torch.from_numpy(grf513_field).cuda()
    pk = torch.empty(x.numel(), dtype=x.dtype, device="cuda")
    codes = torch.empty(x.numel(), dtype=torch.int32, device="cuda")
    sat = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    try:
        want_c = oracle.pack_classes(grf513_oracle, L)
        plan.decompose_packed(x, pk, ws)
        torch.cuda.synchronize()
        gpu_c = pk.cpu().numpy()
        assert rel_linf(gpu_c, want_c) <= 1e-12
        span = float(grf513_field.max() - grf513_field.min())
        for rel in (1e-2, 1e-4):
            tau = rel * span
            bins = np.array(plan.quant_bins(tau))
            np.testing.assert_allclose(bins, oracle.quant_bins(shape, tau, None, L), rtol=1e-12, atol=0)
            sat.zero_()
            plan.decompose_quantized(x, codes, tau, ws, sat)
            torch.cuda.synchronize()
            assert int(sat.item()) == 0
            got = codes.cpu().numpy().astype(np.int64)
            want, wsat = oracle.quantize(want_c, bins, offs, np.float64)
            assert wsat == 0
            amb = near_half(want_c, gpu_c, bins, offs)
            diff = got != want
            assert not np.any(diff & ~amb), f"{int(np.sum(diff & ~amb))} codes differ away from a rounding tie"
            assert np.all(np.abs(got - want) <= 1)
            assert amb.mean() < 1e-3
    finally:
        plan.close()


def near_half(c_ref, c_gpu, bins, offs):
    """Where the oracle's rounding decision c_ref/q lies within the coefficients'
    measured GPU-vs-oracle error (per class, plus a few ulps) of a half-integer."""
    out = np.zeros(c_ref.shape, dtype=bool)
    eps = np.finfo(np.float64).eps
    for l in range(len(bins)):
        a, b = int(offs[l]), int(offs[l + 1])
        q = float(bins[l])
        t = np.abs(c_ref[a:b] / q)
        err = float(np.abs(c_gpu[a:b] - c_ref[a:b]).max()) / q if b > a else 0.0
        out[a:b] = np.abs(t - np.floor(t) - 0.5) <= err + 8 * eps * np.maximum(1.0, t)
    return out
