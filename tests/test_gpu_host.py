"""Host-buffer entry points (mgr_decompose_host / mgr_recompose_host) against
the device-buffer operations on the same input.

Pinned host buffers take the pipelined operations.  Decomposition: the input
is copied in by slabs of planes, the finest level pass runs in parts as the
slabs arrive, and the planes a part finishes are copied back while the
coarser levels run.  Recomposition: the even planes (every coefficient of the
coarser levels) first, the odd planes in slabs that release parts of the
finest load-vector pass, the output copied back part by part behind the
finest interpolation.  Pageable or aliased host buffers, aliased device
buffers and small plans take the plain copy-compute-copy sequence.  Every path runs the same kernels on the same
data, so the host result must equal the device result bit for bit; the host
output is filled with NaN first, so a plane that is never copied back fails.
"""
import pytest

import paper_2105_12764_gb300 as mgr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

FORMS = {
    "fp64": (mgr.MGR_F64, mgr.MGR_PREC_NATIVE, torch.float64),
    "fp32": (mgr.MGR_F32, mgr.MGR_PREC_NATIVE, torch.float32),
    "mixed": (mgr.MGR_F32, mgr.MGR_PREC_MIXED, torch.float32),
}
# odd and even plane counts (an even count ends on a coarse plane with an odd
# index), 2^k+1 and other sizes, few and many z chunks in the finest level pass
SHAPES = [(257, 40, 40), (130, 33, 40), (100, 37, 29), (65, 65, 65), (33, 70, 66)]


@pytest.fixture(scope="module")
def ctx():
    return mgr.Context(0)


def field(shape, td, seed):
    g = torch.Generator().manual_seed(seed)
    return torch.randn(shape, dtype=torch.float64, generator=g).to(td)


def device_result(plan, host_in, op):
    x = host_in.cuda()
    y = torch.empty_like(x)
    ws = torch.empty(max(plan.workspace_bytes, 256), dtype=torch.uint8, device="cuda")
    (plan.decompose if op == "dec" else plan.recompose)(x, y, ws)
    torch.cuda.synchronize()
    return y.cpu()


def host_call(plan, op, host_in, host_out, din, dout, ws):
    (plan.decompose_host if op == "dec" else plan.recompose_host)(host_in, host_out, din, dout, ws,
                                                                 torch.cuda.current_stream())
    torch.cuda.synchronize()


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("pinned", [True, False])
def test_decompose_host_equals_device(ctx, form, shape, pinned):
    dtype, prec, td = FORMS[form]
    plan = mgr.Plan(ctx, shape, None, -1, dtype, prec)
    din = torch.empty(shape, dtype=td, device="cuda")
    dout = torch.empty_like(din)
    ws = torch.empty(max(plan.workspace_bytes, 256), dtype=torch.uint8, device="cuda")
    for rep in range(3):  # first call captures the graph; later calls replay it on new data
        hin = field(shape, td, 10 * rep + 1)
        hout = torch.full(shape, float("nan"), dtype=td)
        if pinned:
            hin, hout = hin.pin_memory(), hout.pin_memory()
        host_call(plan, "dec", hin, hout, din, dout, ws)
        want = device_result(plan, hin, "dec")
        assert torch.equal(hout, want), (form, shape, pinned, rep)
    plan.close()


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("pinned", [True, False])
def test_recompose_host_equals_device(ctx, form, shape, pinned):
    dtype, prec, td = FORMS[form]
    plan = mgr.Plan(ctx, shape, None, -1, dtype, prec)
    din = torch.empty(shape, dtype=td, device="cuda")
    dout = torch.empty_like(din)
    ws = torch.empty(max(plan.workspace_bytes, 256), dtype=torch.uint8, device="cuda")
    for rep in range(3):
        coef = device_result(plan, field(shape, td, 10 * rep + 2), "dec")
        hout = torch.full(shape, float("nan"), dtype=td)
        if pinned:
            coef, hout = coef.pin_memory(), hout.pin_memory()
        host_call(plan, "rec", coef, hout, din, dout, ws)
        want = device_result(plan, coef, "rec")
        assert torch.equal(hout, want), (form, shape, pinned, rep)
    plan.close()


@pytest.mark.parametrize("form", ["fp64", "fp32"])
def test_decompose_host_in_place_on_host(ctx, form):
    """host_out == host_in: the plain sequence."""
    dtype, prec, td = FORMS[form]
    shape = (257, 40, 40)
    plan = mgr.Plan(ctx, shape, None, -1, dtype, prec)
    din = torch.empty(shape, dtype=td, device="cuda")
    dout = torch.empty_like(din)
    ws = torch.empty(max(plan.workspace_bytes, 256), dtype=torch.uint8, device="cuda")
    src = field(shape, td, 7)
    want = device_result(plan, src, "dec")
    buf = src.clone().pin_memory()
    host_call(plan, "dec", buf, buf, din, dout, ws)
    assert torch.equal(buf, want)
    plan.close()


def test_decompose_host_same_device_buffer(ctx):
    """dev_in == dev_out (in place on the device): the plain sequence."""
    shape = (129, 40, 33)
    plan = mgr.Plan(ctx, shape, None, -1, mgr.MGR_F64)
    d = torch.empty(shape, dtype=torch.float64, device="cuda")
    ws = torch.empty(max(plan.workspace_bytes, 256), dtype=torch.uint8, device="cuda")
    hin = field(shape, torch.float64, 3).pin_memory()
    hout = torch.full(shape, float("nan"), dtype=torch.float64).pin_memory()
    host_call(plan, "dec", hin, hout, d, d, ws)
    x = hin.cuda()
    plan.decompose(x, x, ws)  # the in-place device operation (its own rounding order)
    torch.cuda.synchronize()
    assert torch.equal(hout, x.cpu())
    plan.close()


@pytest.mark.parametrize("shape", [(17, 17, 17), (1, 200, 150), (300, 2, 40)])
def test_decompose_host_plain_sequence_shapes(ctx, shape):
    """Plans the pipeline does not take (few planes, 2D, one coarse level)."""
    ndim_shape = tuple(n for n in shape if n > 1) if shape[0] == 1 else shape
    plan = mgr.Plan(ctx, ndim_shape, None, -1, mgr.MGR_F64)
    din = torch.empty(ndim_shape, dtype=torch.float64, device="cuda")
    dout = torch.empty_like(din)
    ws = torch.empty(max(plan.workspace_bytes, 256), dtype=torch.uint8, device="cuda")
    hin = field(ndim_shape, torch.float64, 5).pin_memory()
    hout = torch.full(ndim_shape, float("nan"), dtype=torch.float64).pin_memory()
    host_call(plan, "dec", hin, hout, din, dout, ws)
    assert torch.equal(hout, device_result(plan, hin, "dec"))
    plan.close()


@pytest.mark.parametrize("form", list(FORMS))
def test_host_round_trip(ctx, form):
    """decompose_host then recompose_host (the end-to-end path bench.py times)."""
    dtype, prec, td = FORMS[form]
    shape = (130, 33, 40)
    plan = mgr.Plan(ctx, shape, None, -1, dtype, prec)
    din = torch.empty(shape, dtype=td, device="cuda")
    dout = torch.empty_like(din)
    ws = torch.empty(max(plan.workspace_bytes, 256), dtype=torch.uint8, device="cuda")
    hin = field(shape, td, 11).pin_memory()
    hc = torch.empty_like(hin).pin_memory()
    hback = torch.full(shape, float("nan"), dtype=td).pin_memory()
    host_call(plan, "dec", hin, hc, din, dout, ws)
    host_call(plan, "rec", hc, hback, din, dout, ws)
    assert torch.equal(hc, device_result(plan, hin, "dec"))
    assert torch.equal(hback, device_result(plan, hc, "rec"))
    tol = 1e-13 if dtype == mgr.MGR_F64 else 1e-5
    err = float((hback.double() - hin.double()).abs().max() / hin.double().abs().max())
    assert err <= tol
    plan.close()
