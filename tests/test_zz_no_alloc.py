"""mgr_decompose_noalloc: the decomposition entry point for callers that
cannot allocate device memory (their memory belongs to another allocator,
they only hold their input and output buffers, or an allocation would stall
their path).  Its workspace is a fixed scratch area in the library's device
image; this checks, through the C ABI, that two calls in a row give the same
output as mgr_decompose with a caller workspace, and that fields too large
for the area are refused."""
import ctypes

import numpy as np
import pytest

import paper_2105_12764_gb300 as mgr
from gpu_util import rel_linf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def noalloc(plan, x, y):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return mgr.lib.mgr_decompose_noalloc(plan.handle, x.data_ptr(), y.data_ptr(), stream)


@pytest.mark.parametrize("shape,dtype,coords", [((65, 65, 65), mgr.MGR_F64, False),
                                                ((100, 129, 90), mgr.MGR_F32, True),
                                                ((300, 257), mgr.MGR_F64, True)])
def test_noalloc_matches_decompose_twice(shape, dtype, coords):
    ctx = mgr.Context(0)
    cs = [np.concatenate([[0.0], np.cumsum(1.01 ** np.arange(n - 1))]) for n in shape] if coords else None
    plan = mgr.Plan(ctx, shape, cs, -1, dtype)
    assert plan.workspace_bytes <= mgr.MGR_NOALLOC_SCRATCH_BYTES
    td = torch.float64 if dtype == mgr.MGR_F64 else torch.float32
    g = torch.Generator(device="cuda").manual_seed(3)
    x = torch.randn(shape, dtype=td, device="cuda", generator=g)
    ref = torch.empty_like(x)
    ws = torch.empty(max(plan.workspace_bytes, 256), dtype=torch.uint8, device="cuda")
    plan.decompose(x, ref, ws)
    tol = 1e-12 if dtype == mgr.MGR_F64 else 1e-6
    for _ in range(2):
        y = torch.full_like(x, float("nan"))
        assert noalloc(plan, x, y) == mgr.MGR_OK
        torch.cuda.synchronize()
        assert rel_linf(y.cpu().numpy(), ref.cpu().numpy()) <= tol
    plan.close()
    ctx.close()


def test_noalloc_refuses_fields_beyond_the_scratch_area():
    ctx = mgr.Context(0)
    plan = mgr.Plan(ctx, (257, 257, 257), None, -1, mgr.MGR_F64)
    assert plan.workspace_bytes > mgr.MGR_NOALLOC_SCRATCH_BYTES
    x = torch.zeros((257, 257, 257), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    assert noalloc(plan, x, y) == mgr.MGR_EINVAL
    plan.close()
    ctx.close()
