"""Out-of-bounds write detection without a sanitizer: every operation runs on
buffers carved out of larger allocations with guard bands before and after
(input, output, workspace), the guards filled with a byte pattern; after the
operation every guard byte must be unchanged.  Covers the tiled level pass,
the solves, the interpolation, the coarse-level kernel, the class-packed,
quantized and 4D forms, in place and out of place, on shapes with ragged
tiles and keep-last ends."""
import numpy as np
import pytest

import paper_2105_12764_gb300 as mgr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

GUARD = 4096  # bytes on each side (keeps 256-byte alignment of the payload)
PATTERN = 0xA5


@pytest.fixture(scope="module")
def ctx():
    return mgr.Context(0)


class Guarded:
    def __init__(self, nbytes):
        self.n = int(nbytes)
        self.raw = torch.full((self.n + 2 * GUARD,), PATTERN, dtype=torch.uint8, device="cuda")

    def ptr(self):
        return self.raw.data_ptr() + GUARD

    def view(self, dtype, shape):
        t = self.raw[GUARD:GUARD + self.n].view(dtype)
        return t.view(shape)

    def intact(self):
        head = self.raw[:GUARD]
        tail = self.raw[GUARD + self.n:]
        return bool((head == PATTERN).all().item()) and bool((tail == PATTERN).all().item())


def run_case(ctx, shape, dtype, prec=mgr.MGR_PREC_NATIVE, levels=-1, inplace=False, coords=None):
    td = torch.float64 if dtype == mgr.MGR_F64 else torch.float32
    es = 8 if dtype == mgr.MGR_F64 else 4
    plan = mgr.Plan(ctx, shape, coords, levels, dtype, prec)
    n = int(np.prod(shape))
    try:
        a, b, ws = Guarded(n * es), Guarded(n * es), Guarded(max(plan.workspace_bytes, 256))
        x = a.view(td, shape)
        x.copy_(torch.randn(shape, dtype=torch.float64, device="cuda").to(td))
        out = a if inplace else b
        plan.decompose(a.ptr(), out.ptr(), ws.ptr())
        plan.recompose(out.ptr(), out.ptr() if inplace else a.ptr(), ws.ptr())
        torch.cuda.synchronize()
        assert a.intact() and b.intact() and ws.intact(), (shape, dtype, inplace)
        if len(shape) <= 3:
            c = Guarded(n * es)
            plan.decompose_packed(a.ptr(), c.ptr(), ws.ptr())
            L = plan.levels
            for k in sorted({1, max(1, L), L + 1}):
                plan.recompose_packed(c.ptr(), k, b.ptr(), ws.ptr())
            q = Guarded(n * 4)
            sat = torch.zeros(1, dtype=torch.int64, device="cuda")
            plan.decompose_quantized(a.ptr(), q.ptr(), 1e-3, ws.ptr(), sat)
            plan.recompose_dequantized(q.ptr(), L + 1, 1e-3, b.ptr(), ws.ptr())
            plan.pack_classes(b.ptr(), c.ptr())
            plan.unpack_classes(c.ptr(), L + 1, b.ptr())
            torch.cuda.synchronize()
            assert c.intact() and q.intact() and a.intact() and b.intact() and ws.intact(), shape
    finally:
        plan.close()


SHAPES = [(2,), (7,), (513,), (1000,), (20001,), (17, 17), (65, 40), (257, 300), (3, 3, 3), (9, 6, 7),
          (33, 20, 37), (29, 28, 60), (58, 60, 121), (129, 129, 129), (65, 70, 33)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", [mgr.MGR_F64, mgr.MGR_F32])
def test_guards(ctx, shape, dtype):
    run_case(ctx, shape, dtype)


@pytest.mark.parametrize("shape", [(65, 40), (33, 20, 37), (129, 129, 129)])
def test_guards_inplace_and_mixed(ctx, shape):
    run_case(ctx, shape, mgr.MGR_F64, inplace=True)
    run_case(ctx, shape, mgr.MGR_F32, mgr.MGR_PREC_MIXED)
    run_case(ctx, shape, mgr.MGR_F32, mgr.MGR_PREC_MIXED, inplace=True)


@pytest.mark.parametrize("shape", [(5, 9, 6, 7), (8, 17, 20, 33), (17, 33, 29, 60)])
@pytest.mark.parametrize("dtype", [mgr.MGR_F64, mgr.MGR_F32])
def test_guards_4d(ctx, shape, dtype):
    run_case(ctx, shape, dtype)


def test_guards_partial_depths(ctx):
    for L in range(0, 4):
        run_case(ctx, (33, 20, 37), mgr.MGR_F64, levels=L)
