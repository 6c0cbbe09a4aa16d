"""Failure handling with host-side fault injection (MGR_FAULT_INJECT): device
allocations that fail, operations that fail before any launch, admission that
refuses.  No GPU fault is involved: every injected failure happens on the host
before work reaches the device.  After each failure the library stays usable
and later results are correct."""
import os

import numpy as np
import pytest

import oracle
import paper_2105_12764_gb300 as mgr
from gpu_util import rel_linf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


class inject:
    def __init__(self, what):
        self.what = what

    def __enter__(self):
        os.environ["MGR_FAULT_INJECT"] = self.what

    def __exit__(self, *a):
        os.environ.pop("MGR_FAULT_INJECT", None)


@pytest.fixture(scope="module")
def ctx():
    return mgr.Context(0, mem_budget_bytes=4 << 30)


def field(shape, seed=0):
    return torch.from_numpy(np.random.default_rng(seed).standard_normal(shape)).cuda()


def test_single_field_launch_failure(ctx):
    shape = (33, 20, 37)
    plan = mgr.Plan(ctx, shape, None, -1, mgr.MGR_F64)
    x, y = field(shape), torch.empty(shape, dtype=torch.float64, device="cuda")
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    with inject("launch"):
        with pytest.raises(mgr.MgrError) as ei:
            plan.decompose(x, y, ws)
        assert ei.value.code == mgr.MGR_ECUDA
    plan.decompose(x, y, ws)
    torch.cuda.synchronize()
    assert rel_linf(y.cpu().numpy(), oracle.decompose(x.cpu().numpy())) <= 1e-12
    plan.close()


@pytest.mark.parametrize("what,code", [("alloc", mgr.MGR_ENOMEM), ("launch", mgr.MGR_ECUDA),
                                       ("admit", mgr.MGR_EBUDGET)])
def test_serving_failures(ctx, what, code):
    shape = (40, 41, 42)
    plan = mgr.Plan(ctx, shape, None, -1, mgr.MGR_F64)
    x = field(shape, 1)
    srv = mgr.Server(ctx, slots=2, streams=2)
    try:
        with inject(what):
            rid = srv.enqueue(mgr.MGR_OP_DECOMPOSE, plan, inp=x, keep_resident=1)
            rc, res = srv.wait(rid)
            assert res["status"] == code
        st = srv.stats()
        assert st["used_bytes"] == 0 and st["running"] == 0 and st["resident"] == 0
        # the server keeps serving
        rid = srv.enqueue(mgr.MGR_OP_DECOMPOSE, plan, inp=x, keep_resident=1)
        rc, res = srv.wait(rid)
        assert res["status"] == mgr.MGR_OK
        out = torch.empty_like(x)
        srv.read(res["handle"], out, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert rel_linf(out.cpu().numpy(), oracle.decompose(x.cpu().numpy())) <= 1e-12
        srv.release(res["handle"])
    finally:
        srv.stop()
        plan.close()


def test_batch_failures(ctx):
    shapes = [(17, 19), (23, 21, 20), (30, 31)]
    plans = [mgr.Plan(ctx, s, None, -1, mgr.MGR_F32) for s in shapes]
    xs = [field(s, i).float() for i, s in enumerate(shapes)]
    ys = [torch.empty_like(x) for x in xs]
    reqs = [(mgr.MGR_OP_DECOMPOSE, p, x, y) for p, x, y in zip(plans, xs, ys)]
    with inject("alloc"):
        with pytest.raises(mgr.MgrError) as ei:
            ctx.batch_submit(reqs)
        assert ei.value.code == mgr.MGR_ENOMEM
    with inject("launch"):
        with pytest.raises(mgr.MgrError) as ei:
            ctx.batch_submit(reqs)
        assert ei.value.code == mgr.MGR_ECUDA
    t = ctx.batch_submit(reqs)
    rc, n = ctx.batch_poll(t)
    assert rc == mgr.MGR_OK and n == len(reqs)
    for x, y in zip(xs, ys):
        assert rel_linf(y.cpu().numpy(), oracle.decompose(x.cpu().numpy().astype(np.float64))) <= 1e-5
    for p in plans:
        p.close()
