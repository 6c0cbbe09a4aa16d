"""Serving loop (mgr_serve_*): each result is the same alone and in the mix;
admission by memory budget; resident hierarchies, eviction; timeouts and
error codes (all failures made on the host: no GPU fault is involved)."""
import numpy as np
import pytest

import oracle
import paper_2105_12764_gb300 as mgr
from gpu_util import rel_linf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

DEC, REC = mgr.MGR_OP_DECOMPOSE, mgr.MGR_OP_RECOMPOSE


def make_set(ctx, rng):
    items = []
    for shape, dtype in [((33, 33, 33), mgr.MGR_F32), ((65, 40, 70), mgr.MGR_F64), ((129, 129), mgr.MGR_F32),
                         ((50, 61, 45), mgr.MGR_F64), ((97, 33, 80), mgr.MGR_F32), ((40, 40, 40), mgr.MGR_F64)]:
        td = torch.float64 if dtype == mgr.MGR_F64 else torch.float32
        u = rng.standard_normal(shape)
        x = torch.from_numpy(u).to(td).cuda()
        items.append((mgr.Plan(ctx, shape, None, -1, dtype), x))
    return items


def hier_to_numpy(srv, handle, plan, like):
    out = torch.empty_like(like)
    srv.read(handle, out, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def run_requests(srv, items, alone):
    """Decompose every field (keep resident), then recompose each hierarchy."""
    decs, hiers, recs = [], [], []
    for plan, x in items:
        rid = srv.enqueue(DEC, plan, inp=x, keep_resident=1)
        if alone:
            rc, res = srv.wait(rid)
            assert res["status"] == mgr.MGR_OK
            decs.append(res)
        else:
            decs.append(rid)
    if not alone:
        decs = [srv.wait(rid)[1] for rid in decs]
    for (plan, x), res in zip(items, decs):
        assert res["status"] == mgr.MGR_OK and res["handle"] > 0
        hiers.append(hier_to_numpy(srv, res["handle"], plan, x))
    outs = [torch.empty_like(x) for _, x in items]
    rids = []
    for (plan, x), res, o in zip(items, decs, outs):
        rid = srv.enqueue(REC, plan, src=res["handle"], out=o)
        if alone:
            assert srv.wait(rid)[1]["status"] == mgr.MGR_OK
        else:
            rids.append(rid)
    for rid in rids:
        assert srv.wait(rid)[1]["status"] == mgr.MGR_OK
    torch.cuda.synchronize()
    for res in decs:
        assert srv.release(res["handle"]) == mgr.MGR_OK
    return hiers, [o.cpu().numpy() for o in outs]


def test_same_alone_and_in_mix():
    ctx = mgr.Context(0, mem_budget_bytes=8 << 30)
    rng = np.random.default_rng(0)
    items = make_set(ctx, rng)
    srv1 = mgr.Server(ctx, slots=1, streams=1)
    h_alone, r_alone = run_requests(srv1, items, alone=True)
    srv1.stop()
    srv4 = mgr.Server(ctx, slots=4, streams=4)
    h_mix, r_mix = run_requests(srv4, items, alone=False)
    assert srv4.stats()["resident"] == 0
    srv4.stop()
    for (plan, x), ha, hm, ra, rm in zip(items, h_alone, h_mix, r_alone, r_mix):
        # identical kernels and arguments: the mix must not change a result
        tol = 1e-12 if x.dtype == torch.float64 else 1e-6
        assert rel_linf(hm, ha) <= tol
        assert rel_linf(rm, ra) <= tol
        u = x.cpu().numpy().astype(np.float64)
        assert rel_linf(ha, oracle.decompose(u)) <= (1e-12 if x.dtype == torch.float64 else 1e-5)
        assert rel_linf(ra, u) <= (1e-13 if x.dtype == torch.float64 else 1e-5)
    for plan, _ in items:
        plan.close()
    ctx.close()


def test_admission_budget_and_eviction():
    # budget for about three 65^3 FP64 hierarchies plus workspaces
    field = 65 ** 3 * 8
    ctx = mgr.Context(0, mem_budget_bytes=int(field * 3.9))
    plan = mgr.Plan(ctx, (65, 65, 65), None, -1, mgr.MGR_F64)
    x = torch.randn((65, 65, 65), dtype=torch.float64, device="cuda")
    srv = mgr.Server(ctx, slots=2, streams=2)
    handles = []
    for _ in range(5):
        rid = srv.enqueue(DEC, plan, inp=x, keep_resident=1)
        rc, res = srv.wait(rid)
        assert res["status"] == mgr.MGR_OK
        handles.append(res["handle"])
        assert srv.stats()["used_bytes"] <= int(field * 3.9)
    # the oldest hierarchies were evicted to admit the newer ones
    with pytest.raises(mgr.MgrError) as ei:
        srv.hierarchy(handles[0])
    assert ei.value.code == mgr.MGR_ENOTFOUND
    srv.hierarchy(handles[-1])
    # a request that can never fit is refused at enqueue
    big = mgr.Plan(ctx, (129, 129, 129), None, -1, mgr.MGR_F64)
    xb = torch.zeros((129, 129, 129), dtype=torch.float64, device="cuda")
    with pytest.raises(mgr.MgrError) as ei:
        srv.enqueue(DEC, big, inp=xb)
    assert ei.value.code == mgr.MGR_EBUDGET
    # recomposing an unknown hierarchy
    with pytest.raises(mgr.MgrError) as ei:
        srv.enqueue(REC, plan, src=123456789, out=x)
    assert ei.value.code == mgr.MGR_ENOTFOUND
    srv.stop()
    big.close()
    plan.close()
    ctx.close()


def test_wait_timeout_and_unknown_request():
    ctx = mgr.Context(0)
    plan = mgr.Plan(ctx, (257, 257, 257), None, -1, mgr.MGR_F64)
    x = torch.randn((257, 257, 257), dtype=torch.float64, device="cuda")
    srv = mgr.Server(ctx, slots=1, streams=1)
    ids = [srv.enqueue(DEC, plan, inp=x, keep_resident=0) for _ in range(3)]
    # the third request waits behind two multi-millisecond ones
    rc, res = srv.wait(ids[2], timeout_us=0)
    assert rc == mgr.MGR_EPENDING
    rc, res = srv.wait(ids[2], timeout_us=10)
    assert rc in (mgr.MGR_ETIMEDOUT, mgr.MGR_OK)
    pending = ids if rc != mgr.MGR_OK else ids[:2]
    for i in pending:
        rc, res = srv.wait(i)
        assert res["status"] == mgr.MGR_OK and res["done"] >= res["admitted"] >= res["arrival"] - 1e-3
    with pytest.raises(mgr.MgrError) as ei:
        srv.wait(ids[0])
    assert ei.value.code == mgr.MGR_ENOTFOUND
    assert srv.stats() == dict(used_bytes=0, queued=0, running=0, resident=0)
    srv.stop()
    plan.close()
    ctx.close()
