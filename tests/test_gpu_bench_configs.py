"""Oracle parity at the batched and served bench configurations.

Batched (4096 fields, element counts log-uniform on [17^2, 129^3], 2D and 3D,
half on coordinates stretched by 1.01 per cell, k^-5/3 fields): the whole set
is submitted in one mgr_batch_submit exactly as the benchmark does (same
generator, same seeds, autotuned tiles), then a sample of 72 fields -- the
largest 3D and 2D fields, the smallest, and a seeded random draw, both
coordinate kinds -- is compared element by element with the FP64 oracle:
FP64 <= 1e-12, FP32 <= 1e-5 (against the oracle on the FP32-rounded input);
the round trip of the same fields <= 1e-13 / 1e-5.

Served (Poisson-like mix of decompositions and recompositions of cubes 33^3 ..
513^3, FP32 and FP64, 100 GB admission cap, 4 slots): 257^3 and 513^3
requests in FP32 and FP64 submitted among smaller ones, so their work overlaps
others' on the device; their resident hierarchies are compared with the
oracle and the recompositions of those hierarchies with the inputs.
"""
import numpy as np
import pytest

import oracle
import paper_2105_12764_gb300 as mgr
from gpu_util import rel_linf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2105_12764_gb300 import synth  # noqa: E402

DEC, REC = mgr.MGR_OP_DECOMPOSE, mgr.MGR_OP_RECOMPOSE


@pytest.fixture(scope="module")
def batch_fields():
    """The benchmark's 4096 fields (FP64 masters on the device) and their coordinates."""
    specs = synth.batch_field_specs(4096, seed=0)
    coords = [[synth.stretched_coords(n) for n in shape] if st else None for shape, st in specs]
    fields = [synth.grf_field_torch(shape, seed=1000 + i) for i, (shape, _) in enumerate(specs)]
    return specs, coords, fields


def sample_indices(specs, k_random=48):
    sizes = np.array([int(np.prod(s)) for s, _ in specs])
    is3 = np.array([len(s) == 3 for s, _ in specs])
    order = np.argsort(sizes)
    big3 = [int(i) for i in order[::-1] if is3[i]][:8]
    big2 = [int(i) for i in order[::-1] if not is3[i]][:8]
    small = [int(i) for i in order[:8]]
    chosen = set(big3 + big2 + small)
    rest = [i for i in range(len(specs)) if i not in chosen]
    rng = np.random.default_rng(2024)
    chosen.update(int(i) for i in rng.choice(rest, k_random, replace=False))
    return sorted(chosen)


@pytest.mark.parametrize("dtype,tol,rt_tol", [(mgr.MGR_F32, 1e-5, 1e-5), (mgr.MGR_F64, 1e-12, 1e-13)])
def test_batched_4096_fields_sample_matches_oracle(batch_fields, dtype, tol, rt_tol):
    specs, coords, fields = batch_fields
    ctx = mgr.Context(0)
    td = torch.float32 if dtype == mgr.MGR_F32 else torch.float64
    plans = [mgr.Plan(ctx, s, c, -1, dtype) for (s, _), c in zip(specs, coords)]
    xs = [f.to(td) for f in fields]
    ys = [torch.empty_like(x) for x in xs]
    zs = [torch.empty_like(x) for x in xs]
    try:
        t = ctx.batch_submit([(DEC, p, x, y) for p, x, y in zip(plans, xs, ys)])
        assert ctx.batch_poll(t, -1) == (mgr.MGR_OK, len(specs))
        t = ctx.batch_submit([(REC, p, y, z) for p, y, z in zip(plans, ys, zs)])
        assert ctx.batch_poll(t, -1)[0] == mgr.MGR_OK
        torch.cuda.synchronize()
        assert "chosen tile" in ctx.batch_tuning()
        idx = sample_indices(specs)
        assert {len(specs[i][0]) for i in idx} == {2, 3}
        assert {specs[i][1] for i in idx} == {False, True}
        assert max(int(np.prod(specs[i][0])) for i in idx) > 100 ** 3
        worst = 0.0
        for i in idx:
            u = xs[i].cpu().numpy().astype(np.float64)
            ref = oracle.decompose(u, coords[i])
            err = rel_linf(ys[i].cpu().numpy(), ref)
            worst = max(worst, err)
            assert err <= tol, (i, specs[i], err)
            assert rel_linf(zs[i].cpu().numpy(), u) <= rt_tol, (i, specs[i])
        print(f"batched sample of {len(idx)} fields: worst error vs oracle {worst:.3e}")
    finally:
        for p in plans:
            p.close()
        ctx.close()


def test_served_mix_large_requests_match_oracle():
    ctx = mgr.Context(0, mem_budget_bytes=100 << 30)
    rng = np.random.default_rng(3)
    targets = [(257, mgr.MGR_F32), (257, mgr.MGR_F64), (513, mgr.MGR_F32), (513, mgr.MGR_F64)]
    fillers = [(int(n), dt) for n, dt in zip(rng.integers(33, 160, 24), rng.integers(0, 2, 24))]
    plans, inputs = {}, {}
    for i, key in enumerate(sorted(set(targets + fillers))):
        n, dt = key
        plans[key] = mgr.Plan(ctx, (n, n, n), None, -1, dt)
        f = synth.grf_field_torch((n, n, n), seed=500 + i)
        inputs[key] = f.float() if dt == mgr.MGR_F32 else f
    srv = mgr.Server(ctx, slots=4, streams=4)
    try:
        # targets interleaved with smaller requests: their work overlaps others' on the device
        order = []
        for k, tgt in enumerate(targets):
            order += fillers[6 * k: 6 * k + 3] + [tgt] + fillers[6 * k + 3: 6 * k + 6]
        rids = [(key, srv.enqueue(DEC, plans[key], inp=inputs[key], keep_resident=1)) for key in order]
        done = {}
        for key, rid in rids:
            rc, res = srv.wait(rid)
            assert res["status"] == mgr.MGR_OK
            done.setdefault(key, res)
        # recompositions of the target hierarchies, again among filler decompositions
        outs, rrids = {}, []
        for k, tgt in enumerate(targets):
            outs[tgt] = torch.empty_like(inputs[tgt])
            rrids.append(srv.enqueue(REC, plans[tgt], src=done[tgt]["handle"], out=outs[tgt]))
            f = fillers[k]
            rrids.append(srv.enqueue(DEC, plans[f], inp=inputs[f], keep_resident=0))
        for rid in rrids:
            assert srv.wait(rid)[1]["status"] == mgr.MGR_OK
        torch.cuda.synchronize()
        for tgt in targets:
            n, dt = tgt
            x = inputs[tgt]
            h = torch.empty_like(x)
            srv.read(done[tgt]["handle"], h, torch.cuda.current_stream())
            torch.cuda.synchronize()
            u = x.cpu().numpy().astype(np.float64)
            ref = oracle.decompose(u)
            tol, rt = (1e-12, 1e-13) if dt == mgr.MGR_F64 else (1e-5, 1e-5)
            err = rel_linf(h.cpu().numpy(), ref)
            assert err <= tol, (tgt, err)
            del ref
            assert rel_linf(outs[tgt].cpu().numpy(), u) <= rt, tgt
    finally:
        srv.stop()
        for p in plans.values():
            p.close()
        ctx.close()
