"""Batched refactoring (mgr_batch_submit / mgr_batch_poll) vs the single-field
path and the FP64 oracle: fields of uneven 2D/3D shapes, uniform and
stretched coordinates, in one submit; graph replay on a second submit."""
import numpy as np
import pytest

import oracle
import paper_2105_12764_gb300 as mgr
from gpu_util import rel_linf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def stretched(n, ratio=1.01):
    return np.concatenate([[0.0], np.cumsum(ratio ** np.arange(n - 1))])


def make_fields(rng, count, dtype):
    fields = []
    for i in range(count):
        if rng.random() < 0.45:
            shape = tuple(int(v) for v in rng.integers(17, 130, 2))
        else:
            shape = tuple(int(v) for v in rng.integers(17, 66, 3))
        coords = None if rng.random() < 0.5 else [stretched(s) for s in shape]
        u = rng.standard_normal(shape)
        if dtype == mgr.MGR_F32:
            u = u.astype(np.float32)
        fields.append((u, coords))
    return fields


@pytest.fixture(scope="module")
def ctx():
    return mgr.Context(0)


@pytest.mark.parametrize("dtype,prec,tol", [(mgr.MGR_F64, mgr.MGR_PREC_NATIVE, 1e-12),
                                            (mgr.MGR_F32, mgr.MGR_PREC_NATIVE, 1e-5),
                                            (mgr.MGR_F32, mgr.MGR_PREC_MIXED, 1e-5)])
def test_batch_matches_oracle_and_single(ctx, dtype, prec, tol):
    rng = np.random.default_rng(7 + dtype + 2 * prec)
    fields = make_fields(rng, 24, dtype)
    td = torch.float64 if dtype == mgr.MGR_F64 else torch.float32
    plans, ins, outs, backs = [], [], [], []
    for u, coords in fields:
        plans.append(mgr.Plan(ctx, u.shape, coords, -1, dtype, prec))
        ins.append(torch.from_numpy(u).cuda())
        outs.append(torch.empty_like(ins[-1]))
        backs.append(torch.empty_like(ins[-1]))
    t = ctx.batch_submit([(mgr.MGR_OP_DECOMPOSE, p, a, b) for p, a, b in zip(plans, ins, outs)])
    assert ctx.batch_poll(t, -1) == (mgr.MGR_OK, len(fields))
    t = ctx.batch_submit([(mgr.MGR_OP_RECOMPOSE, p, b, c) for p, b, c in zip(plans, outs, backs)])
    assert ctx.batch_poll(t, -1)[0] == mgr.MGR_OK
    for (u, coords), p, a, b, c in zip(fields, plans, ins, outs, backs):
        ref = oracle.decompose(u.astype(np.float64), coords)
        got = b.cpu().numpy()
        assert rel_linf(got, ref) <= tol, u.shape
        assert rel_linf(c.cpu().numpy(), u) <= max(tol, 1e-13), u.shape
        # single-field path on the same plan
        single = torch.empty_like(a)
        ws = torch.empty(max(p.workspace_bytes, 256), dtype=torch.uint8, device="cuda")
        p.decompose(a, single, ws)
        torch.cuda.synchronize()
        assert rel_linf(got, single.cpu().numpy()) <= (1e-13 if dtype == mgr.MGR_F64 else 1e-6)
    # replay: the same request list runs from the cached graph
    outs2 = [torch.empty_like(x) for x in ins]
    first = [o.clone() for o in outs]
    t = ctx.batch_submit([(mgr.MGR_OP_DECOMPOSE, p, a, b) for p, a, b in zip(plans, ins, outs)])
    assert ctx.batch_poll(t, -1)[0] == mgr.MGR_OK
    for o, f in zip(outs, first):
        assert torch.equal(o, f)
    assert "chosen tile" in ctx.batch_tuning()
    for p in plans:
        p.close()


def test_batch_errors(ctx):
    p64 = mgr.Plan(ctx, (33, 33), None, -1, mgr.MGR_F64)
    p32 = mgr.Plan(ctx, (33, 33), None, -1, mgr.MGR_F32)
    a = torch.zeros((33, 33), dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    with pytest.raises(mgr.MgrError) as ei:
        ctx.batch_submit([(0, p64, a, a)])  # in == out
    assert ei.value.code == mgr.MGR_EINVAL
    with pytest.raises(mgr.MgrError) as ei:
        ctx.batch_submit([(0, p64, a, b), (0, p32, a, b)])  # mixed dtypes
    assert ei.value.code == mgr.MGR_EINVAL
    with pytest.raises(mgr.MgrError) as ei:
        ctx.batch_poll(987654321, 0)
    assert ei.value.code == mgr.MGR_ENOTFOUND
    small = mgr.Context(0, mem_budget_bytes=1024)
    q = mgr.Plan(small, (65, 65, 65), None, -1, mgr.MGR_F64)
    c = torch.zeros((65, 65, 65), dtype=torch.float64, device="cuda")
    d = torch.zeros_like(c)
    with pytest.raises(mgr.MgrError) as ei:
        small.batch_submit([(0, q, c, d)])
    assert ei.value.code == mgr.MGR_EBUDGET
    q.close()
    small.close()
    p64.close()
    p32.close()


def test_autotune_decision_persists_across_contexts(tmp_path, monkeypatch):
    """MGR_AUTOTUNE_CACHE: the first context times the candidates and appends its
    decision, keyed by GPU and batch shape; a later context (another process
    would be the same) reads it instead of timing, and computes the same result."""
    path = tmp_path / "autotune.txt"
    monkeypatch.setenv("MGR_AUTOTUNE_CACHE", str(path))
    rng = np.random.default_rng(21)
    fields = make_fields(rng, 8, mgr.MGR_F32)
    results = []
    for round_ in range(2):
        c = mgr.Context(0)
        plans = [mgr.Plan(c, u.shape, coords, -1, mgr.MGR_F32) for u, coords in fields]
        ins = [torch.from_numpy(u).cuda() for u, _ in fields]
        outs = [torch.empty_like(x) for x in ins]
        t = c.batch_submit([(mgr.MGR_OP_DECOMPOSE, p, a, b) for p, a, b in zip(plans, ins, outs)])
        assert c.batch_poll(t, -1)[0] == mgr.MGR_OK
        report = c.batch_tuning()
        assert ("from the persisted cache" in report) == (round_ == 1), report
        if round_ == 0:
            lines = path.read_text().split("\n")
            assert len([ln for ln in lines if ln.strip()]) == 1
            name = torch.cuda.get_device_name(0).replace(" ", "_")
            assert lines[0].startswith(name)
        results.append([o.cpu().numpy() for o in outs])
        for p in plans:
            p.close()
        c.close()
    for a, b in zip(*results):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("dtype,tol", [(mgr.MGR_F32, 1e-5), (mgr.MGR_F64, 1e-12)])
def test_every_tile_shape_matches_oracle(tmp_path, monkeypatch, dtype, tol):
    """Each level-pass tile shape of the batched form (30x14, 30x6, and 14x14 in
    half-warp row groups) and two chunk lengths, forced through the persisted
    decision file: the first context records its decisions, each later one
    reads an edited file and runs that shape, and every result equals the
    oracle (decomposition) and the input (recomposition)."""
    path = tmp_path / "autotune.txt"
    monkeypatch.setenv("MGR_AUTOTUNE_CACHE", str(path))
    rng = np.random.default_rng(33 + dtype)
    fields = make_fields(rng, 12, dtype)
    # coarse rows shorter and longer than one tile, ragged in every axis
    extra = [(97, 45, 70), (33, 18, 129), (9, 65, 31)]
    for shape in extra:
        u = rng.standard_normal(shape)
        fields.append((u.astype(np.float32) if dtype == mgr.MGR_F32 else u, [stretched(s) for s in shape]))
    refs = [oracle.decompose(u.astype(np.float64), coords) for u, coords in fields]

    def run():
        c = mgr.Context(0)
        plans = [mgr.Plan(c, u.shape, coords, -1, dtype) for u, coords in fields]
        ins = [torch.from_numpy(u).cuda() for u, _ in fields]
        outs = [torch.full_like(x, float("nan")) for x in ins]
        backs = [torch.full_like(x, float("nan")) for x in ins]
        t = c.batch_submit([(mgr.MGR_OP_DECOMPOSE, p, a, b) for p, a, b in zip(plans, ins, outs)])
        assert c.batch_poll(t, -1)[0] == mgr.MGR_OK
        t = c.batch_submit([(mgr.MGR_OP_RECOMPOSE, p, b, d) for p, b, d in zip(plans, outs, backs)])
        assert c.batch_poll(t, -1)[0] == mgr.MGR_OK
        torch.cuda.synchronize()
        report = c.batch_tuning()
        res = [(o.cpu().numpy(), r.cpu().numpy()) for o, r in zip(outs, backs)]
        for p in plans:
            p.close()
        c.close()
        return report, res

    run()  # records the two decisions (decomposition, recomposition)
    recorded = [ln.split() for ln in path.read_text().split("\n") if ln.strip()]
    assert len(recorded) == 2
    for cfg, name in enumerate(["30x14", "30x6", "14x14"]):
        for chunk in (8, 16):
            path.write_text("".join(f"{g} {h} {cfg} {chunk}\n" for g, h, _, _ in recorded))
            report, res = run()
            assert f"chosen tile={name} chunk={chunk}" in report and "persisted cache" in report, report
            for (u, _), ref, (got, back) in zip(fields, refs, res):
                assert rel_linf(got, ref) <= tol, (name, chunk, u.shape)
                assert rel_linf(back, u) <= max(tol, 1e-13), (name, chunk, u.shape)
