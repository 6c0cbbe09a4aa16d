"""Largest sizes: fields of more than 2^31 nodes (64-bit element offsets in
every kernel), checked through properties that hold at any size, since the
oracle cannot run at this scale:

* the finest-level coefficients are local, c = u - (interpolant of u on the
  coarse nodes), so sampled ones are recomputed on the CPU from the field;
* recompose(decompose(u)) == u;
* a field that is multilinear in the coordinates has zero coefficients.
"""
import numpy as np
import pytest

import paper_2105_12764_gb300 as mgr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def finest_coeff(u, idx):
    """c at full-grid index idx (fine in at least one axis) of the finest level,
    unit spacing: separable linear interpolation from the even neighbours."""
    opts = []
    for k, i in enumerate(idx):
        n = u.shape[k]
        if i % 2 == 0 or i == n - 1:
            opts.append([(i, 1.0)])
        else:
            opts.append([(i - 1, 0.5), (i + 1, 0.5)])
    interp = 0.0
    for a, wa in opts[0]:
        for b, wb in opts[1]:
            for c, wc in opts[2]:
                interp += wa * wb * wc * float(u[a, b, c])
    return float(u[idx]) - interp


@pytest.mark.parametrize("n,dtype,tol,rt_tol", [(1300, mgr.MGR_F32, 1e-5, 1e-5), (1025, mgr.MGR_F64, 1e-12, 1e-13)])
def test_largest_fields(n, dtype, tol, rt_tol):
    td = torch.float32 if dtype == mgr.MGR_F32 else torch.float64
    shape = (n, n, n)
    ctx = mgr.Context(0)
    plan = mgr.Plan(ctx, shape, None, -1, dtype)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(shape, dtype=td, device="cuda", generator=g)
    y = torch.empty_like(x)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    try:
        plan.decompose(x, y, ws)
        torch.cuda.synchronize()
        # sampled finest-level coefficients, against the local definition
        rng = np.random.default_rng(1)
        xs = x.cpu().numpy()
        ys = y.cpu().numpy()
        scale = float(np.abs(xs).max())
        checked = 0
        while checked < 2000:
            idx = tuple(int(v) for v in rng.integers(0, n, 3))
            if all(i % 2 == 0 or i == n - 1 for i in idx):
                continue
            assert abs(float(ys[idx]) - finest_coeff(xs, idx)) <= tol * scale, idx
            checked += 1
        del xs, ys
        # round trip, compared on the device
        z = torch.empty_like(x)
        plan.recompose(y, z, ws)
        torch.cuda.synchronize()
        err = float((z - x).abs().max().item()) / scale
        assert err <= rt_tol, err
        del z
        # a multilinear field has zero coefficients (all but the coarsest nodes)
        ar = torch.arange(n, dtype=td, device="cuda") / n
        x.copy_(1.0 + 0.5 * ar.view(n, 1, 1) - 0.25 * ar.view(1, n, 1) * ar.view(1, 1, n))
        plan.decompose(x, y, ws)
        torch.cuda.synchronize()
        # coarsest nodes: multiples of 2^L and the last node (keep-last nesting)
        s = 1 << plan.levels
        co = torch.tensor(sorted(set(range(0, n, s)) | {n - 1}), device="cuda")
        keep = torch.ones(shape, dtype=torch.bool, device="cuda")
        keep[co.view(-1, 1, 1), co.view(1, -1, 1), co.view(1, 1, -1)] = False
        assert float(y[keep].abs().max().item()) <= (1e-5 if dtype == mgr.MGR_F32 else 1e-12) * 1.5
    finally:
        plan.close()
        ctx.close()
