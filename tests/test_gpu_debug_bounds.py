"""The bounds-checking build (libmgr_debug.so, MGR_DEBUG_BOUNDS) runs the hot
path clean: every global index of the level pass, interpolation, solves,
one-CTA coarse levels and coarsest copy inside its buffer, and the level
pass's shared-tile indices inside the tile, on ragged non-2^k+1 shapes, every
form and layout, the batched, served, host-buffer, no-allocation and 4D
entry points.  Each operation must return MGR_OK (an out-of-bounds index
would return MGR_EDEVICE) and its result must equal the FP64 oracle's.  Runs
in a fresh process that loads the bounds-checking library."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import atexit, ctypes, sys, numpy as np, torch
    sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
    import paper_2105_12764_gb300 as mgr, oracle
    from gpu_util import Runner, rel_linf
    assert mgr.lib.mgr_debug_bounds() == 1, "not the bounds-checking build"
    def report():
        code = ctypes.c_int(); idx = ctypes.c_int64(); ext = ctypes.c_int64()
        if mgr.lib.mgr_debug_last(ctypes.byref(code), ctypes.byref(idx), ctypes.byref(ext)) == 0:
            print(f"out-of-bounds access recorded: code {{code.value}} index {{idx.value}} extent {{ext.value}}")
    atexit.register(report)
    rng = np.random.default_rng(1)
    def stretched(n): return np.concatenate([[0.0], np.cumsum(1.01 ** np.arange(n - 1))])
    ctx = mgr.Context(0, mem_budget_bytes=8 << 30)
    cases = [((70, 45, 101), True), ((129, 17), False), ((33, 40, 65), True), ((300,), False), ((95, 80, 140), False)]
    for shape, st in cases:
        coords = [stretched(n) for n in shape] if st else None
        for dtype, prec, tol in ((mgr.MGR_F64, 0, 1e-12), (mgr.MGR_F32, 0, 1e-5), (mgr.MGR_F32, 1, 1e-5)):
            for levels in (-1, 1):
                u = rng.standard_normal(shape)
                if dtype == mgr.MGR_F32: u = u.astype(np.float32)
                r = Runner(ctx, shape, coords, levels, dtype, prec)
                got = r.decompose(u)
                ref = oracle.decompose(u.astype(np.float64), coords, r.plan.levels)
                assert rel_linf(got, ref) <= tol, (shape, dtype, prec, levels)
                back = r.recompose(got)
                assert rel_linf(back, u) <= max(tol, 1e-13), (shape, dtype, prec, levels)
                inplace = r.decompose(u, inplace=True)
                assert rel_linf(inplace, ref) <= tol
                r.close()
    # class-packed, progressive and quantized forms
    shape = (65, 50, 77)
    plan = mgr.Plan(ctx, shape, None, -1, mgr.MGR_F64)
    L = plan.levels
    u = rng.standard_normal(shape)
    x = torch.from_numpy(u).cuda(); pk = torch.empty(x.numel(), dtype=x.dtype, device="cuda"); y = torch.empty_like(x)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.decompose_packed(x, pk, ws); plan.recompose_packed(pk, L, y, ws); torch.cuda.synchronize()
    want = oracle.pack_classes(oracle.decompose(u), L)
    assert rel_linf(pk.cpu().numpy(), want) <= 1e-12
    assert rel_linf(y.cpu().numpy(), oracle.recompose_classes(want, shape, L, None, L)) <= 1e-12
    codes = torch.empty(x.numel(), dtype=torch.int32, device="cuda")
    plan.decompose_quantized(x, codes, 1e-3, ws); plan.recompose_dequantized(codes, L + 1, 1e-3, y, ws)
    torch.cuda.synchronize()
    assert float((y - x).abs().max()) <= 1e-3 * (1 + 1e-9)
    # host buffers (pipelined path) and the no-allocation entry point
    pin = torch.from_numpy(u).pin_memory(); pc = torch.empty_like(pin).pin_memory(); po = torch.empty_like(pin).pin_memory()
    plan.decompose_host(pin, pc, x, y, ws); plan.recompose_host(pc, po, y, x, ws); torch.cuda.synchronize()
    assert rel_linf(pc.numpy(), oracle.decompose(u)) <= 1e-12 and rel_linf(po.numpy(), u) <= 1e-13
    x.copy_(torch.from_numpy(u))
    rc = mgr.lib.mgr_decompose_noalloc(plan.handle, x.data_ptr(), y.data_ptr(),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == 0 and rel_linf(y.cpu().numpy(), oracle.decompose(u)) <= 1e-12
    plan.close()
    # 4D
    shape4 = (9, 17, 20, 33)
    u4 = rng.standard_normal(shape4)
    r4 = Runner(ctx, shape4, None, -1, mgr.MGR_F64)
    assert rel_linf(r4.decompose(u4), oracle.decompose(u4)) <= 1e-12
    r4.close()
    # batched and served
    shapes = [(40, 33), (20, 30, 50), (65, 65, 65), (17, 129), (100, 37, 45)]
    plans = [mgr.Plan(ctx, s, None, -1, mgr.MGR_F32) for s in shapes]
    us = [rng.standard_normal(s).astype(np.float32) for s in shapes]
    xs = [torch.from_numpy(v).cuda() for v in us]; ys = [torch.empty_like(v) for v in xs]
    t = ctx.batch_submit([(0, p, a, b) for p, a, b in zip(plans, xs, ys)])
    assert ctx.batch_poll(t, -1) == (0, len(shapes))
    for v, b in zip(us, ys):
        assert rel_linf(b.cpu().numpy(), oracle.decompose(v.astype(np.float64))) <= 1e-5
    srv = mgr.Server(ctx, slots=2, streams=2)
    rid = srv.enqueue(0, plans[2], inp=xs[2], keep_resident=0)
    assert srv.wait(rid)[1]["status"] == 0
    srv.stop()
    for p in plans: p.close()
    code = ctypes.c_int(); idx = ctypes.c_int64(); ext = ctypes.c_int64()
    assert mgr.lib.mgr_debug_last(ctypes.byref(code), ctypes.byref(idx), ctypes.byref(ext)) == mgr.MGR_ENOTFOUND
    ctx.close()
    print("bounds-checking build clean")
""")


def test_bounds_checking_build_runs_clean():
    lib = os.path.join(ROOT, "paper_2105_12764_gb300", "libmgr_debug.so")
    if not os.path.exists(lib):
        import importlib.util

        spec = importlib.util.spec_from_file_location("mgr_build", os.path.join(ROOT, "paper_2105_12764_gb300", "build.py"))
        b = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(b)
        lib = b.build(debug_bounds=True)
    env = dict(os.environ, MGR_LIBRARY=lib)
    code = SCRIPT.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900, env=env)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "clean" in r.stdout
