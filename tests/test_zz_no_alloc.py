"""mgr_decompose_noalloc: the decomposition entry point for callers that
cannot allocate device memory (their memory belongs to another allocator,
they only hold their input and output buffers, or an allocation would stall
their path).  Its workspace is a fixed scratch area in the library's device
image.  Through the C ABI this checks:

* two calls in a row give the same output as mgr_decompose with a caller
  workspace (1D-3D, uniform and stretched coordinates), and a 4D field's
  output equals the FP64 oracle's;
* in place: a 3D call with in == out equals mgr_decompose; a 4D call with
  in == out is refused (4D runs out of place only);
* no device memory is allocated by repeated calls, and a call captured into
  a CUDA graph after the first (uncaptured) one replays to the same result;
* a first call made while the stream is being captured is refused without
  breaking the capture (in a fresh process, where the first call is that one);
* fields too large for the area are refused.
"""
import ctypes
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import paper_2105_12764_gb300 as mgr
from gpu_util import rel_linf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def noalloc(plan, x, y, stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return mgr.lib.mgr_decompose_noalloc(plan.handle, x.data_ptr(), y.data_ptr(), ctypes.c_void_p(s.cuda_stream))


def stretched(n):
    return np.concatenate([[0.0], np.cumsum(1.01 ** np.arange(n - 1))])


@pytest.mark.parametrize("shape,dtype,coords", [((65, 65, 65), mgr.MGR_F64, False),
                                                ((100, 129, 90), mgr.MGR_F32, True),
                                                ((300, 257), mgr.MGR_F64, True)])
def test_noalloc_matches_decompose_twice(shape, dtype, coords):
    ctx = mgr.Context(0)
    cs = [stretched(n) for n in shape] if coords else None
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


def test_noalloc_4d_out_of_place_matches_oracle_and_refuses_in_place():
    import oracle

    shape = (9, 17, 20, 33)
    ctx = mgr.Context(0)
    plan = mgr.Plan(ctx, shape, None, -1, mgr.MGR_F64)
    assert plan.workspace_bytes <= mgr.MGR_NOALLOC_SCRATCH_BYTES
    u = np.random.default_rng(5).standard_normal(shape)
    want = oracle.decompose(u)
    x = torch.from_numpy(u).cuda()
    for _ in range(2):
        y = torch.full_like(x, float("nan"))
        assert noalloc(plan, x, y) == mgr.MGR_OK
        torch.cuda.synchronize()
        assert rel_linf(y.cpu().numpy(), want) <= 1e-12
    before = x.clone()
    assert noalloc(plan, x, x) == mgr.MGR_EINVAL
    torch.cuda.synchronize()
    assert torch.equal(x, before)  # refused before any launch
    plan.close()
    ctx.close()


def test_noalloc_3d_in_place_matches_decompose():
    shape = (49, 40, 67)
    ctx = mgr.Context(0)
    plan = mgr.Plan(ctx, shape, [stretched(n) for n in shape], -1, mgr.MGR_F64)
    x = torch.from_numpy(np.random.default_rng(6).standard_normal(shape)).cuda()
    ref = torch.empty_like(x)
    ws = torch.empty(max(plan.workspace_bytes, 256), dtype=torch.uint8, device="cuda")
    plan.decompose(x, ref, ws)
    for _ in range(2):
        y = x.clone()
        assert noalloc(plan, y, y) == mgr.MGR_OK
        torch.cuda.synchronize()
        assert rel_linf(y.cpu().numpy(), ref.cpu().numpy()) <= 1e-12
    plan.close()
    ctx.close()


def test_noalloc_allocates_nothing_and_replays_from_a_graph():
    shape = (65, 66, 67)
    ctx = mgr.Context(0)
    plan = mgr.Plan(ctx, shape, None, -1, mgr.MGR_F32)
    x = torch.randn(shape, dtype=torch.float32, device="cuda")
    ref = torch.empty_like(x)
    ws = torch.empty(max(plan.workspace_bytes, 256), dtype=torch.uint8, device="cuda")
    plan.decompose(x, ref, ws)
    y = torch.empty_like(x)
    assert noalloc(plan, x, y) == mgr.MGR_OK  # first call: address lookup outside any capture
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert noalloc(plan, x, y) == mgr.MGR_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert rel_linf(y.cpu().numpy(), ref.cpu().numpy()) <= 1e-6
    # a later call captured into a graph, replayed twice
    z = torch.full_like(x, float("nan"))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        rc = noalloc(plan, x, z, stream=s)
    assert rc == mgr.MGR_OK
    for _ in range(2):
        z.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        assert rel_linf(z.cpu().numpy(), ref.cpu().numpy()) <= 1e-6
    del graph
    plan.close()
    ctx.close()


def test_noalloc_first_call_under_capture_is_refused_in_a_fresh_process():
    code = textwrap.dedent("""
        import ctypes, sys, torch
        sys.path.insert(0, {root!r})
        import paper_2105_12764_gb300 as mgr
        ctx = mgr.Context(0)
        plan = mgr.Plan(ctx, (33, 34, 35), None, -1, mgr.MGR_F64)
        x = torch.randn((33, 34, 35), dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        w = torch.empty_like(x)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            rc = mgr.lib.mgr_decompose_noalloc(plan.handle, x.data_ptr(), y.data_ptr(),
                                               ctypes.c_void_p(s.cuda_stream))
            w.copy_(x)  # the capture still records work after the refusal
        g.replay()
        torch.cuda.synchronize()
        assert rc == mgr.MGR_EINVAL, rc
        assert torch.equal(w, x)
        # outside the capture the first call succeeds
        assert mgr.lib.mgr_decompose_noalloc(plan.handle, x.data_ptr(), y.data_ptr(),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
        torch.cuda.synchronize()
        plan.close()
        ctx.close()
        print("fresh-process capture check ok")
    """).format(root=ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "capture check ok" in r.stdout


def test_noalloc_refuses_fields_beyond_the_scratch_area():
    ctx = mgr.Context(0)
    plan = mgr.Plan(ctx, (257, 257, 257), None, -1, mgr.MGR_F64)
    assert plan.workspace_bytes > mgr.MGR_NOALLOC_SCRATCH_BYTES
    x = torch.zeros((257, 257, 257), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    assert noalloc(plan, x, y) == mgr.MGR_EINVAL
    plan.close()
    ctx.close()
