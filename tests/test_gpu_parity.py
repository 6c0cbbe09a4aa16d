"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (normwise relative L-infinity, max|a-b| / max|ref|):
  FP64 decompose / recompose vs oracle   <= 1e-12
  FP64 round trip                        <= 1e-13
  FP32 and mixed forms vs FP64 oracle    <= 1e-5  (oracle run on the same
                                                   FP32-rounded input values)
"""
import numpy as np
import pytest

import oracle
import paper_2105_12764_gb300 as mgr
from gpu_util import Runner, rel_linf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

TOL64, TOL64_RT, TOL32 = 1e-12, 1e-13, 1e-5


@pytest.fixture(scope="module")
def ctx():
    c = mgr.Context(0)
    yield c


def stretched(n, ratio):
    return np.concatenate([[0.0], np.cumsum(ratio ** np.arange(n - 1))])


def random_coords(rng, n):
    return np.concatenate([[0.0], np.cumsum(rng.uniform(0.2, 3.0, n - 1))])


def check_f64(ctx, u, coords=None, levels=-1, inplace=False):
    r = Runner(ctx, u.shape, coords, levels, mgr.MGR_F64)
    try:
        ref = oracle.decompose(u, coords, levels)
        got = r.decompose(u, inplace=inplace)
        e = rel_linf(got, ref)
        assert e <= TOL64, f"decompose {u.shape} levels={levels}: {e:.3e}"
        back = r.recompose(got, inplace=inplace)
        rt = rel_linf(back, u)
        assert rt <= TOL64_RT, f"round trip {u.shape}: {rt:.3e}"
        rec_ref = oracle.recompose(ref, coords, levels)
        assert rel_linf(r.recompose(ref), rec_ref) <= TOL64
    finally:
        r.close()


# --------------------------------------------------------------- sweeps ----

@pytest.mark.parametrize("n", list(range(2, 41)))
def test_1d_every_size(ctx, n):
    rng = np.random.default_rng(n)
    u = rng.standard_normal(n)
    check_f64(ctx, u)
    check_f64(ctx, u, [random_coords(rng, n)], levels=oracle.max_levels((n,)))


@pytest.mark.parametrize("n", list(range(2, 41)))
def test_2d_every_size(ctx, n):
    rng = np.random.default_rng(100 + n)
    for shape in [(n, 7), (7, n)]:
        u = rng.standard_normal(shape)
        check_f64(ctx, u)
        check_f64(ctx, u, [random_coords(rng, s) for s in shape])


@pytest.mark.parametrize("n", list(range(2, 41)))
def test_3d_every_size(ctx, n):
    rng = np.random.default_rng(200 + n)
    for shape in [(n, 5, 6), (5, n, 6), (5, 6, n)]:
        u = rng.standard_normal(shape)
        check_f64(ctx, u, [random_coords(rng, s) for s in shape])


# ------------------------------------------------- multi-tile, ragged tails --

# tile edges: 30 coarse x and 14 coarse y per CTA; n = 60 (m = 31) and n = 28
# (m = 15) put a keep-last coarse node alone in the last tile
MULTI = [(65, 65, 65), (70, 45, 100), (33, 130, 67), (129, 20, 9), (17, 17, 200), (2, 90, 90), (300, 70),
         (29, 28, 60), (58, 60, 121), (31, 57, 62), (12, 29, 59), (140, 30, 61)]


@pytest.mark.parametrize("shape", MULTI)
@pytest.mark.parametrize("kind", ["uniform", "stretched"])
def test_multi_tile_f64(ctx, shape, kind):
    rng = np.random.default_rng(sum(shape))
    u = rng.standard_normal(shape)
    coords = None if kind == "uniform" else [stretched(s, 1.01) for s in shape]
    check_f64(ctx, u, coords)


@pytest.mark.parametrize("levels", [0, 1, 2, 3])
def test_partial_depths(ctx, levels):
    rng = np.random.default_rng(levels)
    u = rng.standard_normal((40, 37, 45))
    check_f64(ctx, u, levels=levels)


def test_inplace(ctx):
    rng = np.random.default_rng(3)
    shape = (37, 66, 70)
    u = rng.standard_normal(shape)
    coords = [random_coords(rng, s) for s in shape]
    check_f64(ctx, u, coords, inplace=True)


def test_sines65_workload(ctx):
    from paper_2105_12764_gb300 import synth

    u, coords = synth.workload("sines65")
    check_f64(ctx, u, coords)


# ------------------------------------------------------- precision forms ----

@pytest.mark.parametrize("prec", [mgr.MGR_PREC_NATIVE, mgr.MGR_PREC_MIXED])
@pytest.mark.parametrize("kind", ["uniform", "stretched"])
def test_f32_forms(ctx, prec, kind):
    rng = np.random.default_rng(11)
    shape = (45, 66, 71)
    u = rng.standard_normal(shape).astype(np.float32)
    coords = None if kind == "uniform" else [stretched(s, 1.01) for s in shape]
    r = Runner(ctx, shape, coords, -1, mgr.MGR_F32, prec)
    try:
        ref = oracle.decompose(u.astype(np.float64), coords)
        got = r.decompose(u)
        assert rel_linf(got, ref) <= TOL32
        back = r.recompose(got)
        assert rel_linf(back, u) <= TOL32
        rec = r.recompose(ref.astype(np.float32))
        assert rel_linf(rec, oracle.recompose(ref, coords)) <= TOL32
    finally:
        r.close()


# -------------------------------------------------------------- errors -----

def test_invalid_arguments(ctx):
    import torch

    with pytest.raises(mgr.MgrError):
        mgr.Plan(ctx, (1, 5))
    with pytest.raises(mgr.MgrError):
        mgr.Plan(ctx, (9,), levels=10)
    with pytest.raises(mgr.MgrError):
        mgr.Plan(ctx, (9,), dtype=mgr.MGR_F64, prec=mgr.MGR_PREC_MIXED)
    with pytest.raises(mgr.MgrError):
        mgr.Plan(ctx, (5,), coords=[np.array([0, 1, 1, 2, 3.0])])
    p = mgr.Plan(ctx, (33, 33))
    buf = torch.zeros(2 * 33 * 33, dtype=torch.float64, device="cuda")
    ws = torch.empty(p.workspace_bytes + 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(mgr.MgrError) as ei:
        p.decompose(buf[0:], buf[5:], ws)  # partial overlap
    assert ei.value.code == mgr.MGR_EINVAL
    with pytest.raises(mgr.MgrError):
        p.decompose(buf, buf[33 * 33:], ws[1:])  # misaligned workspace
    p.close()


def test_long_1d_lines(ctx):
    # x lines longer than the shared-memory staging of the contiguous solve
    rng = np.random.default_rng(21)
    u = rng.standard_normal(20001)
    check_f64(ctx, u, [random_coords(rng, 20001)])
    r = Runner(ctx, u.shape, None, -1, mgr.MGR_F32, mgr.MGR_PREC_NATIVE)
    try:
        got = r.decompose(u.astype(np.float32))
        assert rel_linf(got, oracle.decompose(u.astype(np.float32).astype(np.float64))) <= TOL32
    finally:
        r.close()
