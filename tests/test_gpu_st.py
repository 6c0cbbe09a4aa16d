"""GPU parity of the spatiotemporal (3+1)-D form (Sec. III.E: the method in
four dimensions, time slowest) against the FP64 oracle.

Tolerances as for the 3D form: FP64 vs oracle <= 1e-12, FP64 round trip
<= 1e-13, FP32 and mixed forms <= 1e-5 (normwise relative L-infinity).
Shapes cover even and odd time lengths (keep-last in time), several level-pass
tiles with ragged tails, stretched and random coordinates, partial depths.
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
    return mgr.Context(0)


def random_coords(rng, n):
    return np.concatenate([[0.0], np.cumsum(rng.uniform(0.2, 3.0, n - 1))])


def check(ctx, u, coords=None, levels=-1, dtype=mgr.MGR_F64, prec=mgr.MGR_PREC_NATIVE):
    r = Runner(ctx, u.shape, coords, levels, dtype, prec)
    try:
        L = r.plan.levels
        u64 = np.asarray(u, dtype=np.float64)
        ref = oracle.decompose(u64, coords, L)
        got = r.decompose(u)
        tol = TOL64 if dtype == mgr.MGR_F64 else TOL32
        e = rel_linf(got, ref)
        assert e <= tol, f"decompose {u.shape} L={L}: {e:.3e}"
        rt = rel_linf(r.recompose(got), u64)
        assert rt <= (TOL64_RT if dtype == mgr.MGR_F64 else TOL32), f"round trip {u.shape}: {rt:.3e}"
        want = oracle.recompose(ref, coords, L)
        assert rel_linf(r.recompose(ref), want) <= tol
    finally:
        r.close()


SMALL = [(2, 3, 4, 5), (3, 3, 3, 3), (5, 5, 5, 5), (4, 9, 6, 7), (6, 9, 5, 7), (9, 6, 7, 5), (5, 3, 9, 4),
         (8, 5, 6, 9), (9, 9, 9, 9), (10, 7, 12, 11)]


@pytest.mark.parametrize("shape", SMALL)
def test_small(ctx, shape):
    rng = np.random.default_rng(sum(shape))
    u = rng.standard_normal(shape)
    check(ctx, u)
    check(ctx, u, [random_coords(rng, s) for s in shape])
    for L in range(0, oracle.max_levels(shape) + 1):
        check(ctx, u, None, L)


# several level-pass tiles (30 x 14 coarse nodes) and interpolation tiles, ragged tails
MULTI = [(17, 29, 28, 60), (12, 31, 57, 62), (33, 20, 33, 65), (6, 58, 30, 121), (20, 12, 29, 59)]


@pytest.mark.parametrize("shape", MULTI)
def test_multi_tile(ctx, shape):
    rng = np.random.default_rng(sum(shape))
    u = rng.standard_normal(shape)
    check(ctx, u, [random_coords(rng, s) for s in shape])


@pytest.mark.parametrize("form", ["fp32", "mixed"])
def test_fp32_forms(ctx, form):
    shape = (13, 33, 20, 37)
    rng = np.random.default_rng(4)
    coords = [random_coords(rng, s) for s in shape]
    u = rng.standard_normal(shape).astype(np.float32)
    prec = mgr.MGR_PREC_MIXED if form == "mixed" else mgr.MGR_PREC_NATIVE
    check(ctx, u, coords, -1, mgr.MGR_F32, prec)


def test_spatiotemporal_field(ctx):
    """A moving Gaussian bump over 33 time steps on a 33 x 65 x 65 grid: smooth in
    time, so the fine-time coefficients are small."""
    nt, nz, ny, nx = 33, 33, 65, 65
    t, z, y, x = np.meshgrid(np.linspace(0, 1, nt), np.linspace(0, 1, nz), np.linspace(0, 1, ny),
                             np.linspace(0, 1, nx), indexing="ij")
    u = np.exp(-((x - 0.3 - 0.4 * t) ** 2 + (y - 0.5) ** 2 + (z - 0.4 - 0.2 * t) ** 2) / 0.02)
    check(ctx, u)


def test_out_of_place_only_and_nodal_only(ctx):
    shape = (5, 9, 9, 9)
    r = Runner(ctx, shape)
    try:
        with pytest.raises(mgr.MgrError) as ei:
            r.plan.decompose(r.a, r.a, r.ws)
        assert ei.value.code == mgr.MGR_EINVAL
        p = torch.empty(r.a.numel(), dtype=r.a.dtype, device="cuda")
        with pytest.raises(mgr.MgrError) as ei:
            r.plan.decompose_packed(r.a, p, r.ws)
        assert ei.value.code == mgr.MGR_EINVAL
        with pytest.raises(mgr.MgrError) as ei:
            r.plan.class_offsets()
        assert ei.value.code == mgr.MGR_EINVAL
    finally:
        r.close()
