"""GPU parity of the coefficient-class layout (Sec. I: coefficient classes,
approximations rebuilt from a prefix of them) against the FP64 oracle.

* mgr_decompose_packed = oracle.pack_classes(oracle.decompose(u))   <= 1e-12
* mgr_recompose_packed from classes 0..k-1 = oracle.recompose_classes <= 1e-12
  (the dense-projection pin of the oracle makes this Q_{k-1} u)
* every class, exact round trip                                      <= 1e-13
* mgr_pack_classes / mgr_unpack_classes: bit-exact permutations
* FP32 and mixed forms                                                <= 1e-5
"""
import numpy as np
import pytest

import oracle
import paper_2105_12764_gb300 as mgr
from gpu_util import np_dtype, rel_linf, torch_dtype

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


class Packed:
    def __init__(self, ctx, shape, coords=None, levels=-1, dtype=mgr.MGR_F64, prec=mgr.MGR_PREC_NATIVE):
        self.plan = mgr.Plan(ctx, shape, coords, levels, dtype, prec)
        self.shape = tuple(shape)
        self.td, self.nd = torch_dtype(dtype), np_dtype(dtype)
        self.ws = torch.empty(max(self.plan.workspace_bytes, 256), dtype=torch.uint8, device="cuda")
        self.x = torch.empty(self.shape, dtype=self.td, device="cuda")
        self.p = torch.empty(int(np.prod(self.shape)), dtype=self.td, device="cuda")
        self.y = torch.empty(self.shape, dtype=self.td, device="cuda")

    def decompose(self, u):
        self.x.copy_(torch.from_numpy(np.ascontiguousarray(u, dtype=self.nd)))
        self.plan.decompose_packed(self.x, self.p, self.ws)
        torch.cuda.synchronize()
        return self.p.cpu().numpy()

    def recompose(self, packed, k):
        self.p.copy_(torch.from_numpy(np.ascontiguousarray(packed, dtype=self.nd)))
        self.plan.recompose_packed(self.p, k, self.y, self.ws)
        torch.cuda.synchronize()
        return self.y.cpu().numpy()

    def close(self):
        self.plan.close()


def check(ctx, u, coords=None, levels=-1, all_prefixes=True):
    r = Packed(ctx, u.shape, coords, levels)
    try:
        L = r.plan.levels
        assert r.plan.class_offsets() == list(oracle.class_offsets(u.shape, L))
        ref = oracle.pack_classes(oracle.decompose(u, coords, L), L)
        got = r.decompose(u)
        assert rel_linf(got, ref) <= TOL64, f"decompose_packed {u.shape}: {rel_linf(got, ref):.3e}"
        assert rel_linf(r.recompose(got, L + 1), u) <= TOL64_RT
        for k in (range(1, L + 2) if all_prefixes else [1, L, L + 1]):
            if k < 1:
                continue
            want = oracle.recompose_classes(ref, u.shape, k, coords, L)
            e = rel_linf(r.recompose(ref, k), want)
            assert e <= TOL64, f"recompose_packed {u.shape} classes {k}: {e:.3e}"
    finally:
        r.close()


@pytest.mark.parametrize("n", list(range(2, 34)))
def test_1d_sizes(ctx, n):
    rng = np.random.default_rng(n)
    u = rng.standard_normal(n)
    check(ctx, u)
    check(ctx, u, [random_coords(rng, n)], oracle.max_levels((n,)))


@pytest.mark.parametrize("n", list(range(2, 34, 3)))
def test_2d_3d_sizes(ctx, n):
    rng = np.random.default_rng(50 + n)
    for shape in [(n, 9), (9, n), (n, 5, 6), (5, n, 6), (5, 6, n)]:
        u = rng.standard_normal(shape)
        check(ctx, u, [random_coords(rng, s) for s in shape])


# several level-pass tiles (30 x 14 coarse nodes) and interpolation tiles
# (32 x 16) with ragged tails and keep-last ends
MULTI = [(29, 28, 60), (58, 60, 121), (31, 57, 62), (12, 29, 59), (70, 45, 66), (2, 64, 130), (256, 300)]


@pytest.mark.parametrize("shape", MULTI)
def test_multi_tile(ctx, shape):
    rng = np.random.default_rng(sum(shape))
    u = rng.standard_normal(shape)
    check(ctx, u, [random_coords(rng, s) for s in shape], all_prefixes=len(shape) == 2)
    check(ctx, u, None, levels=min(2, oracle.max_levels(shape)), all_prefixes=True)


def test_packed_equals_pack_of_nodal(ctx):
    """The fused class-packed decomposition writes the same values as the
    nodal one followed by the conversion kernel: bit for bit on the levels both
    run through the tiled kernels, to rounding on the coarse levels the nodal
    form finishes in its single-CTA kernel."""
    shape = (45, 61, 70)
    rng = np.random.default_rng(3)
    u = torch.from_numpy(rng.standard_normal(shape)).cuda()
    plan = mgr.Plan(ctx, shape, None, -1, mgr.MGR_F64)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    nodal, p1, p2 = torch.empty_like(u), torch.empty(u.numel(), dtype=u.dtype, device="cuda"), \
        torch.empty(u.numel(), dtype=u.dtype, device="cuda")
    plan.decompose(u, nodal, ws)
    plan.pack_classes(nodal, p1)
    plan.decompose_packed(u, p2, ws)
    torch.cuda.synchronize()
    offs = plan.class_offsets()
    L = plan.levels
    a, b = p1.cpu().numpy(), p2.cpu().numpy()
    # the finest class comes from the same tiled level pass in both forms
    assert np.array_equal(a[offs[L]:], b[offs[L]:])
    assert rel_linf(a, b) <= 1e-13
    plan.close()


@pytest.mark.parametrize("dtype", [mgr.MGR_F64, mgr.MGR_F32])
@pytest.mark.parametrize("shape", [(17,), (40, 33), (9, 21, 70), (33, 20, 37)])
def test_pack_unpack_bit_exact(ctx, dtype, shape):
    plan = mgr.Plan(ctx, shape, None, -1, dtype)
    L = plan.levels
    rng = np.random.default_rng(7)
    x = rng.standard_normal(shape).astype(np_dtype(dtype))
    xd = torch.from_numpy(x).cuda()
    pk = torch.empty(x.size, dtype=xd.dtype, device="cuda")
    plan.pack_classes(xd, pk)
    torch.cuda.synchronize()
    want = oracle.pack_classes(x.astype(np.float64), L)
    np.testing.assert_array_equal(pk.cpu().numpy().astype(np.float64), want)
    back = torch.empty_like(xd)
    for k in range(1, L + 2):
        plan.unpack_classes(pk, k, back)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(back.cpu().numpy().astype(np.float64),
                                      oracle.unpack_classes(want, shape, k, L))
    plan.close()


@pytest.mark.parametrize("form", ["fp32", "mixed"])
def test_fp32_forms(ctx, form):
    shape = (33, 40, 71)
    rng = np.random.default_rng(11)
    coords = [random_coords(rng, s) for s in shape]
    u = rng.standard_normal(shape).astype(np.float32)
    prec = mgr.MGR_PREC_MIXED if form == "mixed" else mgr.MGR_PREC_NATIVE
    r = Packed(ctx, shape, coords, -1, mgr.MGR_F32, prec)
    try:
        L = r.plan.levels
        u64 = u.astype(np.float64)
        ref = oracle.pack_classes(oracle.decompose(u64, coords, L), L)
        got = r.decompose(u)
        assert rel_linf(got, ref) <= TOL32
        assert rel_linf(r.recompose(got, L + 1), u64) <= TOL32
        for k in range(1, L + 1):
            want = oracle.recompose_classes(ref, shape, k, coords, L)
            assert rel_linf(r.recompose(ref.astype(np.float32), k), want) <= TOL32
    finally:
        r.close()


def test_prefix_reads_only_its_classes(ctx):
    """The classes after the prefix are never read: NaN there changes nothing."""
    shape = (40, 50, 61)
    rng = np.random.default_rng(2)
    u = rng.standard_normal(shape)
    r = Packed(ctx, shape)
    try:
        L = r.plan.levels
        offs = r.plan.class_offsets()
        packed = r.decompose(u)
        for k in (1, 2, L):
            tail = packed.copy()
            tail[offs[k]:] = np.nan
            got = r.recompose(tail, k)
            assert np.isfinite(got).all()
            assert rel_linf(got, oracle.recompose_classes(packed, shape, k, None, L)) <= TOL64
    finally:
        r.close()


def test_invalid_arguments(ctx):
    shape = (17, 18, 19)
    r = Packed(ctx, shape)
    L = r.plan.levels
    for k in (0, L + 2, -1):
        with pytest.raises(mgr.MgrError) as ei:
            r.plan.recompose_packed(r.p, k, r.y, r.ws)
        assert ei.value.code == mgr.MGR_EINVAL
        with pytest.raises(mgr.MgrError) as ei:
            r.plan.unpack_classes(r.p, k, r.y)
        assert ei.value.code == mgr.MGR_EINVAL
    # in == out and partial overlap are refused for the packed forms
    with pytest.raises(mgr.MgrError) as ei:
        r.plan.decompose_packed(r.x, r.x, r.ws)
    assert ei.value.code == mgr.MGR_EINVAL
    with pytest.raises(mgr.MgrError) as ei:
        r.plan.recompose_packed(r.x, L + 1, r.x, r.ws)
    assert ei.value.code == mgr.MGR_EINVAL
    big = torch.empty(2 * r.x.numel(), dtype=r.x.dtype, device="cuda")
    with pytest.raises(mgr.MgrError) as ei:
        r.plan.pack_classes(big, big[5:])
    assert ei.value.code == mgr.MGR_EINVAL
    r.close()


def test_levels_zero(ctx):
    u = np.random.default_rng(0).standard_normal((6, 7))
    r = Packed(ctx, u.shape, None, 0)
    try:
        assert r.plan.class_offsets() == [0, 42]
        np.testing.assert_array_equal(r.decompose(u), u.ravel())
        np.testing.assert_array_equal(r.recompose(u.ravel(), 1), u)
    finally:
        r.close()


def test_profile_packed_ops(ctx):
    shape = (65, 65, 65)
    r = Packed(ctx, shape)
    r.x.normal_()
    recs = r.plan.profile(mgr.MGR_OP_DECOMPOSE_PACKED, r.x, r.p, r.ws)
    assert any(x["name"] == "level_load_dec" for x in recs)
    recs = r.plan.profile(mgr.MGR_OP_RECOMPOSE_PACKED, r.p, r.y, r.ws)
    assert any(x["name"] == "interp" for x in recs)
    torch.cuda.synchronize()
    assert rel_linf(r.y.cpu().numpy(), r.x.cpu().numpy()) <= TOL64_RT
    r.close()
