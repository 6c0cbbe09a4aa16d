"""The C ABI library (no GPU needed): it builds, loads, exports every entry
point that include/mgr.h declares, the Python binding covers exactly those,
and the host-only entry points agree with the oracle's hierarchy depths."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mgr.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|int|double)\s+(mgr_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    import importlib.util

    spec = importlib.util.spec_from_file_location("mgr_build", os.path.join(ROOT, "paper_2105_12764_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b.build()


def test_header_declares_the_entry_points():
    names = declared()
    for must in ("mgr_init", "mgr_plan_create", "mgr_decompose", "mgr_recompose", "mgr_decompose_packed",
                 "mgr_recompose_packed", "mgr_batch_submit", "mgr_serve_start", "mgr_decompose_noalloc"):
        assert must in names
    assert len(names) >= 30


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True)
    if out.returncode == 0:
        exported = set(re.findall(r"\sT\s(mgr_\w+)", out.stdout))
        assert set(declared()) <= exported


def test_binding_covers_exactly_the_header(lib_path):
    import paper_2105_12764_gb300 as mgr

    assert sorted(mgr.EXPORTED) == declared()


def test_host_only_entry_points(lib_path):
    import oracle
    import paper_2105_12764_gb300 as mgr

    assert mgr.lib.mgr_version().decode().count(".") == 2
    assert mgr.mgr_strerror(mgr.MGR_EINVAL) == "invalid argument"
    for shape in [(2,), (5,), (65,), (513,), (1000, 700, 300), (17, 17), (24, 9, 33), (3, 100), (9, 17, 33, 65)]:
        assert mgr.max_levels(shape) == oracle.max_levels(shape)
        assert mgr.default_levels(shape) == oracle.default_levels(shape)
    with pytest.raises(mgr.MgrError):
        mgr.max_levels((1, 5))
    # planes of 2^31 nodes or more are refused (32-bit in-plane offsets)
    assert mgr.max_levels((3, 46340, 46340)) == 1
    for shape in [(2, 46341, 46341), (65536, 32768), (5, 2048, 1024, 1024)]:
        with pytest.raises(mgr.MgrError) as ei:
            mgr.max_levels(shape)
        assert ei.value.code == mgr.MGR_EINVAL


def test_no_device_fails_loudly(lib_path):
    """Without a GPU the product path reports an error; there is no CPU fallback."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import paper_2105_12764_gb300 as mgr

    with pytest.raises(mgr.MgrError) as ei:
        mgr.Context(0)
    assert ei.value.code in (mgr.MGR_ECUDA, mgr.MGR_EINVAL)


def test_class_offsets_match_oracle_without_device():
    """Class sizes on the host side of the ABI come from the plan; here the
    closed form |N_l| - |N_{l-1}| is recomputed from the level-size rule
    n -> n//2 + 1 used by both sides, and compared with the oracle."""
    import oracle

    for shape in [(5,), (33, 20, 37), (24, 9, 33), (1000, 700, 300)]:
        L = oracle.default_levels(shape)
        sizes = [list(shape)]
        for _ in range(L):
            sizes.append([s // 2 + 1 for s in sizes[-1]])
        sizes = sizes[::-1]
        cnt = [int(np.prod(s)) for s in sizes]
        expect = np.cumsum([0, cnt[0]] + [cnt[l] - cnt[l - 1] for l in range(1, L + 1)])
        if np.prod(shape) < 5e6:
            np.testing.assert_array_equal(oracle.class_offsets(shape, L), expect)


def test_bounds_checking_variant_exports_the_same_abi(lib_path):
    """libmgr_debug.so (MGR_DEBUG_BOUNDS) exports every declared symbol and says
    it checks; the release build says it does not (no GPU needed for either)."""
    import importlib.util

    spec = importlib.util.spec_from_file_location("mgr_build2", os.path.join(ROOT, "paper_2105_12764_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    dbg = ctypes.CDLL(b.build(debug_bounds=True))
    missing = [n for n in declared() if not hasattr(dbg, n)]
    assert not missing, missing
    assert dbg.mgr_debug_bounds() == 1
    assert ctypes.CDLL(lib_path).mgr_debug_bounds() == 0
    code = ctypes.c_int()
    idx, ext = ctypes.c_int64(), ctypes.c_int64()
    assert dbg.mgr_debug_last(ctypes.byref(code), ctypes.byref(idx), ctypes.byref(ext)) == -8  # MGR_ENOTFOUND
