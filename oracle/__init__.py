"""FP64 CPU oracle for multigrid hierarchical decomposition / recomposition.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library
(``paper_2105_12764_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``mgr_oracle.c`` (plain C, FP64, the steps of
Section II.A of arXiv 2105.12764 in the paper's order); this module is a
ctypes wrapper around it.  Every function here is pinned by the
``-m "not gpu"`` tests in ``tests/test_oracle_pins.py``.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_max_levels.argtypes = [ctypes.c_int, i64p]
        lib.oracle_max_levels.restype = ctypes.c_int
        lib.oracle_default_levels.argtypes = [ctypes.c_int, i64p]
        lib.oracle_default_levels.restype = ctypes.c_int
        for name in ("oracle_decompose", "oracle_recompose"):
            f = getattr(lib, name)
            f.argtypes = [ctypes.c_int, i64p, ctypes.POINTER(dp), ctypes.c_int, dp, dp]
            f.restype = ctypes.c_int
        lib.oracle_mass_1d.argtypes = [ctypes.c_int64, dp, dp, dp, dp]
        lib.oracle_mass_1d.restype = None
        lib.oracle_transfer_1d.argtypes = [ctypes.c_int64, dp, dp]
        lib.oracle_transfer_1d.restype = ctypes.c_int64
        lib.oracle_interp_1d.argtypes = [ctypes.c_int64, dp, dp]
        lib.oracle_interp_1d.restype = ctypes.c_int64
        lib.oracle_class_offsets.argtypes = [ctypes.c_int, i64p, ctypes.c_int, i64p]
        lib.oracle_class_offsets.restype = ctypes.c_int
        lib.oracle_pack_classes.argtypes = [ctypes.c_int, i64p, ctypes.c_int, dp, dp]
        lib.oracle_pack_classes.restype = ctypes.c_int
        lib.oracle_unpack_classes.argtypes = [ctypes.c_int, i64p, ctypes.c_int, ctypes.c_int, dp, dp]
        lib.oracle_unpack_classes.restype = ctypes.c_int
        lib.oracle_quant_bins.argtypes = [ctypes.c_int, i64p, ctypes.POINTER(dp), ctypes.c_int, ctypes.c_double, dp]
        lib.oracle_quant_bins.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _shape_arr(shape):
    return (ctypes.c_int64 * len(shape))(*[int(s) for s in shape])


def max_levels(shape):
    """Deepest allowed hierarchy: coarsenings until the smallest dimension has 2 nodes."""
    lib = _load()
    r = lib.oracle_max_levels(len(shape), _shape_arr(shape))
    if r < 0:
        raise ValueError(f"invalid shape {shape}")
    return r


def default_levels(shape):
    """Default depth (levels=-1): coarsenings until the smallest dimension has 3 nodes."""
    lib = _load()
    r = lib.oracle_default_levels(len(shape), _shape_arr(shape))
    if r < 0:
        raise ValueError(f"invalid shape {shape}")
    return r


def _coords_arg(shape, coords):
    keep = []
    arr = (ctypes.POINTER(ctypes.c_double) * len(shape))()
    for k in range(len(shape)):
        c = None if coords is None else coords[k]
        if c is None:
            arr[k] = ctypes.POINTER(ctypes.c_double)()
        else:
            c = np.ascontiguousarray(c, dtype=np.float64)
            if c.shape != (shape[k],):
                raise ValueError("coordinate array length must match the shape")
            keep.append(c)
            arr[k] = _dptr(c)
    return arr, keep


def _run(fn, u, coords, levels):
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty_like(u)
    carr, keep = _coords_arg(u.shape, coords)
    rc = getattr(lib, fn)(u.ndim, _shape_arr(u.shape), carr, int(levels), _dptr(u), _dptr(out))
    del keep
    if rc == -1:
        raise ValueError(f"{fn}: invalid arguments (shape {u.shape}, levels {levels})")
    if rc != 0:
        raise MemoryError(f"{fn}: allocation failed ({rc})")
    return out


def decompose(u, coords=None, levels=-1):
    """Nodal-layout hierarchical coefficients of ``u`` (FP64), Section II.A."""
    return _run("oracle_decompose", u, coords, levels)


def recompose(c, coords=None, levels=-1):
    """Inverse of :func:`decompose` (Section II.A, recomposition)."""
    return _run("oracle_recompose", c, coords, levels)


def mass_1d(x):
    """(sub, diag, super) of the P1 mass matrix on coordinates ``x``."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    a, b, c = np.empty(n), np.empty(n), np.empty(n)
    lib.oracle_mass_1d(n, _dptr(x), _dptr(a), _dptr(b), _dptr(c))
    return a, b, c


def transfer_1d(x):
    """Dense K = P^T M (m x n) of one level with fine coordinates ``x``."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    m = lib.oracle_transfer_1d(n, _dptr(x), ctypes.POINTER(ctypes.c_double)())
    K = np.empty((m, n))
    lib.oracle_transfer_1d(n, _dptr(x), _dptr(K))
    return K


def interp_1d(x):
    """Dense interpolation P (n x m) of one level with fine coordinates ``x``."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    m = lib.oracle_interp_1d(n, _dptr(x), ctypes.POINTER(ctypes.c_double)())
    P = np.empty((n, m))
    lib.oracle_interp_1d(n, _dptr(x), _dptr(P))
    return P


def class_offsets(shape, levels=-1):
    """Start of every coefficient class in the class-packed layout (length L+2, last = N).

    Class 0 is the coarsest grid N_0, class l the coefficients on N_l \\ N_{l-1}
    (Sec. I, coefficient classes)."""
    lib = _load()
    out = (ctypes.c_int64 * 66)()
    r = lib.oracle_class_offsets(len(shape), _shape_arr(shape), int(levels), out)
    if r < 0:
        raise ValueError(f"invalid shape {shape} / levels {levels}")
    return np.array(out[: r + 1], dtype=np.int64)


def pack_classes(nodal, levels=-1):
    """Nodal layout -> class-packed layout (flat array; classes coarsest first)."""
    lib = _load()
    u = np.ascontiguousarray(nodal, dtype=np.float64)
    out = np.empty(u.size)
    rc = lib.oracle_pack_classes(u.ndim, _shape_arr(u.shape), int(levels), _dptr(u), _dptr(out))
    if rc != 0:
        raise ValueError(f"pack_classes: invalid arguments ({rc})")
    return out


def unpack_classes(packed, shape, nclasses=None, levels=-1):
    """Class-packed layout -> nodal layout keeping classes 0..nclasses-1 (dropped classes are 0)."""
    lib = _load()
    offs = class_offsets(shape, levels)
    if nclasses is None:
        nclasses = len(offs) - 1
    p = np.ascontiguousarray(packed, dtype=np.float64).ravel()
    if p.size < offs[nclasses]:
        raise ValueError("packed input shorter than the requested classes")
    out = np.empty(tuple(shape))
    rc = lib.oracle_unpack_classes(len(shape), _shape_arr(shape), int(levels), int(nclasses), _dptr(p), _dptr(out))
    if rc != 0:
        raise ValueError(f"unpack_classes: invalid arguments ({rc})")
    return out


def recompose_classes(packed, shape, nclasses=None, coords=None, levels=-1):
    """Progressive recomposition: the field rebuilt from classes 0..nclasses-1 of a
    class-packed decomposition, the dropped classes taken as zero."""
    return recompose(unpack_classes(packed, shape, nclasses, levels), coords, levels)


def quant_bins(shape, tau, coords=None, levels=-1):
    """Bin width of every coefficient class (length L+1) for the L-infinity tolerance ``tau``.

    Reading of the quantization stage of Sec. V (the paper does not state the
    quantizer): q_0 = 2 tau/(L+1), q_l = 2 tau/((L+1)(1 + |Z_l|_inf)) with Z_l the
    level-l correction operator, which bounds the recomposed field's error by tau."""
    lib = _load()
    carr, keep = _coords_arg(shape, coords)
    out = np.empty(64)
    r = lib.oracle_quant_bins(len(shape), _shape_arr(shape), carr, int(levels), float(tau), _dptr(out))
    del keep
    if r < 0:
        raise ValueError(f"quant_bins: invalid arguments ({r})")
    return out[:r].copy()


INT32_LIMIT = 2147483647


def quantize(packed, bins, offsets, precision=np.float64):
    """Codes of a class-packed coefficient array: k = round_half_even(c * (1/q_class)).

    The rounding decision is taken in ``precision`` (the arithmetic type of the
    coefficients); |k| is capped at 2^31-1.  Returns (int64 codes, saturated count)."""
    c = np.asarray(packed).astype(precision)
    codes = np.empty(c.shape, dtype=np.int64)
    sat = 0
    for l in range(len(bins)):
        a, b = int(offsets[l]), int(offsets[l + 1])
        qinv = precision(1.0 / float(bins[l]))
        r = np.rint(c[a:b] * qinv)
        bad = ~(np.abs(r) < precision(2147483648.0))
        sat += int(bad.sum())
        r = np.where(bad, np.where(r > 0, INT32_LIMIT, -INT32_LIMIT), r)
        codes[a:b] = r.astype(np.int64)
    return codes, sat


def dequantize(codes, bins, offsets):
    """Class-packed coefficient values k * q_class (FP64)."""
    k = np.asarray(codes, dtype=np.float64)
    out = np.empty(k.shape)
    for l in range(len(bins)):
        a, b = int(offsets[l]), int(offsets[l + 1])
        out[a:b] = k[a:b] * float(bins[l])
    return out


def library_path():
    return _build.build()


__all__ = ["max_levels", "default_levels", "decompose", "recompose", "mass_1d", "transfer_1d", "interp_1d",
           "class_offsets", "pack_classes", "unpack_classes", "recompose_classes", "quant_bins", "quantize",
           "dequantize"]
