"""Python binding of the GB300 multigrid hierarchical refactoring library.

Argument marshalling only: every step of decomposition / recomposition runs
in the CUDA kernels of ``libmgr.so`` (built from ``csrc/`` for sm_103a).
The functions carry the names of the C ABI in ``include/mgr.h``; the small
``Context`` / ``Plan`` classes only hold handles and pass device pointers
(``torch.Tensor.data_ptr()``) and CUDA stream handles through.

There is no CPU fallback: importing this package raises if ``libmgr.so`` is
missing (build it with ``python -c "import __graft_entry__ as g; g.build()"``).
"""
import ctypes
import os

__all__ = [
    "MGR_OK", "MGR_EINVAL", "MGR_ENOMEM", "MGR_EBUDGET", "MGR_ECUDA", "MGR_EPENDING", "MGR_ETIMEDOUT",
    "MGR_EDEVICE", "MGR_ENOTFOUND", "MGR_EBUSY", "MGR_F32", "MGR_F64", "MGR_PREC_NATIVE", "MGR_PREC_MIXED",
    "MgrError", "mgr_desc", "mgr_kernel_time", "mgr_request", "MGR_OP_DECOMPOSE", "MGR_OP_RECOMPOSE",
    "MGR_OP_DECOMPOSE_PACKED", "MGR_OP_RECOMPOSE_PACKED", "Server", "lib", "library_path", "Context", "Plan", "EXPORTED",
    "PreparedBatch", "plan_tables_host", "fp64_fma_rate",
]

HERE = os.path.dirname(os.path.abspath(__file__))
# MGR_LIBRARY selects another build of the library (the bounds-checking
# libmgr_debug.so); the default is the release build next to this file
_LIB_PATH = os.environ.get("MGR_LIBRARY") or os.path.join(HERE, "libmgr.so")

MGR_OK, MGR_EINVAL, MGR_ENOMEM, MGR_EBUDGET, MGR_ECUDA = 0, -1, -2, -3, -4
MGR_EPENDING, MGR_ETIMEDOUT, MGR_EDEVICE, MGR_ENOTFOUND, MGR_EBUSY = -5, -6, -7, -8, -9
MGR_F32, MGR_F64 = 0, 1
MGR_PREC_NATIVE, MGR_PREC_MIXED = 0, 1
MGR_NOALLOC_SCRATCH_BYTES = 32 << 20


class MgrError(RuntimeError):
    def __init__(self, fn, code):
        self.code = code
        super().__init__(f"{fn} failed: {mgr_strerror(code)} ({code})")


class mgr_desc(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("shape", ctypes.c_int64 * 4),
        ("coords", ctypes.POINTER(ctypes.c_double) * 4),
        ("levels", ctypes.c_int),
        ("dtype", ctypes.c_int),
        ("prec", ctypes.c_int),
    ]


class mgr_kernel_time(ctypes.Structure):
    _fields_ = [
        ("name", ctypes.c_char * 32),
        ("level", ctypes.c_int),
        ("ms", ctypes.c_float),
        ("bytes", ctypes.c_double),
        ("flops", ctypes.c_double),
    ]


class mgr_request(ctypes.Structure):
    _fields_ = [
        ("op", ctypes.c_int),
        ("plan", ctypes.c_void_p),
        ("in_", ctypes.c_void_p),
        ("out", ctypes.c_void_p),
        ("user_tag", ctypes.c_uint64),
        ("keep_resident", ctypes.c_int),
    ]


MGR_OP_DECOMPOSE, MGR_OP_RECOMPOSE = 0, 1
MGR_OP_DECOMPOSE_PACKED, MGR_OP_RECOMPOSE_PACKED = 2, 3  # mgr_profile only


class mgr_serve_request(ctypes.Structure):
    _fields_ = [
        ("op", ctypes.c_int),
        ("plan", ctypes.c_void_p),
        ("in_", ctypes.c_void_p),
        ("src", ctypes.c_uint64),
        ("out", ctypes.c_void_p),
        ("keep_resident", ctypes.c_int),
        ("arrival", ctypes.c_double),
    ]


class mgr_serve_result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("arrival", ctypes.c_double),
        ("admitted", ctypes.c_double),
        ("done", ctypes.c_double),
        ("handle", ctypes.c_uint64),
    ]

_vp = ctypes.c_void_p
_i = ctypes.c_int
# name -> (restype, argtypes): every entry point declared in include/mgr.h
EXPORTED = {
    "mgr_strerror": (ctypes.c_char_p, [_i]),
    "mgr_version": (ctypes.c_char_p, []),
    "mgr_init": (_i, [_i, ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "mgr_shutdown": (_i, [_vp]),
    "mgr_max_levels": (_i, [ctypes.POINTER(mgr_desc), ctypes.POINTER(_i)]),
    "mgr_default_levels": (_i, [ctypes.POINTER(mgr_desc), ctypes.POINTER(_i)]),
    "mgr_plan_tables_host": (_i, [ctypes.POINTER(mgr_desc), _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_i),
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double), _i]),
    "mgr_plan_create": (_i, [_vp, ctypes.POINTER(mgr_desc), ctypes.POINTER(_vp)]),
    "mgr_plan_destroy": (_i, [_vp]),
    "mgr_plan_levels": (_i, [_vp, ctypes.POINTER(_i)]),
    "mgr_workspace_size": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "mgr_decompose": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "mgr_recompose": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "mgr_decompose_host": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "mgr_recompose_host": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "mgr_profile": (_i, [_vp, _i, _vp, _vp, _vp, _vp, ctypes.POINTER(mgr_kernel_time), _i, ctypes.POINTER(_i)]),
    "mgr_decompose_noalloc": (_i, [_vp, _vp, _vp, _vp]),
    "mgr_fp64_fma_rate": (_i, [_i, ctypes.POINTER(ctypes.c_double)]),
    "mgr_debug_bounds": (_i, []),
    "mgr_debug_last": (_i, [ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "mgr_class_offsets": (_i, [_vp, ctypes.POINTER(ctypes.c_int64), _i, ctypes.POINTER(_i)]),
    "mgr_decompose_packed": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "mgr_recompose_packed": (_i, [_vp, _vp, _i, _vp, _vp, _vp]),
    "mgr_pack_classes": (_i, [_vp, _vp, _vp, _vp]),
    "mgr_unpack_classes": (_i, [_vp, _vp, _i, _vp, _vp]),
    "mgr_quant_bins": (_i, [_vp, ctypes.c_double, ctypes.POINTER(ctypes.c_double), _i]),
    "mgr_decompose_quantized": (_i, [_vp, _vp, _vp, ctypes.c_double, _vp, _vp, _vp]),
    "mgr_recompose_dequantized": (_i, [_vp, _vp, _i, ctypes.c_double, _vp, _vp, _vp]),
    "mgr_batch_submit": (_i, [_vp, ctypes.POINTER(mgr_request), _i, ctypes.POINTER(ctypes.c_uint64)]),
    "mgr_batch_poll": (_i, [_vp, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(_i)]),
    "mgr_batch_tuning": (_i, [_vp, ctypes.c_char_p, ctypes.c_size_t]),
    "mgr_serve_now": (ctypes.c_double, []),
    "mgr_serve_start": (_i, [_vp, _i, _i, ctypes.POINTER(_vp)]),
    "mgr_serve_enqueue": (_i, [_vp, ctypes.POINTER(mgr_serve_request), ctypes.POINTER(ctypes.c_uint64)]),
    "mgr_serve_wait": (_i, [_vp, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(mgr_serve_result)]),
    "mgr_serve_hierarchy": (_i, [_vp, ctypes.c_uint64, ctypes.POINTER(_vp)]),
    "mgr_serve_read": (_i, [_vp, ctypes.c_uint64, _vp, _vp]),
    "mgr_serve_release": (_i, [_vp, ctypes.c_uint64]),
    "mgr_serve_stats": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_i), ctypes.POINTER(_i),
                             ctypes.POINTER(_i)]),
    "mgr_serve_stop": (_i, [_vp]),
}


def library_path():
    return _LIB_PATH


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(
            f"{_LIB_PATH} is missing: the multigrid library has no CPU fallback; build it with "
            "`python -c \"import __graft_entry__ as g; g.build()\"`")
    handle = ctypes.CDLL(_LIB_PATH)
    for name, (res, args) in EXPORTED.items():
        f = getattr(handle, name)
        f.restype = res
        f.argtypes = args
    return handle


lib = _load()


def mgr_strerror(code):
    return lib.mgr_strerror(int(code)).decode()


def _check(fn, rc):
    if rc != MGR_OK:
        raise MgrError(fn, rc)


def _ptr(x):
    """Device/host address of a torch tensor, an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def make_desc(shape, coords=None, levels=-1, dtype=MGR_F64, prec=MGR_PREC_NATIVE):
    """Fill an mgr_desc; returns (desc, keepalive) -- keep both alive until plan creation returns."""
    import numpy as np

    d = mgr_desc()
    d.ndim = len(shape)
    for k, s in enumerate(shape):
        d.shape[k] = int(s)
    keep = []
    for k in range(len(shape)):
        c = None if coords is None else coords[k]
        if c is not None:
            c = np.ascontiguousarray(c, dtype=np.float64)
            keep.append(c)
            d.coords[k] = c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.levels = int(levels)
    d.dtype = int(dtype)
    d.prec = int(prec)
    return d, keep


def fp64_fma_rate(device=0):
    """mgr_fp64_fma_rate: measured FP64 FMAs per second of `device` (2 flops each)."""
    v = ctypes.c_double()
    _check("mgr_fp64_fma_rate", lib.mgr_fp64_fma_rate(int(device), ctypes.byref(v)))
    return v.value


def plan_tables_host(shape, coords=None, levels=-1, level=1, axis=0, dtype=MGR_F64, prec=MGR_PREC_NATIVE):
    """mgr_plan_tables_host: the FP64 tables of one axis at one level, built on the
    host (no device).  Returns dict(n, m, wa, wb, k (m x 5), ta, tb) of numpy arrays."""
    import numpy as np

    d, keep = make_desc(shape, coords, levels, dtype, prec)
    n, m = _i(), _i()
    _check("mgr_plan_tables_host", lib.mgr_plan_tables_host(ctypes.byref(d), int(level), int(axis), ctypes.byref(n),
                                                             ctypes.byref(m), None, None, None, None, None, 0))
    cap = max(n.value, 5 * m.value)
    bufs = [np.zeros(cap) for _ in range(5)]
    dp = [b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for b in bufs]
    _check("mgr_plan_tables_host", lib.mgr_plan_tables_host(ctypes.byref(d), int(level), int(axis), ctypes.byref(n),
                                                             ctypes.byref(m), *dp, cap))
    del keep
    nn, mm = n.value, m.value
    return dict(n=nn, m=mm, wa=bufs[0][:nn].copy(), wb=bufs[1][:nn].copy(), k=bufs[2][:5 * mm].reshape(mm, 5).copy(),
                ta=bufs[3][:mm].copy(), tb=bufs[4][:mm].copy())


class Context:
    """mgr_init / mgr_shutdown."""

    def __init__(self, device=0, mem_budget_bytes=0):
        h = _vp()
        _check("mgr_init", lib.mgr_init(int(device), int(mem_budget_bytes), ctypes.byref(h)))
        self.handle = h.value
        self.device = device

    def close(self):
        if self.handle:
            _check("mgr_shutdown", lib.mgr_shutdown(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @staticmethod
    def batch_prepare(requests):
        """The mgr_request array of a request list, marshalled once: a list that is
        submitted again and again (every step of a loop) can be passed to
        batch_submit as this object, without re-marshalling thousands of entries
        per call.  Holds references to the plans and tensors it names."""
        return PreparedBatch(requests)

    def batch_submit(self, requests):
        """mgr_batch_submit; requests: iterable of (op, plan, in, out[, user_tag]), or a
        PreparedBatch (batch_prepare).  Returns the ticket."""
        pb = requests if isinstance(requests, PreparedBatch) else PreparedBatch(requests)
        t = ctypes.c_uint64()
        _check("mgr_batch_submit", lib.mgr_batch_submit(self.handle, pb.arr, pb.n, ctypes.byref(t)))
        return t.value

    def batch_poll(self, ticket, timeout_us=-1):
        """mgr_batch_poll: returns (code, n_done); raises only on errors other than pending/timeout."""
        n = _i()
        rc = lib.mgr_batch_poll(self.handle, int(ticket), int(timeout_us), ctypes.byref(n))
        if rc not in (MGR_OK, MGR_EPENDING, MGR_ETIMEDOUT):
            raise MgrError("mgr_batch_poll", rc)
        return rc, n.value

    def batch_tuning(self):
        buf = ctypes.create_string_buffer(1 << 16)
        lib.mgr_batch_tuning(self.handle, buf, len(buf))
        return buf.value.decode()


class PreparedBatch:
    """A marshalled mgr_request array (see Context.batch_prepare)."""

    def __init__(self, requests):
        reqs = list(requests)
        self.n = len(reqs)
        self.arr = (mgr_request * max(1, self.n))()
        self._refs = reqs  # the plans and buffers must outlive the array's use
        for i, r in enumerate(reqs):
            op, plan, src, dst = r[:4]
            self.arr[i].op = int(op)
            self.arr[i].plan = plan.handle
            self.arr[i].in_ = _ptr(src)
            self.arr[i].out = _ptr(dst)
            self.arr[i].user_tag = int(r[4]) if len(r) > 4 else i
            self.arr[i].keep_resident = 0


class Plan:
    """mgr_plan_create / mgr_decompose / mgr_recompose on device pointers."""

    def __init__(self, ctx, shape, coords=None, levels=-1, dtype=MGR_F64, prec=MGR_PREC_NATIVE):
        d, keep = make_desc(shape, coords, levels, dtype, prec)
        h = _vp()
        _check("mgr_plan_create", lib.mgr_plan_create(ctx.handle, ctypes.byref(d), ctypes.byref(h)))
        del keep
        self.handle = h.value
        self.ctx = ctx
        self.shape = tuple(int(s) for s in shape)
        self.dtype = dtype
        self.prec = prec
        lv = _i()
        _check("mgr_plan_levels", lib.mgr_plan_levels(self.handle, ctypes.byref(lv)))
        self.levels = lv.value
        ws = ctypes.c_size_t()
        _check("mgr_workspace_size", lib.mgr_workspace_size(self.handle, ctypes.byref(ws)))
        self.workspace_bytes = ws.value

    def decompose(self, inp, out, workspace, stream=None):
        _check("mgr_decompose", lib.mgr_decompose(self.handle, _ptr(inp), _ptr(out), _ptr(workspace), _stream(stream)))

    def recompose(self, inp, out, workspace, stream=None):
        _check("mgr_recompose", lib.mgr_recompose(self.handle, _ptr(inp), _ptr(out), _ptr(workspace), _stream(stream)))

    def decompose_noalloc(self, inp, out, stream=None):
        """mgr_decompose_noalloc: no workspace argument, no device allocation (fields whose workspace
        fits MGR_NOALLOC_SCRATCH_BYTES; calls that overlap on the GPU must be serialised)."""
        _check("mgr_decompose_noalloc", lib.mgr_decompose_noalloc(self.handle, _ptr(inp), _ptr(out), _stream(stream)))

    def class_offsets(self):
        """mgr_class_offsets: start of every coefficient class in the class-packed layout (L+2 entries)."""
        arr = (ctypes.c_int64 * (self.levels + 2))()
        n = _i()
        _check("mgr_class_offsets", lib.mgr_class_offsets(self.handle, arr, self.levels + 2, ctypes.byref(n)))
        return list(arr)

    def decompose_packed(self, inp, out, workspace, stream=None):
        _check("mgr_decompose_packed", lib.mgr_decompose_packed(self.handle, _ptr(inp), _ptr(out), _ptr(workspace),
                                                                _stream(stream)))

    def recompose_packed(self, inp, nclasses, out, workspace, stream=None):
        """mgr_recompose_packed: the field from classes 0..nclasses-1 (dropped classes are zero)."""
        _check("mgr_recompose_packed", lib.mgr_recompose_packed(self.handle, _ptr(inp), int(nclasses), _ptr(out),
                                                                _ptr(workspace), _stream(stream)))

    def pack_classes(self, nodal, packed, stream=None):
        _check("mgr_pack_classes", lib.mgr_pack_classes(self.handle, _ptr(nodal), _ptr(packed), _stream(stream)))

    def unpack_classes(self, packed, nclasses, nodal, stream=None):
        _check("mgr_unpack_classes", lib.mgr_unpack_classes(self.handle, _ptr(packed), int(nclasses), _ptr(nodal),
                                                            _stream(stream)))

    def quant_bins(self, tau):
        """mgr_quant_bins: bin width of every class (L+1 entries) for the max-norm tolerance tau."""
        arr = (ctypes.c_double * (self.levels + 1))()
        _check("mgr_quant_bins", lib.mgr_quant_bins(self.handle, float(tau), arr, self.levels + 1))
        return list(arr)

    def decompose_quantized(self, inp, codes, tau, workspace, saturated=None, stream=None):
        """mgr_decompose_quantized: int32 codes (class-packed) of the decomposition of `inp`."""
        _check("mgr_decompose_quantized", lib.mgr_decompose_quantized(
            self.handle, _ptr(inp), _ptr(codes), float(tau), _ptr(workspace), _ptr(saturated), _stream(stream)))

    def recompose_dequantized(self, codes, nclasses, tau, out, workspace, stream=None):
        _check("mgr_recompose_dequantized", lib.mgr_recompose_dequantized(
            self.handle, _ptr(codes), int(nclasses), float(tau), _ptr(out), _ptr(workspace), _stream(stream)))

    def decompose_host(self, host_in, host_out, dev_in, dev_out, workspace, stream=None):
        _check("mgr_decompose_host", lib.mgr_decompose_host(self.handle, _ptr(host_in), _ptr(host_out), _ptr(dev_in),
                                                            _ptr(dev_out), _ptr(workspace), _stream(stream)))

    def recompose_host(self, host_in, host_out, dev_in, dev_out, workspace, stream=None):
        _check("mgr_recompose_host", lib.mgr_recompose_host(self.handle, _ptr(host_in), _ptr(host_out), _ptr(dev_in),
                                                            _ptr(dev_out), _ptr(workspace), _stream(stream)))

    def profile(self, op, inp, out, workspace, stream=None, cap=512):
        """mgr_profile: list of dicts (name, level, ms, bytes, flops), one per kernel launch."""
        arr = (mgr_kernel_time * cap)()
        n = _i()
        _check("mgr_profile", lib.mgr_profile(self.handle, int(op), _ptr(inp), _ptr(out), _ptr(workspace),
                                              _stream(stream), arr, cap, ctypes.byref(n)))
        return [dict(name=arr[i].name.decode(), level=arr[i].level, ms=arr[i].ms, bytes=arr[i].bytes,
                     flops=arr[i].flops) for i in range(min(n.value, cap))]

    def close(self):
        if self.handle:
            _check("mgr_plan_destroy", lib.mgr_plan_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def max_levels(shape):
    d, keep = make_desc(shape)
    v = _i()
    _check("mgr_max_levels", lib.mgr_max_levels(ctypes.byref(d), ctypes.byref(v)))
    return v.value


def default_levels(shape):
    d, keep = make_desc(shape)
    v = _i()
    _check("mgr_default_levels", lib.mgr_default_levels(ctypes.byref(d), ctypes.byref(v)))
    return v.value


class Server:
    """mgr_serve_*: continuous-batching request loop on one context."""

    def __init__(self, ctx, slots=4, streams=4):
        h = _vp()
        _check("mgr_serve_start", lib.mgr_serve_start(ctx.handle, int(slots), int(streams), ctypes.byref(h)))
        self.handle = h.value
        self.ctx = ctx

    @staticmethod
    def now():
        return lib.mgr_serve_now()

    def enqueue(self, op, plan, inp=None, src=0, out=None, keep_resident=1, arrival=0.0):
        r = mgr_serve_request()
        r.op = int(op)
        r.plan = plan.handle
        r.in_ = _ptr(inp)
        r.src = int(src)
        r.out = _ptr(out)
        r.keep_resident = int(keep_resident)
        r.arrival = float(arrival)
        i = ctypes.c_uint64()
        _check("mgr_serve_enqueue", lib.mgr_serve_enqueue(self.handle, ctypes.byref(r), ctypes.byref(i)))
        return i.value

    def wait(self, rid, timeout_us=-1):
        """Returns (code, result dict or None)."""
        res = mgr_serve_result()
        rc = lib.mgr_serve_wait(self.handle, int(rid), int(timeout_us), ctypes.byref(res))
        if rc in (MGR_EPENDING, MGR_ETIMEDOUT):
            return rc, None
        _check("mgr_serve_wait", rc)
        return rc, dict(status=res.status, arrival=res.arrival, admitted=res.admitted, done=res.done,
                        handle=res.handle)

    def hierarchy(self, handle):
        p = _vp()
        _check("mgr_serve_hierarchy", lib.mgr_serve_hierarchy(self.handle, int(handle), ctypes.byref(p)))
        return p.value

    def read(self, handle, dst, stream=None):
        """mgr_serve_read: copy a finished resident hierarchy into device buffer `dst`."""
        _check("mgr_serve_read", lib.mgr_serve_read(self.handle, int(handle), _ptr(dst), _stream(stream)))

    def release(self, handle):
        return lib.mgr_serve_release(self.handle, int(handle))

    def stats(self):
        u, q, r, h = ctypes.c_size_t(), _i(), _i(), _i()
        _check("mgr_serve_stats", lib.mgr_serve_stats(self.handle, ctypes.byref(u), ctypes.byref(q), ctypes.byref(r),
                                                      ctypes.byref(h)))
        return dict(used_bytes=u.value, queued=q.value, running=r.value, resident=h.value)

    def stop(self):
        if self.handle:
            _check("mgr_serve_stop", lib.mgr_serve_stop(self.handle))
            self.handle = None

