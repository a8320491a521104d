"""ctypes binding of libsarabande_gb300.so: argument marshalling only.

Every function of the C ABI (include/sarabande_gb300.h) is exposed under the
same name; `Context` adds allocation of the float64 output arrays.  Fields may
be numpy arrays (host) or CUDA torch tensors (device; SBG_FIELD_ON_DEVICE is set
automatically).  There is no fallback: if the library is missing, loading
raises.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsarabande_gb300.so")

SBG_OK = 0
SBG_F32, SBG_F64 = 0, 1
SBG_PREC_FP32, SBG_PREC_BF16X3, SBG_PREC_TF32X3 = 0, 1, 3
HAS_BF16X3 = True  # the tcgen05 split-BF16 4PCF combination is built in
SBG_3PCF, SBG_4PCF, SBG_NORMALIZED, SBG_SUBTRACT_MEAN, SBG_FIELD_ON_DEVICE = 1, 2, 4, 8, 16
(SBG_ERR_INVALID_ARG, SBG_ERR_UNSUPPORTED_SHAPE, SBG_ERR_BIN_RANGE, SBG_ERR_EMPTY_BIN, SBG_ERR_OUT_OF_MEMORY,
 SBG_ERR_CUDA, SBG_ERR_TIMEOUT, SBG_ERR_INTERNAL) = (-1, -2, -3, -4, -5, -6, -7, -8)
STATUS = {0: "SBG_OK", -1: "SBG_ERR_INVALID_ARG", -2: "SBG_ERR_UNSUPPORTED_SHAPE", -3: "SBG_ERR_BIN_RANGE",
          -4: "SBG_ERR_EMPTY_BIN", -5: "SBG_ERR_OUT_OF_MEMORY", -6: "SBG_ERR_CUDA", -7: "SBG_ERR_TIMEOUT",
          -8: "SBG_ERR_INTERNAL"}

_lib = None


class SbgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Field2D(ctypes.Structure):
    _fields_ = [("field", ctypes.c_void_p), ("dtype", ctypes.c_int), ("shape", ctypes.c_int64 * 2),
                ("edges", ctypes.c_void_p), ("zeta3", ctypes.c_void_p), ("zeta4", ctypes.c_void_p)]


def lib():
    """Load the library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, st = ctypes.c_void_p, ctypes.c_int, ctypes.c_int
        L.sbg_create.argtypes = [i, ctypes.c_size_t, ctypes.POINTER(vp)]
        L.sbg_create.restype = st
        L.sbg_destroy.argtypes = [vp]
        L.sbg_destroy.restype = None
        L.sbg_set_stream.argtypes = [vp, vp]
        L.sbg_set_stream.restype = st
        L.sbg_status_string.argtypes = [st]
        L.sbg_status_string.restype = ctypes.c_char_p
        L.sbg_last_error.argtypes = [vp]
        L.sbg_last_error.restype = ctypes.c_char_p
        L.sbg_lambda_count.argtypes = [i, ctypes.POINTER(i)]
        L.sbg_lambda_count.restype = st
        L.sbg_lambda_list.argtypes = [i, vp]
        L.sbg_lambda_list.restype = st
        L.sbg_full.argtypes = [vp, vp, i, vp, vp, i, i, i, i, ctypes.c_uint, vp, vp]
        L.sbg_full.restype = st
        L.sbg_projected.argtypes = [vp, vp, i, vp, vp, i, i, i, ctypes.c_uint, vp, vp]
        L.sbg_projected.restype = st
        L.sbg_projected_batch.argtypes = [vp, ctypes.POINTER(Field2D), i, i, i, i, ctypes.c_uint]
        L.sbg_projected_batch.restype = st
        L.sbg_last_timings.argtypes = [vp, vp, ctypes.POINTER(i)]
        L.sbg_last_timings.restype = st
        L.sbg_last_contraction_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        L.sbg_last_contraction_ms.restype = st
        L.sbg_plan4_info.argtypes = [i, i, i, i, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
        L.sbg_projected_slices.argtypes = [vp, vp, i, vp, vp, i, i, i, ctypes.c_uint, vp, vp]
        L.sbg_projected_slices.restype = st
        L.sbg_unique_bins.argtypes = [i, i, ctypes.POINTER(i), vp]
        L.sbg_unique_bins.restype = st
        L.sbg_unique_gather.argtypes = [vp, ctypes.c_longlong, i, i, i, vp]
        L.sbg_unique_gather.restype = st
        L.sbg_zero_overlap.argtypes = [vp, ctypes.c_longlong, i, i, i]
        L.sbg_zero_overlap.restype = st
        L.sbg_lambda_odd_count.argtypes = [i, ctypes.POINTER(i)]
        L.sbg_lambda_odd_count.restype = st
        L.sbg_lambda_odd_list.argtypes = [i, vp]
        L.sbg_lambda_odd_list.restype = st
        L.sbg_full_odd.argtypes = [vp, vp, i, vp, vp, i, i, i, ctypes.c_uint, vp]
        L.sbg_full_odd.restype = st
        L.sbg_plan4_info.restype = st
        L.sbg_projected3_noalloc.argtypes = [vp, i, ctypes.c_int64, vp, i, i, ctypes.c_uint, vp, vp]
        L.sbg_projected3_noalloc.restype = st
        L.sbg_set_wait_limit.argtypes = [vp, ctypes.c_ulonglong, i]
        L.sbg_set_wait_limit.restype = st
        L.sbg_autotune_report.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
        L.sbg_autotune_report.restype = st
        L.sbg_set_autotune.argtypes = [vp, i]
        L.sbg_set_autotune.restype = st
        _lib = L
    return _lib


# ---- same-name wrappers of the C ABI ----
def sbg_create(device=0, budget=0):
    h = ctypes.c_void_p()
    s = lib().sbg_create(device, budget, ctypes.byref(h))
    if s != SBG_OK:
        raise SbgError(s, "sbg_create failed")
    return h


def sbg_destroy(h):
    lib().sbg_destroy(h)


def sbg_set_stream(h, stream):
    return lib().sbg_set_stream(h, ctypes.c_void_p(stream))


def sbg_set_wait_limit(h, wait_ns, test_stall=0):
    return lib().sbg_set_wait_limit(h, int(wait_ns), int(test_stall))


def sbg_set_autotune(h, enable):
    return lib().sbg_set_autotune(h, int(enable))


def sbg_autotune_report(h):
    """The autotuner's choices so far as a dict key -> choice."""
    need = ctypes.c_size_t()
    lib().sbg_autotune_report(h, None, 0, ctypes.byref(need))
    buf = ctypes.create_string_buffer(need.value)
    lib().sbg_autotune_report(h, buf, need.value, None)
    out = {}
    for line in buf.value.decode().splitlines():
        k, v = line.rsplit("=", 1)
        out[k] = int(v)
    return out


def sbg_status_string(s):
    return lib().sbg_status_string(s).decode()


def sbg_last_error(h):
    return lib().sbg_last_error(h).decode()


def sbg_lambda_count(lmax):
    n = ctypes.c_int()
    s = lib().sbg_lambda_count(lmax, ctypes.byref(n))
    if s != SBG_OK:
        raise SbgError(s, "sbg_lambda_count")
    return n.value


def sbg_lambda_list(lmax):
    n = sbg_lambda_count(lmax)
    out = np.zeros((n, 3), dtype=np.int32)
    s = lib().sbg_lambda_list(lmax, out.ctypes.data)
    if s != SBG_OK:
        raise SbgError(s, "sbg_lambda_list")
    return out


def sbg_projected_slices(h, cube, edges, mmax, prec, flags, zeta3=None, zeta4=None):
    ptr, dt, shape, on_dev, keep = _field_ptr(cube)
    if len(shape) != 3:
        raise ValueError("cube must be 3D")
    e = _edges(edges)
    nb = len(e) - 1
    if on_dev:
        flags |= SBG_FIELD_ON_DEVICE
    w = 2 * mmax + 1
    zeta3 = _out(zeta3, (shape[0], mmax + 1, nb, nb, 2), "zeta3") if flags & SBG_3PCF else None
    zeta4 = _out(zeta4, (shape[0], w, w, nb, nb, nb, 2), "zeta4") if flags & SBG_4PCF else None
    shp = (ctypes.c_int64 * 3)(*shape)
    s = lib().sbg_projected_slices(h, ptr, dt, shp, e.ctypes.data, nb, mmax, prec, flags,
                                   zeta3.ctypes.data if zeta3 is not None else None,
                                   zeta4.ctypes.data if zeta4 is not None else None)
    del keep
    if s != SBG_OK:
        raise SbgError(s, sbg_last_error(h))
    return zeta3, zeta4


def sbg_unique_bins(nbins, order):
    """[n_index, order - 1] bin combinations in the 1D bin-index order."""
    n = ctypes.c_int()
    s = lib().sbg_unique_bins(nbins, order, ctypes.byref(n), None)
    if s != SBG_OK:
        raise SbgError(s, "sbg_unique_bins")
    out = np.zeros((max(n.value, 1), order - 1), dtype=np.int32)
    s = lib().sbg_unique_bins(nbins, order, ctypes.byref(n), out.ctypes.data)
    if s != SBG_OK:
        raise SbgError(s, "sbg_unique_bins")
    return out[:n.value]


def sbg_unique_gather(zeta, order, ncomp=1):
    """Unique coefficients of a dense output: zeta of shape [..., nbins x
    (order - 1)] (plus a trailing axis of 2 when ncomp = 2) to [..., n_index]
    (plus the trailing axis)."""
    z = np.ascontiguousarray(zeta, dtype=np.float64)
    nlead = z.ndim - (order - 1) - (1 if ncomp == 2 else 0)
    nbins = z.shape[nlead]
    nouter = int(np.prod(z.shape[:nlead])) if nlead else 1
    n = len(sbg_unique_bins(nbins, order))
    out = np.zeros(z.shape[:nlead] + (n,) + ((2,) if ncomp == 2 else ()))
    s = lib().sbg_unique_gather(z.ctypes.data, nouter, nbins, order, ncomp, out.ctypes.data)
    if s != SBG_OK:
        raise SbgError(s, "sbg_unique_gather")
    return out


def sbg_zero_overlap(zeta, order, ncomp=1):
    """Zero, in place, the entries of a dense output (the layout of
    sbg_unique_gather: float64, C-contiguous, writable) whose bins coincide;
    returns the array."""
    if not (isinstance(zeta, np.ndarray) and zeta.dtype == np.float64 and zeta.flags.c_contiguous
            and zeta.flags.writeable):
        raise ValueError("sbg_zero_overlap needs a writable C-contiguous float64 array")
    nlead = zeta.ndim - (order - 1) - (1 if ncomp == 2 else 0)
    if nlead < 0 or len(set(zeta.shape[nlead:nlead + order - 1])) != 1 or (ncomp == 2 and zeta.shape[-1] != 2):
        raise ValueError("sbg_zero_overlap: trailing axes must be [nbins]^(order - 1) (then 2 when ncomp = 2)")
    nbins = zeta.shape[nlead]
    nouter = int(np.prod(zeta.shape[:nlead])) if nlead else 1
    s = lib().sbg_zero_overlap(zeta.ctypes.data, nouter, nbins, order, ncomp)
    if s != SBG_OK:
        raise SbgError(s, "sbg_zero_overlap")
    return zeta


def sbg_lambda_odd_count(lmax):
    n = ctypes.c_int()
    s = lib().sbg_lambda_odd_count(lmax, ctypes.byref(n))
    if s != SBG_OK:
        raise SbgError(s, "sbg_lambda_odd_count")
    return n.value


def sbg_lambda_odd_list(lmax):
    n = sbg_lambda_odd_count(lmax)
    out = np.zeros((max(n, 1), 3), dtype=np.int32)
    s = lib().sbg_lambda_odd_list(lmax, out.ctypes.data)
    if s != SBG_OK:
        raise SbgError(s, "sbg_lambda_odd_list")
    return out[:n]


def _field_ptr(field):
    """(pointer, dtype code, shape, on_device, keepalive)."""
    if hasattr(field, "data_ptr"):  # torch tensor
        import torch
        if not field.is_contiguous():
            raise ValueError("field must be contiguous")
        if field.dtype not in (torch.float32, torch.float64):
            raise ValueError("field dtype must be float32 or float64")
        dt = SBG_F64 if field.dtype == torch.float64 else SBG_F32
        return field.data_ptr(), dt, tuple(field.shape), field.is_cuda, field
    a = np.asarray(field)
    if a.dtype not in (np.float32, np.float64):
        raise ValueError("field dtype must be float32 or float64")
    a = np.ascontiguousarray(a)
    return a.ctypes.data, (SBG_F64 if a.dtype == np.float64 else SBG_F32), a.shape, False, a


def _edges(edges):
    return np.ascontiguousarray(np.asarray(edges, dtype=np.float64))


def _out(a, shape, name):
    """A result array: a new zeroed one, or the caller's (reused across calls),
    which must be a writable C-contiguous float64 array of exactly this shape
    (the library writes every element through its pointer)."""
    shape = tuple(int(x) for x in shape)
    if a is None:
        return np.zeros(shape)
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or a.shape != shape \
            or not a.flags.c_contiguous or not a.flags.writeable:
        raise ValueError(f"{name} must be a writable C-contiguous float64 array of shape {shape}")
    return a


def sbg_full(h, field, edges, lmax3, lmax4, prec, flags, zeta3=None, zeta4=None):
    ptr, dt, shape, on_dev, keep = _field_ptr(field)
    e = _edges(edges)
    nb = len(e) - 1
    if on_dev:
        flags |= SBG_FIELD_ON_DEVICE
    zeta3 = _out(zeta3, (lmax3 + 1, nb, nb), "zeta3") if flags & SBG_3PCF else None
    zeta4 = _out(zeta4, (sbg_lambda_count(lmax4), nb, nb, nb), "zeta4") if flags & SBG_4PCF else None
    shp = (ctypes.c_int64 * 3)(*shape) if len(shape) == 3 else (ctypes.c_int64 * 3)(*(list(shape) + [0, 0, 0])[:3])
    s = lib().sbg_full(h, ptr, dt, shp, e.ctypes.data, nb, int(lmax3 or 0), int(lmax4 or 0), prec, flags,
                       zeta3.ctypes.data if zeta3 is not None else None,
                       zeta4.ctypes.data if zeta4 is not None else None)
    del keep
    if s != SBG_OK:
        raise SbgError(s, sbg_last_error(h))
    return zeta3, zeta4


def sbg_full_odd(h, field, edges, lmax4, prec, flags, zeta4_odd=None):
    ptr, dt, shape, on_dev, keep = _field_ptr(field)
    e = _edges(edges)
    nb = len(e) - 1
    if on_dev:
        flags |= SBG_FIELD_ON_DEVICE
    zeta4_odd = _out(zeta4_odd, (sbg_lambda_odd_count(lmax4), nb, nb, nb), "zeta4_odd")
    shp = (ctypes.c_int64 * 3)(*shape) if len(shape) == 3 else (ctypes.c_int64 * 3)(*(list(shape) + [0, 0, 0])[:3])
    s = lib().sbg_full_odd(h, ptr, dt, shp, e.ctypes.data, nb, int(lmax4), prec, flags, zeta4_odd.ctypes.data)
    del keep
    if s != SBG_OK:
        raise SbgError(s, sbg_last_error(h))
    return zeta4_odd


def sbg_projected(h, field, edges, mmax, prec, flags, zeta3=None, zeta4=None):
    ptr, dt, shape, on_dev, keep = _field_ptr(field)
    e = _edges(edges)
    nb = len(e) - 1
    if on_dev:
        flags |= SBG_FIELD_ON_DEVICE
    w = 2 * mmax + 1
    zeta3 = _out(zeta3, (mmax + 1, nb, nb, 2), "zeta3") if flags & SBG_3PCF else None
    zeta4 = _out(zeta4, (w, w, nb, nb, nb, 2), "zeta4") if flags & SBG_4PCF else None
    shp = (ctypes.c_int64 * 2)(*(list(shape) + [0, 0])[:2])
    s = lib().sbg_projected(h, ptr, dt, shp, e.ctypes.data, nb, mmax, prec, flags,
                            zeta3.ctypes.data if zeta3 is not None else None,
                            zeta4.ctypes.data if zeta4 is not None else None)
    del keep
    if s != SBG_OK:
        raise SbgError(s, sbg_last_error(h))
    return zeta3, zeta4


def sbg_projected_batch(h, fields, edges_list, nbins, mmax, prec, flags, outs=None):
    """outs: None, or one (zeta3, zeta4) pair per field to write into."""
    n = len(fields)
    if outs is not None and len(outs) != n:
        raise ValueError("outs must hold one (zeta3, zeta4) pair per field")
    arr = (Field2D * n)()
    keep, res = [], []
    w = 2 * mmax + 1
    for i, (f, e) in enumerate(zip(fields, edges_list)):
        ptr, dt, shape, on_dev, k = _field_ptr(f)
        ee = _edges(e)
        o3, o4 = outs[i] if outs is not None else (None, None)
        z3 = _out(o3, (mmax + 1, nbins, nbins, 2), "zeta3") if flags & SBG_3PCF else None
        z4 = _out(o4, (w, w, nbins, nbins, nbins, 2), "zeta4") if flags & SBG_4PCF else None
        keep += [k, ee]
        res.append((z3, z4))
        arr[i].field = ptr
        arr[i].dtype = dt
        arr[i].shape[0], arr[i].shape[1] = shape[0], shape[1]
        arr[i].edges = ee.ctypes.data
        arr[i].zeta3 = z3.ctypes.data if z3 is not None else None
        arr[i].zeta4 = z4.ctypes.data if z4 is not None else None
        if on_dev:
            flags |= SBG_FIELD_ON_DEVICE
    s = lib().sbg_projected_batch(h, arr, n, nbins, mmax, prec, flags)
    del keep
    if s != SBG_OK:
        raise SbgError(s, sbg_last_error(h))
    return res


def sbg_last_timings(h):
    out = np.zeros(8)
    n = ctypes.c_int()
    lib().sbg_last_timings(h, out.ctypes.data, ctypes.byref(n))
    return out[: n.value]


def sbg_last_contraction_ms(h):
    out = ctypes.c_double()
    lib().sbg_last_contraction_ms(h, ctypes.byref(out))
    return out.value


def sbg_plan4_info(dim, nbins, lmax, prec, odd=0):
    """(ntiles, nrows, covering) of the 4PCF tile plan; host only."""
    nt, nr, cv = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    s = lib().sbg_plan4_info(dim, nbins, lmax, prec, odd, ctypes.byref(nt), ctypes.byref(nr), ctypes.byref(cv))
    if s != SBG_OK:
        raise SbgError(s, "sbg_plan4_info")
    return nt.value, nr.value, cv.value


def sbg_projected3_noalloc(field, edges, mmax, flags, zeta3, stream=0):
    """Projected 3PCF with no device allocation: `field` and `zeta3` are CUDA
    torch tensors ([n][n] float32/float64 and [mmax+1][nb][nb][2] float64);
    work is queued on `stream` (a cudaStream_t as int)."""
    ptr, dt, shape, on_dev, keep = _field_ptr(field)
    if not on_dev or not hasattr(zeta3, "data_ptr") or not zeta3.is_cuda:
        raise ValueError("field and zeta3 must be device tensors")
    e = _edges(edges)
    s = lib().sbg_projected3_noalloc(ptr, dt, shape[0], e.ctypes.data, len(e) - 1, mmax, flags,
                                     zeta3.data_ptr(), ctypes.c_void_p(stream))
    del keep
    if s != SBG_OK:
        raise SbgError(s, "sbg_projected3_noalloc")
    return zeta3


class Context:
    """Owns one sbg_context (one per host thread)."""

    def __init__(self, device=0, budget=0):
        self.h = sbg_create(device, budget)

    def close(self):
        if self.h:
            sbg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        return sbg_set_stream(self.h, stream)

    def set_wait_limit(self, wait_ns, test_stall=0):
        s = sbg_set_wait_limit(self.h, wait_ns, test_stall)
        if s != SBG_OK:
            raise SbgError(s, sbg_last_error(self.h))

    # out: arrays from an earlier call of the same shapes, written again in
    # place (no allocation or first-touch page faults per call)
    def full(self, field, edges, lmax3=None, lmax4=None, prec=SBG_PREC_FP32, flags=SBG_SUBTRACT_MEAN, out=None):
        if lmax3 is not None:
            flags |= SBG_3PCF
        if lmax4 is not None:
            flags |= SBG_4PCF
        z3, z4 = out if out is not None else (None, None)
        return sbg_full(self.h, field, edges, lmax3, lmax4, prec, flags, z3, z4)

    def full_odd(self, field, edges, lmax4, prec=SBG_PREC_FP32, flags=SBG_SUBTRACT_MEAN):
        return sbg_full_odd(self.h, field, edges, lmax4, prec, flags)

    def projected(self, field, edges, mmax, npcf=(3, 4), prec=SBG_PREC_FP32, flags=SBG_SUBTRACT_MEAN, out=None):
        if 3 in npcf:
            flags |= SBG_3PCF
        if 4 in npcf:
            flags |= SBG_4PCF
        z3, z4 = out if out is not None else (None, None)
        return sbg_projected(self.h, field, edges, mmax, prec, flags, z3, z4)

    def projected_batch(self, fields, edges_list, nbins, mmax, npcf=(3, 4), prec=SBG_PREC_FP32,
                        flags=SBG_SUBTRACT_MEAN, out=None):
        if 3 in npcf:
            flags |= SBG_3PCF
        if 4 in npcf:
            flags |= SBG_4PCF
        return sbg_projected_batch(self.h, fields, edges_list, nbins, mmax, prec, flags, out)

    def projected_slices(self, cube, edges, mmax, npcf=(3, 4), prec=SBG_PREC_FP32, flags=SBG_SUBTRACT_MEAN,
                         out=None):
        if 3 in npcf:
            flags |= SBG_3PCF
        if 4 in npcf:
            flags |= SBG_4PCF
        z3, z4 = out if out is not None else (None, None)
        return sbg_projected_slices(self.h, cube, edges, mmax, prec, flags, z3, z4)

    def timings(self):
        return sbg_last_timings(self.h)
