"""ctypes shim of the FP64 C++ oracle (oracle/sarabande_oracle.cpp).

TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the
CPU-baseline legs of bench.py, never by the product library.  build() compiles
the oracle with the host C++ compiler (g++ -O2, OpenMP when available) into
oracle/_build/; the functions below mirror oracle/sarabande_oracle.py and take
float64 numpy arrays.
"""
import ctypes
import hashlib
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sarabande_oracle.cpp")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle_cpp.so")
_lib = None


def build(force=False):
    """Compile the C++ oracle (rebuilt when its source changes)."""
    os.makedirs(BUILD, exist_ok=True)
    dig = hashlib.sha256(open(SRC, "rb").read() + open(__file__, "rb").read() + os.uname().machine.encode()).hexdigest()
    stamp = os.path.join(BUILD, "stamp")
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    cxx = os.environ.get("CXX", "g++")
    # -fcx-limited-range: complex products by the textbook formula (no NaN/Inf
    # recovery calls), the same values for finite operands
    base = [cxx, "-O2", "-fcx-limited-range", "-std=c++17", "-shared", "-fPIC", SRC, "-o", LIB + ".tmp"]
    r = subprocess.run(base[:2] + ["-fopenmp"] + base[2:], stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:  # no OpenMP: serial build
        r = subprocess.run(base, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError("C++ oracle build failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(LIB + ".tmp", LIB)
    with open(stamp, "w") as fh:
        fh.write(dig)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        vp, i, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        L.oc_fftn.argtypes = [vp, i, vp, i]
        L.oc_coefficient.argtypes = [vp, i, i64, vp, i, i, i, i, vp]
        L.oc_zeta3_full.argtypes = [vp, i64, vp, i, i, vp]
        L.oc_zeta3_projected.argtypes = [vp, i64, vp, i, i, vp]
        L.oc_zeta4_full.argtypes = [vp, i64, vp, i, i, i, vp]
        L.oc_zeta4_combine.argtypes = [vp, vp, i64, i, i, i, vp]
        L.oc_zeta4_projected.argtypes = [vp, i64, vp, i, i, vp]
        L.oc_lambda_list.argtypes = [i, i, vp]
        L.oc_wigner3j.argtypes = [i, i, i, i, i, i]
        L.oc_wigner3j.restype = d
        L.oc_threads.argtypes = []
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _edges(edges):
    return _f64(np.asarray(edges, dtype=np.float64))


def _check(rc, name):
    if rc != 0:
        raise ValueError(f"{name}: invalid arguments")


def threads():
    return lib().oc_threads()


def fftn(x, sign):
    """Unnormalised DFT with exp(sign 2 pi i j.k / N) over every axis."""
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    dims = np.array(a.shape, dtype=np.int64)
    _check(lib().oc_fftn(a.ctypes.data, a.ndim, dims.ctypes.data, int(sign)), "fftn")
    return a


def coefficient(delta, edges, l, m, b):
    """a^b_lm (3D) or c^b_m (2D; l ignored) of a real field."""
    d = _f64(delta)
    e = _edges(edges)
    out = np.empty(d.shape, dtype=np.complex128)
    _check(lib().oc_coefficient(d.ctypes.data, d.ndim, d.shape[0], e.ctypes.data, len(e) - 1, l, m, b,
                                out.ctypes.data), "coefficient")
    return out


def zeta3_full(delta, edges, lmax):
    d, e = _f64(delta), _edges(edges)
    nb = len(e) - 1
    out = np.empty((lmax + 1, nb, nb))
    _check(lib().oc_zeta3_full(d.ctypes.data, d.shape[0], e.ctypes.data, nb, lmax, out.ctypes.data), "zeta3_full")
    return out


def zeta3_projected(delta, edges, mmax):
    d, e = _f64(delta), _edges(edges)
    nb = len(e) - 1
    out = np.empty((mmax + 1, nb, nb, 2))
    _check(lib().oc_zeta3_projected(d.ctypes.data, d.shape[0], e.ctypes.data, nb, mmax, out.ctypes.data),
           "zeta3_projected")
    return out[..., 0] + 1j * out[..., 1]


def lambda_list(lmax, odd=False):
    n = lib().oc_lambda_list(lmax, int(odd), None)
    out = np.empty(3 * n, dtype=np.int32)
    lib().oc_lambda_list(lmax, int(odd), out.ctypes.data)
    return [tuple(int(v) for v in out[3 * k:3 * k + 3]) for k in range(n)]


def wigner3j(j1, j2, j3, m1, m2, m3):
    return lib().oc_wigner3j(j1, j2, j3, m1, m2, m3)


def zeta4_full(delta, edges, lmax, odd=False):
    """Even (odd=False, real part) or odd (odd=True, imaginary part) full 4PCF."""
    d, e = _f64(delta), _edges(edges)
    nb = len(e) - 1
    nl = lib().oc_lambda_list(lmax, int(odd), None)
    out = np.empty((nl, nb, nb, nb))
    _check(lib().oc_zeta4_full(d.ctypes.data, d.shape[0], e.ctypes.data, nb, lmax, int(odd), out.ctypes.data),
           "zeta4_full")
    return out


def zeta4_combine(delta_pts, a, lmax, odd=False):
    """The combination step of the full 4PCF over the points of delta_pts [npts]
    from coefficient arrays a [(lmax+1)^2][nb][npts] complex ((l, m) at
    l*l + l + m)."""
    d = _f64(np.ravel(delta_pts))
    a = np.ascontiguousarray(a, dtype=np.complex128)
    nb = a.shape[1]
    nl = lib().oc_lambda_list(lmax, int(odd), None)
    out = np.empty((nl, nb, nb, nb))
    _check(lib().oc_zeta4_combine(d.ctypes.data, a.ctypes.data, len(d), nb, lmax, int(odd), out.ctypes.data),
           "zeta4_combine")
    return out


def zeta4_projected(delta, edges, mmax):
    d, e = _f64(delta), _edges(edges)
    nb = len(e) - 1
    w = 2 * mmax + 1
    out = np.empty((w, w, nb, nb, nb, 2))
    _check(lib().oc_zeta4_projected(d.ctypes.data, d.shape[0], e.ctypes.data, nb, mmax, out.ctypes.data),
           "zeta4_projected")
    return out[..., 0] + 1j * out[..., 1]
