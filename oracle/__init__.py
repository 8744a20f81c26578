"""CPU Delaunay oracle — TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  It shares no code with the CUDA path.

Functions (each cites the paper's passage in dt_oracle.c):

- ``delaunay(xy, seed=...)``: canonical sorted (T, 3) int32 triangle list of the
  unique (SoS) Delaunay triangulation, by Bowyer-Watson from scratch
  (Section I definition, Section IV Bowyer-Watson, Fig. 4 output per step).
- ``check_dt(xy, tris)``: 0 if ``tris`` is that triangulation, else the number of
  the failed property (see dt_oracle.c).
- ``orient2d``, ``incircle_raw``, ``incircle_sos``: the exact predicates.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

ORC_ERRORS = {
    -1: "bad argument", -2: "coordinate out of range", -3: "duplicate points",
    -4: "degenerate (n < 3 or all collinear)", -5: "capacity", -6: "out of memory",
    -7: "internal error",
}


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__("oracle error %d (%s)" % (code, ORC_ERRORS.get(code, "?")))
        self.code = code


def _bind(L):
    p32 = ctypes.POINTER(ctypes.c_int32)
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    L.oracle_orient2d.argtypes = [p32, i32, i32, i32]
    L.oracle_orient2d.restype = ctypes.c_int
    L.oracle_incircle_raw.argtypes = [p32, i32, i32, i32, i32]
    L.oracle_incircle_raw.restype = ctypes.c_int
    L.oracle_incircle_sos.argtypes = [p32, i32, i32, i32, i32]
    L.oracle_incircle_sos.restype = ctypes.c_int
    L.oracle_delaunay.argtypes = [p32, i64, ctypes.c_uint64, p32, i64,
                                  ctypes.POINTER(i64)]
    L.oracle_delaunay.restype = ctypes.c_int
    L.oracle_check_dt.argtypes = [p32, i64, p32, i64, ctypes.POINTER(i64)]
    L.oracle_check_dt.restype = ctypes.c_int
    L.oracle_version.restype = ctypes.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(_build.build()))
    return _lib


class Oracle:
    """The oracle's functions bound to one shared library (the built one by default).

    Tests use other instances to load deliberately broken copies of the oracle and
    show that the pins catch them."""

    def __init__(self, path=None):
        self.L = lib() if path is None else _bind(ctypes.CDLL(path))

    def orient2d(self, xy, a, b, c):
        xy = _pts(xy)
        return self.L.oracle_orient2d(_ptr(xy), a, b, c)

    def incircle_raw(self, xy, a, b, c, d):
        xy = _pts(xy)
        return self.L.oracle_incircle_raw(_ptr(xy), a, b, c, d)

    def incircle_sos(self, xy, a, b, c, d):
        xy = _pts(xy)
        return self.L.oracle_incircle_sos(_ptr(xy), a, b, c, d)

    def delaunay(self, xy, seed=0x2308_06484):
        xy = _pts(xy)
        n = xy.shape[0]
        cap = max(2 * n, 1)
        out = np.empty((cap, 3), dtype=np.int32)
        nt = ctypes.c_int64(0)
        rc = self.L.oracle_delaunay(_ptr(xy), n, ctypes.c_uint64(seed & (2**64 - 1)),
                                    _ptr(out), cap, ctypes.byref(nt))
        if rc != 0:
            raise OracleError(rc)
        return out[: nt.value].copy()

    def check_dt(self, xy, tris):
        xy = _pts(xy)
        t = np.ascontiguousarray(np.asarray(tris, dtype=np.int32).reshape(-1, 3))
        detail = ctypes.c_int64(-1)
        return self.L.oracle_check_dt(_ptr(xy), xy.shape[0], _ptr(t), t.shape[0],
                                      ctypes.byref(detail))


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _pts(xy):
    a = np.ascontiguousarray(np.asarray(xy, dtype=np.int32).reshape(-1, 2))
    return a


_default = None


def _d():
    global _default
    if _default is None:
        _default = Oracle()
    return _default


def orient2d(xy, a, b, c):
    return _d().orient2d(xy, a, b, c)


def incircle_raw(xy, a, b, c, d):
    return _d().incircle_raw(xy, a, b, c, d)


def incircle_sos(xy, a, b, c, d):
    return _d().incircle_sos(xy, a, b, c, d)


def delaunay(xy, seed=0x2308_06484):
    """Canonical sorted triangle list (T, 3) of the SoS Delaunay triangulation."""
    return _d().delaunay(xy, seed)


def check_dt(xy, tris):
    """0 if ``tris`` is the SoS Delaunay triangulation of ``xy``, else the failed property."""
    return _d().check_dt(xy, tris)
