"""ctypes wrapper of the C oracle (test infrastructure only).

The oracle computes T = n * D_n(z), Eq. (1), by the subset loop of Algorithm 1
with Algorithm 2 as the inner bivariate count, in exact integer arithmetic.
The readings of the paper it takes are listed at the top of tukey_oracle.c.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tukey_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


class OracleError(RuntimeError):
    pass


_ERRORS = {-1: "invalid argument", -2: "coordinates exceed the exact-arithmetic bound", -3: "out of memory",
           -4: "internal inconsistency"}


def build(force=False):
    """Compile tukey_oracle.c into liboracle.so next to it (gcc, no GPU)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            lib.oracle_depth.argtypes = [i32p, ctypes.c_int64, ctypes.c_int, i32p, i64p]
            lib.oracle_depth.restype = ctypes.c_int
            lib.oracle_depth_range.argtypes = [i32p, ctypes.c_int64, ctypes.c_int, i32p,
                                               ctypes.c_int64, ctypes.c_int64, i64p, i64p, u64p]
            lib.oracle_depth_range.restype = ctypes.c_int
            lib.oracle_bivariate_closed.argtypes = [i64p, ctypes.c_int64, i64p]
            lib.oracle_bivariate_closed.restype = ctypes.c_int
            lib.oracle_rank.argtypes = [i32p, ctypes.c_int64, ctypes.c_int, i32p, i32p]
            lib.oracle_rank.restype = ctypes.c_int
            lib.oracle_adia.argtypes = [i32p, ctypes.c_int64, ctypes.c_int, i32p, i64p, i64p]
            lib.oracle_adia.restype = ctypes.c_int
            lib.oracle_critical.argtypes = [i64p, ctypes.c_int64, i64p, ctypes.POINTER(ctypes.c_uint8)]
            lib.oracle_subset_min.argtypes = [i32p, ctypes.c_int64, ctypes.c_int, i32p, i32p, ctypes.c_int64,
                                              i64p, i64p]
            lib.oracle_subset_min.restype = ctypes.c_int
            lib.oracle_critical.restype = ctypes.c_int
            _lib = lib
    return _lib


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _check(rc):
    if rc != 0:
        raise OracleError(_ERRORS.get(rc, "error %d" % rc))


def depth(X, z):
    """Closed halfspace depth count T = n * D_n(z) of z w.r.t. the rows of X."""
    lib = _load()
    X, Xp = _i32(X)
    z, zp = _i32(z)
    n, p = X.shape
    assert z.shape == (p,)
    out = ctypes.c_int64(0)
    _check(lib.oracle_depth(Xp, n, p, zp, ctypes.byref(out)))
    return int(out.value)


def depth_many(X, Z):
    """depth(X, z) for every row z of Z, as an int64 array."""
    Z = np.asarray(Z)
    return np.array([depth(X, z) for z in Z], dtype=np.int64)


def depth_range(X, z, lo, hi):
    """Partial count over the top-level subsets at lexicographic positions [lo, hi).

    Returns (partial, positions, counters): partial = Z + min over the range
    (None if the range holds no independent subset), positions = number of
    top-level positions, counters = (visited, dependent, tight_extra).
    """
    lib = _load()
    X, Xp = _i32(X)
    z, zp = _i32(z)
    n, p = X.shape
    part = ctypes.c_int64(0)
    npos = ctypes.c_int64(0)
    ctr = (ctypes.c_uint64 * 3)()
    _check(lib.oracle_depth_range(Xp, n, p, zp, int(lo), int(hi), ctypes.byref(part),
                                  ctypes.byref(npos), ctr))
    v = int(part.value)
    return (None if v == np.iinfo(np.int64).max else v), int(npos.value), tuple(int(c) for c in ctr)


def subset_min(X, z, subsets):
    """Z + min V(S) over the listed subsets (rows of p-2 increasing indices
    into the nonzero centred points in data order; the points must span R^p).
    Returns (value or None when no listed subset is independent, dependent)."""
    lib = _load()
    X, Xp = _i32(X)
    z, zp = _i32(z)
    n, p = X.shape
    S = np.ascontiguousarray(np.asarray(subsets, dtype=np.int32).reshape(-1, p - 2))
    out = ctypes.c_int64(0)
    dep = ctypes.c_int64(0)
    _check(lib.oracle_subset_min(Xp, n, p, zp, S.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), S.shape[0],
                                 ctypes.byref(out), ctypes.byref(dep)))
    v = int(out.value)
    return (None if v == np.iinfo(np.int64).max else v), int(dep.value)


def bivariate_closed(Y):
    """Algorithm 2 alone: closed depth count of the origin for 2-D integer points."""
    lib = _load()
    Y = np.ascontiguousarray(Y, dtype=np.int64).reshape(-1, 2)
    out = ctypes.c_int64(0)
    _check(lib.oracle_bivariate_closed(Y.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                       Y.shape[0], ctypes.byref(out)))
    return int(out.value)


def rank(X, z):
    """(rank, pivot columns) of the centred points X - z."""
    lib = _load()
    X, Xp = _i32(X)
    z, zp = _i32(z)
    n, p = X.shape
    piv = (ctypes.c_int32 * 6)()
    r = lib.oracle_rank(Xp, n, p, zp, piv)
    if r < 0:
        _check(r)
    return r, [int(piv[i]) for i in range(r)]


ADIA_STATS = ("pops", "step4_subsets", "nodes", "max_stack", "union_points", "step5_subsets",
              "d0_after_search", "algorithm1", "union_hash")


def adia(X, z):
    """Algorithm 3 (ADIA): (count, stats).  The count is never below depth(X, z)."""
    lib = _load()
    X, Xp = _i32(X)
    z, zp = _i32(z)
    n, p = X.shape
    out = ctypes.c_int64(0)
    st = (ctypes.c_int64 * 9)()
    _check(lib.oracle_adia(Xp, n, p, zp, ctypes.byref(out), st))
    return int(out.value), dict(zip(ADIA_STATS, (int(v) for v in st)))


def critical(Y):
    """(G, crit): Algorithm 2's minimum over generic directions for the 2-D
    points Y and the 0/1 flags of the critical points (lines bounding a cell
    whose count is G)."""
    lib = _load()
    Y = np.ascontiguousarray(Y, dtype=np.int64).reshape(-1, 2)
    G = ctypes.c_int64(0)
    crit = np.zeros(Y.shape[0], dtype=np.uint8)
    _check(lib.oracle_critical(Y.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), Y.shape[0],
                               ctypes.byref(G), crit.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))
    return int(G.value), crit

