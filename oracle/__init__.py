"""ctypes front end of the CPU oracle (``prgb_oracle.c``).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it; the CUDA library never does.  The
oracle is a plain single-threaded C99 file compiled with gcc; it shares no
code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prgb_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")

NORM_L1 = 0
NORM_LINF = 1
TYPE_CAC = 0
TYPE_SCC = 1

_lib = None


class OracleError(RuntimeError):
    pass


def build(force=False):
    """Compile the oracle shared library with gcc (-O2, no -march)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        lib.oracle_partition.argtypes = [C.c_int32, i32p, i32p, C.c_int, i32p, u8p, i32p,
                                         C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        lib.oracle_partition.restype = C.c_int
        lib.oracle_solve_cw.argtypes = [C.c_int32, i32p, i32p, i32p, u8p, i32p, C.c_int32,
                                        C.c_double, f64p, C.c_double, C.c_int, C.c_int32,
                                        C.c_int32, C.c_void_p, f64p, i32p]
        lib.oracle_solve_cw.restype = C.c_int
        lib.oracle_solve_global.argtypes = [C.c_int32, i32p, i32p, C.c_double, f64p, C.c_double,
                                            C.c_int, C.c_int32, C.c_int32, f64p,
                                            C.POINTER(C.c_int32)]
        lib.oracle_solve_global.restype = C.c_int
        lib.oracle_residual_l1.argtypes = [C.c_int32, i32p, i32p, C.c_double, f64p, f64p]
        lib.oracle_residual_l1.restype = C.c_double
        lib.oracle_dense_solve.argtypes = [C.c_int32, i32p, i32p, C.c_double, f64p, f64p]
        lib.oracle_dense_solve.restype = C.c_int
        _lib = lib
    return _lib


def _csr(rowptr, col):
    return (np.ascontiguousarray(rowptr, dtype=np.int32),
            np.ascontiguousarray(col, dtype=np.int32))


class Partition:
    """Canonical partition: comp ids, types (0 CAC / 1 SCC), 0-based levels."""

    def __init__(self, comp, type_, level, n_comp, n_levels):
        self.comp = comp
        self.type = type_
        self.level = level
        self.n_comp = n_comp
        self.n_levels = n_levels

    def sizes(self):
        return np.bincount(self.comp, minlength=self.n_comp)


def partition(rowptr, col, merge=True):
    """Sec. 4.1 modified Tarjan DFS; merge=False gives the plain SCC split."""
    lib = _load()
    rowptr, col = _csr(rowptr, col)
    n = rowptr.shape[0] - 1
    comp = np.empty(max(n, 1), np.int32)
    typ = np.empty(max(n, 1), np.uint8)
    lev = np.empty(max(n, 1), np.int32)
    nc, nl = C.c_int32(0), C.c_int32(0)
    rc = lib.oracle_partition(n, rowptr, col, int(merge), comp, typ, lev, C.byref(nc), C.byref(nl))
    if rc:
        raise OracleError(f"oracle_partition failed: {rc}")
    return Partition(comp[:n], typ[:n], lev[:n], nc.value, nl.value)


def solve_cw(rowptr, col, part, c, u, tol, norm=NORM_L1, max_iter=10_000,
             lu_threshold=0, replay_iters=None):
    """Sec. 4.3 componentwise solve; returns (R, per-component iterations)."""
    lib = _load()
    rowptr, col = _csr(rowptr, col)
    n = rowptr.shape[0] - 1
    u = np.ascontiguousarray(u, dtype=np.float64)
    R = np.empty(max(n, 1), np.float64)
    its = np.zeros(max(part.n_comp, 1), np.int32)
    rep = None
    if replay_iters is not None:
        rep_arr = np.ascontiguousarray(replay_iters, dtype=np.int32)
        rep = rep_arr.ctypes.data_as(C.c_void_p)
    rc = lib.oracle_solve_cw(n, rowptr, col, part.comp if n else np.zeros(1, np.int32),
                             part.type if n else np.zeros(1, np.uint8),
                             part.level if n else np.zeros(1, np.int32), part.n_comp,
                             float(c), u if n else np.zeros(1), float(tol), int(norm),
                             int(max_iter), int(lu_threshold), rep, R, its)
    if rc == 4:
        raise OracleError("oracle_solve_cw: max_iter reached")
    if rc:
        raise OracleError(f"oracle_solve_cw failed: {rc}")
    return R[:n], its[: part.n_comp]


def solve_global(rowptr, col, c, u, tol, norm=NORM_L1, max_iter=10_000, replay_iters=-1):
    """Baseline power series on the whole graph; returns (R, iterations)."""
    lib = _load()
    rowptr, col = _csr(rowptr, col)
    n = rowptr.shape[0] - 1
    u = np.ascontiguousarray(u, dtype=np.float64)
    R = np.empty(max(n, 1), np.float64)
    it = C.c_int32(0)
    rc = lib.oracle_solve_global(n, rowptr, col, float(c), u if n else np.zeros(1), float(tol),
                                 int(norm), int(max_iter), int(replay_iters), R, C.byref(it))
    if rc == 4:
        raise OracleError("oracle_solve_global: max_iter reached")
    if rc:
        raise OracleError(f"oracle_solve_global failed: {rc}")
    return R[:n], it.value


def residual_l1(rowptr, col, c, u, R):
    lib = _load()
    rowptr, col = _csr(rowptr, col)
    n = rowptr.shape[0] - 1
    return lib.oracle_residual_l1(n, rowptr, col, float(c),
                                  np.ascontiguousarray(u, dtype=np.float64),
                                  np.ascontiguousarray(R, dtype=np.float64))


def dense_solve(rowptr, col, c, u):
    lib = _load()
    rowptr, col = _csr(rowptr, col)
    n = rowptr.shape[0] - 1
    R = np.empty(max(n, 1), np.float64)
    rc = lib.oracle_dense_solve(n, rowptr, col, float(c),
                                np.ascontiguousarray(u, dtype=np.float64), R)
    if rc:
        raise OracleError(f"oracle_dense_solve failed: {rc}")
    return R[:n]


class use_library:
    """Context manager that points this module at another build of the
    oracle (used by the tests that plant mistakes in a copy of it)."""

    def __init__(self, path):
        self.path = path
        self.saved = None

    def __enter__(self):
        global _lib
        self.saved = _load()
        _lib = None
        real_build = globals()["build"]
        globals()["build"] = lambda force=False: self.path
        try:
            _load()
        finally:
            globals()["build"] = real_build
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False
