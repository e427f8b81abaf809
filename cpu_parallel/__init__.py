"""ctypes front end of the multi-core CPU baseline (``prgb_cpu_parallel.c``):
the componentwise PageRank step (Sec. 4.3) and the global power series
(Sec. 4.3.2) parallelised with OpenMP over the host's cores, for timing next
to the GPU path.

It takes a partition (component id, type and level per vertex, canonical
ids) as input and shares no code with the GPU path or the oracle.  The
library is compiled on first use with the system's gcc (``-O3 -fopenmp``);
``available()`` says whether that worked.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prgb_cpu_parallel.c")
_LIB = os.path.join(_HERE, "_libcpupar.so")
_lib = None
_err = None


class CpuParallelError(RuntimeError):
    pass


def build():
    """Compile the library if it is missing or older than its source."""
    if os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O3", "-std=c99", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"],
                   check=True, capture_output=True)
    os.replace(tmp, _LIB)


def _load():
    global _lib, _err
    if _lib is not None:
        return _lib
    try:
        build()
        lib = C.CDLL(_LIB)
    except (OSError, subprocess.CalledProcessError) as e:
        _err = str(e)
        raise CpuParallelError(f"CPU baseline library unavailable: {e}") from e
    p32, pd, vp = C.POINTER(C.c_int32), C.POINTER(C.c_double), C.c_void_p
    lib.cpb_plan_create.restype = C.c_int
    lib.cpb_plan_create.argtypes = [C.c_int32, p32, p32, p32, C.POINTER(C.c_uint8), p32, C.c_int32,
                                    C.POINTER(vp)]
    lib.cpb_plan_destroy.restype = None
    lib.cpb_plan_destroy.argtypes = [vp]
    lib.cpb_solve_cw.restype = C.c_int
    lib.cpb_solve_cw.argtypes = [vp, C.c_double, pd, C.c_double, C.c_int32, C.c_int32, C.c_int32, pd, p32]
    lib.cpb_solve_global.restype = C.c_int
    lib.cpb_solve_global.argtypes = [vp, C.c_double, pd, C.c_double, C.c_int32, C.c_int32, pd, p32]
    lib.cpb_max_threads.restype = C.c_int
    lib.cpb_max_threads.argtypes = []
    _lib = lib
    return lib


def available() -> bool:
    try:
        _load()
        return True
    except CpuParallelError:
        return False


def max_threads() -> int:
    return int(_load().cpb_max_threads())


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


class Plan:
    """The layout of one partitioned graph (built once, untimed)."""

    def __init__(self, rowptr, col, comp, ctype, level):
        lib = _load()
        self.n = int(len(rowptr) - 1)
        self._keep = [np.ascontiguousarray(rowptr, np.int32), np.ascontiguousarray(col, np.int32),
                      np.ascontiguousarray(comp, np.int32), np.ascontiguousarray(ctype, np.uint8),
                      np.ascontiguousarray(level, np.int32)]
        rp, cl, cm, ty, lv = self._keep
        n_comp = int(cm.max()) + 1 if self.n else 0
        h = C.c_void_p()
        rc = lib.cpb_plan_create(self.n, _p(rp, C.c_int32), _p(cl, C.c_int32), _p(cm, C.c_int32),
                                 _p(ty, C.c_uint8), _p(lv, C.c_int32), n_comp, C.byref(h))
        if rc:
            raise CpuParallelError(f"cpb_plan_create failed ({rc})")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.cpb_plan_destroy(self._h)
            self._h = None

    def solve_cw(self, c, u, tol, threads=0, big=16384, max_iter=10_000):
        """Componentwise step; returns (R, largest SCC sweep count)."""
        u = np.ascontiguousarray(u, np.float64)
        R = np.empty(self.n, np.float64)
        it = C.c_int32()
        rc = _lib.cpb_solve_cw(self._h, float(c), _p(u, C.c_double), float(tol), int(max_iter), int(threads),
                               int(big), _p(R, C.c_double), C.byref(it))
        if rc:
            raise CpuParallelError(f"cpb_solve_cw failed ({rc})")
        return R, it.value

    def solve_global(self, c, u, tol, threads=0, max_iter=10_000):
        """Global power series; returns (R, sweeps)."""
        u = np.ascontiguousarray(u, np.float64)
        R = np.empty(self.n, np.float64)
        it = C.c_int32()
        rc = _lib.cpb_solve_global(self._h, float(c), _p(u, C.c_double), float(tol), int(max_iter), int(threads),
                                   _p(R, C.c_double), C.byref(it))
        if rc:
            raise CpuParallelError(f"cpb_solve_global failed ({rc})")
        return R, it.value
