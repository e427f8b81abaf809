"""Componentwise PageRank on GB300: thin Python binding of ``libprgb.so``.

The C library (``include/prgb.h``) does all the work in CUDA kernels; this
module only marshals arguments with ctypes.  PyTorch provides device memory
and the current stream.  There is no CPU fallback: if the library is missing
or cannot be loaded, every call raises.

Pipeline (Sec. 4 of arXiv 1609.09068):

    g = graph(rowptr, col)          # validated, loop-free graph + CSC
    p = partition(g)                # SCC/CAC partition with levels + layout
    R = solve(p, 0.85, u, 1e-10)    # level-by-level PageRank step
    Rg, k = global_power(g, 0.85, u, 1e-10)   # the baseline power series
    r = residual_l1(g, 0.85, u, R)  # || u + c A^T (R/outdeg) - R ||_1
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

__all__ = [
    "PrError", "Graph", "Partition", "graph", "partition", "solve", "global_power",
    "residual_l1", "load_library", "library_path", "launch_count", "TYPE_CAC", "TYPE_SCC",
    "NORM_L1", "NORM_LINF", "PREC_FP64", "PREC_MIXED", "Mpnn", "set_wait_limit", "CANONICALIZE",
    "PARTITION_TIMING", "load_partition",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libprgb.so")

TYPE_CAC = 0
TYPE_SCC = 1
NORM_L1 = 0
NORM_LINF = 1
PREC_FP64 = 0
PREC_MIXED = 1

_STATUS = {0: "PR_OK", 1: "PR_EINVAL", 2: "PR_ENOMEM", 3: "PR_ECUDA", 4: "PR_ENOCONV",
           5: "PR_ETIMEOUT", 6: "PR_EINTERNAL"}


class PrError(RuntimeError):
    """A non-OK pr_status; for PR_ECUDA, cuda_error is the cudaError_t the
    library recorded (pr_last_cuda_error)."""

    def __init__(self, code, where, cuda_error=0):
        self.code = code
        self.name = _STATUS.get(code, str(code))
        self.cuda_error = cuda_error
        extra = f" (cudaError {cuda_error})" if cuda_error else ""
        super().__init__(f"{where}: {self.name}{extra}")


class _Csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("on_host", C.c_int32)]


class _Opts(C.Structure):
    _fields_ = [("norm", C.c_int32), ("max_iter", C.c_int32), ("precision", C.c_int32),
                ("io_on_host", C.c_int32), ("replay_iters", C.c_void_p), ("warm_start", C.c_void_p),
                ("lu_threshold", C.c_int32)]


class _Stats(C.Structure):
    _fields_ = [("iters_max", C.c_int32), ("n_levels", C.c_int32), ("edge_visits", C.c_int64),
                ("launches", C.c_int64), ("comp_iters", C.c_void_p), ("timing", C.c_int32),
                ("kernel_ms", C.c_float), ("kernel_bytes", C.c_int64), ("kernel_launches", C.c_int64),
                ("fp64_sweeps_max", C.c_int32), ("fp64_edge_visits", C.c_int64), ("level_ms", C.c_void_p),
                ("counts_off", C.c_int32)]


class _PartTiming(C.Structure):
    _fields_ = [("trim_ms", C.c_float), ("giant_ms", C.c_float), ("colour_ms", C.c_float),
                ("levels_ms", C.c_float), ("layout_ms", C.c_float), ("total_ms", C.c_float),
                ("colour_rounds", C.c_int32), ("waves", (C.c_int32 * 2) * 5)]


_lib = None

# name -> (restype, argtypes), mirroring include/prgb.h
_SIGS = {
    "pr_graph_create": (C.c_int, [C.POINTER(_Csr), C.c_void_p, C.POINTER(C.c_void_p)]),
    "pr_graph_create_ex": (C.c_int, [C.POINTER(_Csr), C.c_uint32, C.c_void_p, C.POINTER(C.c_void_p)]),
    "pr_graph_destroy": (None, [C.c_void_p]),
    "pr_partition_create": (C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p, C.POINTER(C.c_void_p)]),
    "pr_partition_query": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_void_p]),
    "pr_partition_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "pr_partition_destroy": (None, [C.c_void_p]),
    "pr_partition_timing_get": (C.c_int, [C.c_void_p, C.POINTER(_PartTiming)]),
    "pr_partition_save": (C.c_int, [C.c_void_p, C.c_char_p, C.c_void_p]),
    "pr_partition_load": (C.c_int, [C.c_void_p, C.c_char_p, C.c_uint32, C.c_void_p, C.POINTER(C.c_void_p)]),
    "pr_solve": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_double, C.POINTER(_Opts),
                           C.c_void_p, C.POINTER(_Stats), C.c_void_p]),
    "pr_global_power": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_double, C.POINTER(_Opts),
                                  C.c_void_p, C.POINTER(_Stats), C.c_void_p]),
    "pr_residual_l1": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
                                 C.POINTER(C.c_double), C.c_void_p]),
    "pr_status_str": (C.c_char_p, [C.c_int]),
    "pr_last_cuda_error": (C.c_int, []),
    "pr_launch_count": (C.c_int64, []),
    "pr_set_wait_limit": (C.c_int, [C.c_uint32]),
    "pr_last_device_error": (C.c_int, []),
    "pr_residual_l1_static": (C.c_int, [C.POINTER(_Csr), C.c_double, C.c_void_p, C.c_void_p,
                                        C.POINTER(C.c_double), C.c_void_p]),
    "pr_partition_tune": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_double, C.c_void_p,
                                    C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_float)]),
    "pr_partition_set_shape": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32]),
    "pr_mpnn_param_count": (C.c_int64, []),
    "pr_mpnn_create": (C.c_int, [C.c_uint64, C.c_void_p, C.POINTER(C.c_void_p)]),
    "pr_mpnn_destroy": (None, [C.c_void_p]),
    "pr_mpnn_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "pr_mpnn_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "pr_mpnn_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "pr_mpnn_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "pr_mpnn_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
                                     C.c_float, C.POINTER(C.c_double), C.c_void_p]),
}

STATIC_MAX_N = 1 << 20


def library_path():
    return _LIB_PATH


def load_library():
    """Load libprgb.so (built by ``_build.build()``); raises if it is absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing: run __graft_entry__.build() first")
        lib = C.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc, where):
    if rc != 0:
        raise PrError(rc, where, int(_lib.pr_last_cuda_error()) if rc == 3 and _lib is not None else 0)


def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _length(x):
    """Number of elements of a 1-D tensor, array or sequence (no copy to the
    device); raises ValueError for anything that is not one-dimensional."""
    shape = tuple(x.shape) if hasattr(x, "shape") else (len(x),)
    if len(shape) != 1:
        raise ValueError(f"expected a 1-D vector, got shape {shape}")
    return int(shape[0])


def _need_len(x, n, what):
    """Reject a vector whose length is not n before any pointer reaches the
    C ABI: the kernels and host copies read exactly n entries."""
    k = _length(x)
    if k != n:
        raise ValueError(f"{what} has {k} entries, expected {n}")


def _dev_i32(x):
    torch = _torch()
    t = torch.as_tensor(x)
    if t.dtype != torch.int32:
        t = t.to(torch.int32)
    if not t.is_cuda:
        t = t.cuda()
    return t.contiguous()


def _dev_f64(x):
    torch = _torch()
    t = torch.as_tensor(x)
    if t.dtype != torch.float64:
        t = t.to(torch.float64)
    if not t.is_cuda:
        t = t.cuda()
    return t.contiguous()


CANONICALIZE = 1
PARTITION_TIMING = 1


class Graph:
    """Prepared graph (``pr_graph``): validated CSR, loop-free, with CSC.
    ``canonicalize=True`` sorts the rows and drops repeated columns instead
    of rejecting them (PR_CANONICALIZE)."""

    def __init__(self, rowptr, col, on_host=False, canonicalize=False):
        lib = load_library()
        self._h = C.c_void_p()
        if on_host:
            rp = np.ascontiguousarray(rowptr, dtype=np.int32)
            cl = np.ascontiguousarray(col, dtype=np.int32)
            keep = (rp, cl)
            csr = _Csr(rp.shape[0] - 1, cl.shape[0], rp.ctypes.data, cl.ctypes.data, 1)
        else:
            rp = _dev_i32(rowptr)
            cl = _dev_i32(col)
            keep = (rp, cl)
            csr = _Csr(rp.shape[0] - 1, cl.shape[0], rp.data_ptr(), cl.data_ptr() if cl.numel() else None, 0)
        self.n = int(csr.n)
        rc = lib.pr_graph_create_ex(C.byref(csr), CANONICALIZE if canonicalize else 0, _stream(), C.byref(self._h))
        del keep
        _check(rc, "pr_graph_create")

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load_library().pr_graph_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Partition:
    """SCC/CAC partition with levels and the solver layout (``pr_partition``)."""

    def __init__(self, g: Graph, timing=False, path=None):
        lib = load_library()
        self.graph = g  # the partition refers to the graph's buffers
        self._h = C.c_void_p()
        if path is None:
            _check(lib.pr_partition_create(g.handle, PARTITION_TIMING if timing else 0, _stream(),
                                           C.byref(self._h)), "pr_partition_create")
        else:
            _check(lib.pr_partition_load(g.handle, os.fsencode(path), 0, _stream(), C.byref(self._h)),
                   "pr_partition_load")
        n, m, nc, nl, ns, nsv = (C.c_int32(), C.c_int64(), C.c_int32(), C.c_int32(), C.c_int32(),
                                 C.c_int32())
        _check(lib.pr_partition_info(self._h, C.byref(n), C.byref(m), C.byref(nc), C.byref(nl),
                                     C.byref(ns), C.byref(nsv)), "pr_partition_info")
        self.n, self.m, self.n_comp, self.n_levels = n.value, m.value, nc.value, nl.value
        self.n_scc, self.n_scc_vertices = ns.value, nsv.value

    @property
    def handle(self):
        return self._h

    def query(self):
        """(comp_id int32, type uint8, level int32) CUDA tensors, original order."""
        torch = _torch()
        comp = torch.empty(self.n, dtype=torch.int32, device="cuda")
        typ = torch.empty(self.n, dtype=torch.uint8, device="cuda")
        lev = torch.empty(self.n, dtype=torch.int32, device="cuda")
        nc, nl = C.c_int32(), C.c_int32()
        _check(load_library().pr_partition_query(self._h, comp.data_ptr() if self.n else None,
                                                 typ.data_ptr() if self.n else None,
                                                 lev.data_ptr() if self.n else None,
                                                 C.byref(nc), C.byref(nl), _stream()),
               "pr_partition_query")
        return comp, typ, lev

    def timing(self):
        """Phase times (ms) and wave counts of a partition built with
        ``timing=True`` (pr_partition_timing_get)."""
        t = _PartTiming()
        _check(load_library().pr_partition_timing_get(self._h, C.byref(t)), "pr_partition_timing_get")
        kinds = ("trim", "propagate", "reach", "root_bfs", "kahn")
        return {"trim_ms": t.trim_ms, "giant_ms": t.giant_ms, "colour_ms": t.colour_ms,
                "levels_ms": t.levels_ms, "layout_ms": t.layout_ms, "total_ms": t.total_ms,
                "colour_rounds": t.colour_rounds,
                "waves": {k: {"grid": t.waves[i][0], "block": t.waves[i][1]} for i, k in enumerate(kinds)}}

    def save(self, path):
        """Write the partition to a file (pr_partition_save); ``load_partition``
        reads it back for the same graph."""
        _check(load_library().pr_partition_save(self._h, os.fsencode(path), _stream()), "pr_partition_save")

    def tune(self, c, u, tol):
        """Autotune the solve's launch shapes on this partition (see
        pr_partition_tune); returns {"cta_max", "coop_blocks", "balance", "best_ms"}."""
        _need_len(u, self.n, "u")
        ud = _dev_f64(u)
        a, b, bl, t = C.c_int32(), C.c_int32(), C.c_int32(), C.c_float()
        _check(load_library().pr_partition_tune(self._h, float(c), ud.data_ptr() if self.n else None, float(tol),
                                                _stream(), C.byref(a), C.byref(b), C.byref(bl), C.byref(t)),
               "pr_partition_tune")
        return {"cta_max": a.value, "coop_blocks": b.value, "balance": bl.value, "best_ms": t.value}

    def set_shape(self, cta_max, coop_blocks, balance=1):
        """Set the tuner's parameters by hand (pr_partition_set_shape)."""
        _check(load_library().pr_partition_set_shape(self._h, int(cta_max), int(coop_blocks), int(balance)),
               "pr_partition_set_shape")

    def close(self):
        if self._h:
            load_library().pr_partition_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def graph(rowptr, col, on_host=False, canonicalize=False):
    return Graph(rowptr, col, on_host=on_host, canonicalize=canonicalize)


def partition(g, col=None, on_host=False, timing=False):
    """``partition(graph)``, or ``partition(rowptr, col)`` for a CSR (the
    graph is prepared on the way and kept alive by the partition).
    ``timing=True`` records the phase times (PR_PARTITION_TIMING), read by
    ``Partition.timing()``."""
    if col is not None:
        g = Graph(g, col, on_host=on_host)
    elif not isinstance(g, Graph):
        raise TypeError("partition() takes a Graph, or rowptr and col")
    return Partition(g, timing=timing)


def load_partition(g, path):
    """The partition of graph ``g`` saved by ``Partition.save`` (pr_partition_load):
    the same components, levels and solves as ``partition(g)``, without the
    component search."""
    if not isinstance(g, Graph):
        raise TypeError("load_partition() takes a Graph")
    return Partition(g, path=path)


def _opts(norm, max_iter, io_on_host, replay, precision=PREC_FP64, warm=None, lu_threshold=0):
    o = _Opts(int(norm), int(max_iter), int(precision), int(io_on_host), None,
              warm.handle if warm is not None else None, int(lu_threshold))
    keep = None
    if replay is not None:
        keep = np.ascontiguousarray(replay, dtype=np.int32)
        o.replay_iters = keep.ctypes.data
    return o, keep


def launch_count():
    """Kernels launched by the library in this process so far."""
    return int(load_library().pr_launch_count())


def set_wait_limit(microseconds):
    """Time limit of the bounded device-side waits for later calls
    (pr_set_wait_limit); 0 restores the default of two seconds."""
    _check(load_library().pr_set_wait_limit(int(microseconds)), "pr_set_wait_limit")


def _stats_dict(st):
    return {"iters_max": st.iters_max, "n_levels": st.n_levels, "edge_visits": st.edge_visits,
            "launches": st.launches, "kernel_ms": st.kernel_ms, "kernel_bytes": st.kernel_bytes,
            "kernel_launches": st.kernel_launches, "fp64_sweeps_max": st.fp64_sweeps_max,
            "fp64_edge_visits": st.fp64_edge_visits}


def solve(part: Partition, c, u, tol, norm=NORM_L1, max_iter=10_000, replay_iters=None,
          with_stats=False, allow_noconv=False, timing=False, precision=PREC_FP64, warm_start=None,
          lu_threshold=0, level_times=False, counts=True):
    """Sec. 4.3 solve on device tensors; returns R (float64, original order).

    ``u`` may be a CUDA tensor or a numpy array (host I/O through the C ABI's
    io_on_host path; R is then returned as numpy).  ``precision=PREC_MIXED``
    runs the SCC series in FP32 with FP64 residual refinement;
    ``warm_start`` (an ``Mpnn``) starts each SCC's series from the network's
    guess; SCCs of fewer than ``lu_threshold`` vertices are solved by dense
    elimination (Sec. 4.3 item 3).  ``timing`` times the grid-wide series
    kernels (stats ``kernel_ms``); ``level_times`` also records an event
    between the levels (stats ``level_ms``; the events cost a few
    microseconds a level).  ``counts=False`` skips the per-component sweep
    counts and edge visits (read back and summed on the host otherwise)."""
    _need_len(u, part.n, "u")
    if replay_iters is not None:
        _need_len(replay_iters, part.n_comp, "replay_iters")
    lib = load_library()
    on_host = isinstance(u, np.ndarray)
    o, keep = _opts(norm, max_iter, on_host, replay_iters, precision, warm_start, lu_threshold)
    comp_iters = np.zeros(max(part.n_comp, 1), np.int32)
    level_ms = np.zeros(max(part.n_levels, 1), np.float32)
    tmode = 2 if level_times else (1 if timing else 0)
    st = _Stats(0, 0, 0, 0, comp_iters.ctypes.data if counts else None, tmode, 0.0, 0, 0, 0, 0,
                level_ms.ctypes.data, 0 if counts else 1)
    if on_host:
        uh = np.ascontiguousarray(u, dtype=np.float64)
        R = np.empty(part.n, np.float64)
        rc = lib.pr_solve(part.handle, float(c), uh.ctypes.data, float(tol), C.byref(o),
                          R.ctypes.data, C.byref(st), _stream())
    else:
        torch = _torch()
        ud = _dev_f64(u)
        R = torch.empty(part.n, dtype=torch.float64, device="cuda")
        rc = lib.pr_solve(part.handle, float(c), ud.data_ptr() if part.n else None, float(tol),
                          C.byref(o), R.data_ptr() if part.n else None, C.byref(st), _stream())
    if not (allow_noconv and rc == 4):
        _check(rc, "pr_solve")
    del keep
    if with_stats:
        d = _stats_dict(st)
        d.update(status=rc)
        if counts:
            d.update(comp_iters=comp_iters[: part.n_comp].copy())
        if level_times:
            d.update(level_ms=level_ms[: part.n_levels].copy())
        return R, d
    return R


def global_power(g: Graph, c, u, tol, norm=NORM_L1, max_iter=10_000, replay_iters=None,
                 with_stats=False, allow_noconv=False, timing=False):
    """Baseline power series on the whole graph; returns (R, iterations)."""
    _need_len(u, g.n, "u")
    lib = load_library()
    on_host = isinstance(u, np.ndarray)
    rep = None if replay_iters is None else [int(replay_iters)]
    o, keep = _opts(norm, max_iter, on_host, rep)
    st = _Stats(0, 0, 0, 0, None, int(timing), 0.0, 0, 0, 0, 0, None, 0)
    if on_host:
        uh = np.ascontiguousarray(u, dtype=np.float64)
        R = np.empty(g.n, np.float64)
        rc = lib.pr_global_power(g.handle, float(c), uh.ctypes.data, float(tol), C.byref(o),
                                 R.ctypes.data, C.byref(st), _stream())
    else:
        torch = _torch()
        ud = _dev_f64(u)
        R = torch.empty(g.n, dtype=torch.float64, device="cuda")
        rc = lib.pr_global_power(g.handle, float(c), ud.data_ptr() if g.n else None, float(tol),
                                 C.byref(o), R.data_ptr() if g.n else None, C.byref(st), _stream())
    if not (allow_noconv and rc == 4):
        _check(rc, "pr_global_power")
    del keep
    if with_stats:
        d = _stats_dict(st)
        d.update(status=rc)
        return R, st.iters_max, d
    return R, st.iters_max


def residual_l1(g: Graph, c, u, R):
    """|| u + c A^T (R/outdeg) - R ||_1 in FP64 on the device."""
    _need_len(u, g.n, "u")
    _need_len(R, g.n, "R")
    lib = load_library()
    ud = _dev_f64(u)
    Rd = _dev_f64(R)
    out = C.c_double(0.0)
    _check(lib.pr_residual_l1(g.handle, float(c), ud.data_ptr() if g.n else None,
                              Rd.data_ptr() if g.n else None, C.byref(out), _stream()),
           "pr_residual_l1")
    return out.value


def residual_l1_static(rowptr, col, c, u, R):
    """The L1 residual through pr_residual_l1_static, which allocates no device
    memory (for callers that cannot allocate); all arguments on the device,
    n <= STATIC_MAX_N."""
    n = _length(rowptr) - 1
    if n < 0:
        raise ValueError("rowptr needs at least one entry")
    _need_len(u, n, "u")
    _need_len(R, n, "R")
    lib = load_library()
    rp = _dev_i32(rowptr)
    cl = _dev_i32(col)
    ud = _dev_f64(u)
    Rd = _dev_f64(R)
    n = rp.shape[0] - 1
    csr = _Csr(n, cl.shape[0], rp.data_ptr(), cl.data_ptr() if cl.numel() else None, 0)
    out = C.c_double(0.0)
    _check(lib.pr_residual_l1_static(C.byref(csr), float(c), ud.data_ptr() if n else None,
                                     Rd.data_ptr() if n else None, C.byref(out), _stream()),
           "pr_residual_l1_static")
    return out.value


class Mpnn:
    """Learned warm start (``pr_mpnn``): a two-layer message-passing network
    over each SCC's internal in-edges that guesses R_i / W_i; trained with the
    library's own forward and backward kernels."""

    def __init__(self, seed=0):
        lib = load_library()
        self._h = C.c_void_p()
        _check(lib.pr_mpnn_create(C.c_uint64(int(seed)), _stream(), C.byref(self._h)), "pr_mpnn_create")
        self.n_params = int(lib.pr_mpnn_param_count())

    @property
    def handle(self):
        return self._h

    def get_params(self):
        out = np.empty(self.n_params, np.float32)
        _check(load_library().pr_mpnn_get_params(self._h, out.ctypes.data, self.n_params), "pr_mpnn_get_params")
        return out

    def set_params(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        _check(load_library().pr_mpnn_set_params(self._h, theta.ctypes.data, int(theta.size)),
               "pr_mpnn_set_params")

    def predict(self, part: Partition, c, u, R):
        """(yhat float32 CUDA tensor in the original vertex order, loss)."""
        _need_len(u, part.n, "u")
        _need_len(R, part.n, "R")
        torch = _torch()
        ud, Rd = _dev_f64(u), _dev_f64(R)
        y = torch.zeros(part.n, dtype=torch.float32, device="cuda")
        loss = C.c_double(0.0)
        _check(load_library().pr_mpnn_predict(self._h, part.handle, float(c), ud.data_ptr() if part.n else None,
                                              Rd.data_ptr() if part.n else None,
                                              y.data_ptr() if part.n else None, C.byref(loss), _stream()),
               "pr_mpnn_predict")
        return y, loss.value

    def loss_grad(self, part: Partition, c, u, R):
        _need_len(u, part.n, "u")
        _need_len(R, part.n, "R")
        ud, Rd = _dev_f64(u), _dev_f64(R)
        g = np.empty(self.n_params, np.float32)
        loss = C.c_double(0.0)
        _check(load_library().pr_mpnn_loss_grad(self._h, part.handle, float(c), ud.data_ptr() if part.n else None,
                                                Rd.data_ptr() if part.n else None, g.ctypes.data,
                                                C.byref(loss), _stream()),
               "pr_mpnn_loss_grad")
        return loss.value, g

    def train_step(self, part: Partition, c, u, R, lr=1e-3):
        _need_len(u, part.n, "u")
        _need_len(R, part.n, "R")
        ud, Rd = _dev_f64(u), _dev_f64(R)
        loss = C.c_double(0.0)
        _check(load_library().pr_mpnn_train_step(self._h, part.handle, float(c),
                                                 ud.data_ptr() if part.n else None,
                                                 Rd.data_ptr() if part.n else None, C.c_float(lr),
                                                 C.byref(loss), _stream()),
               "pr_mpnn_train_step")
        return loss.value

    def close(self):
        if self._h:
            load_library().pr_mpnn_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
