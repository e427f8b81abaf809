"""pr_residual_l1_static: the residual entry point that allocates nothing.

It exists for callers that cannot allocate device memory (code inside another
framework's memory manager, or on a path where cudaMalloc would synchronise
the device).  Its scratch is a fixed array in the library's device data
segment that every call reuses, so two calls in a row must both agree with
the allocating entry point (a stale accumulator from the first call would
show up in the second).  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

CC = 0.85


@pytest.fixture(scope="module")
def prgb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_09068_gb300 as m
    from paper_1609_09068_gb300 import _build
    _build.build()
    m.load_library()
    return m


def _static_via_abi(prgb, rowptr, col, u, R):
    """Call pr_residual_l1_static through the C ABI with device buffers."""
    lib = prgb.load_library()
    csr = prgb._Csr(rowptr.shape[0] - 1, col.shape[0], rowptr.data_ptr(), col.data_ptr(), 0)
    out = C.c_double(-1.0)
    rc = lib.pr_residual_l1_static(C.byref(csr), CC, u.data_ptr(), R.data_ptr(), C.byref(out), prgb._stream())
    return rc, out.value


def test_static_residual_matches_allocating_one_twice(prgb):
    import torch
    g = gg.web_like(seed=21, n=200_000, n_small=4_000, layers=12, giant_layer=4)
    rowptr = torch.from_numpy(g.rowptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    u = torch.from_numpy(g.u).cuda()
    G = prgb.graph(rowptr, col)
    rng = np.random.default_rng(3)
    cases = [torch.from_numpy(rng.random(g.n) / g.n).cuda(), u.clone()]
    for R in cases:  # two calls in a row, different inputs
        rc, r_static = _static_via_abi(prgb, rowptr, col, u, R)
        assert rc == 0
        r_ref = prgb.residual_l1(G, CC, u, R)
        # both sum non-negative in-flows in different orders: a few ulps of
        # the terms, the same floor the parity tests allow
        floor = 8 * 2.2e-16 * (float(u.sum()) + 2 * float(R.sum()))
        assert abs(r_static - r_ref) <= 1e-12 * abs(r_ref) + floor


def test_static_residual_of_a_solution(prgb):
    import torch
    g = gg.small_planted(seed=5)
    rowptr = torch.from_numpy(g.rowptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    u = torch.from_numpy(g.u).cuda()
    G = prgb.graph(rowptr, col)
    P = prgb.partition(G)
    R = prgb.solve(P, CC, u, 1e-10)
    r1 = prgb.residual_l1_static(rowptr, col, CC, u, R)
    r2 = prgb.residual_l1_static(rowptr, col, CC, u, R)
    r_ref = prgb.residual_l1(G, CC, u, R)
    floor = 8 * 2.2e-16 * (float(u.sum()) + 2 * float(R.sum()))
    for r in (r1, r2):
        assert abs(r - r_ref) <= 1e-12 * abs(r_ref) + floor
        assert r <= CC * 1e-10 + floor


def test_static_residual_rejects_oversized_input(prgb):
    import torch
    n = prgb.STATIC_MAX_N + 1
    rowptr = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    lib = prgb.load_library()
    csr = prgb._Csr(n, 0, rowptr.data_ptr(), col.data_ptr(), 0)
    out = C.c_double(0.0)
    assert lib.pr_residual_l1_static(C.byref(csr), CC, u.data_ptr(), u.data_ptr(), C.byref(out),
                                     prgb._stream()) == 1


def test_static_residual_matches_oracle(prgb):
    """Against the CPU oracle's residual of the same vectors (its own
    definition of u + c A^T (R/outdeg) - R, summed in FP64 on the host)."""
    import torch
    g = gg.small_planted(seed=7)
    rowptr = torch.from_numpy(g.rowptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    u = torch.from_numpy(g.u).cuda()
    P = prgb.partition(prgb.graph(rowptr, col))
    rng = np.random.default_rng(11)
    for R in (prgb.solve(P, CC, u, 1e-10), torch.from_numpy(rng.random(g.n) / g.n).cuda()):
        r_static = prgb.residual_l1_static(rowptr, col, CC, u, R)
        r_oracle = oracle.residual_l1(g.rowptr, g.col, CC, g.u, R.cpu().numpy())
        floor = 8 * 2.2e-16 * (float(u.sum()) + 2 * float(R.sum()))
        assert abs(r_static - r_oracle) <= 1e-12 * abs(r_oracle) + floor


def _driver():
    """libcuda through ctypes: the device's free memory and the high-water mark
    of its default stream-ordered pool (the pool cudaMallocAsync draws from)."""
    cu = C.CDLL("libcuda.so.1")
    dev = C.c_int(0)
    assert cu.cuCtxGetDevice(C.byref(dev)) == 0
    pool = C.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(C.byref(pool), dev) == 0
    used_high = 8  # CU_MEMPOOL_ATTR_USED_MEM_HIGH

    def reset_high():
        zero = C.c_uint64(0)
        assert cu.cuMemPoolSetAttribute(pool, used_high, C.byref(zero)) == 0

    def high():
        v = C.c_uint64(0)
        assert cu.cuMemPoolGetAttribute(pool, used_high, C.byref(v)) == 0
        return v.value

    def free_bytes():
        f, t = C.c_size_t(0), C.c_size_t(0)
        assert cu.cuMemGetInfo_v2(C.byref(f), C.byref(t)) == 0
        return f.value

    return reset_high, high, free_bytes


def test_static_residual_allocates_nothing(prgb):
    """Across a call (after the first, which looks up the scratch address):
    the default pool's high-water mark does not rise above what was in use
    before, device free memory does not move, and torch's allocator is not
    touched."""
    import gc

    import torch
    g = gg.web_like(seed=23, n=100_000, n_small=2_000, layers=10, giant_layer=3)
    rowptr = torch.from_numpy(g.rowptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    u = torch.from_numpy(g.u).cuda()
    R = u * 3.0
    prgb.residual_l1_static(rowptr, col, CC, u, R)  # set-up call
    # objects left by earlier tests are collected now, not inside the window
    # (their destructors release memory through the library and torch)
    gc.collect()
    torch.cuda.synchronize()
    reset_high, high, free_bytes = _driver()
    reset_high()
    h0, f0 = high(), free_bytes()
    t0 = torch.cuda.memory_allocated()
    torch.cuda.reset_peak_memory_stats()
    gc.disable()
    try:
        for _ in range(2):
            prgb.residual_l1_static(rowptr, col, CC, u, R)
        torch.cuda.synchronize()
    finally:
        gc.enable()
    assert high() == h0
    assert free_bytes() == f0
    assert torch.cuda.max_memory_allocated() == t0


def test_static_residual_rejects_unsorted_rows(prgb):
    """A repeated or out-of-order column is a malformed CSR, as for
    pr_graph_create (every index stays in range, so the check reads in
    bounds)."""
    import torch
    n = 4
    for rp, cl in (([0, 2, 3, 4, 5], [1, 1, 2, 3, 0]),    # duplicate 0 -> 1
                   ([0, 2, 3, 4, 5], [2, 1, 2, 3, 0])):   # unsorted row 0
        rowptr = torch.tensor(rp, dtype=torch.int32, device="cuda")
        col = torch.tensor(cl, dtype=torch.int32, device="cuda")
        u = torch.full((n,), 0.25, dtype=torch.float64, device="cuda")
        rc, _ = _static_via_abi(prgb, rowptr, col, u, u)
        assert rc == 1
        with pytest.raises(prgb.PrError):
            prgb.graph(rowptr, col)
