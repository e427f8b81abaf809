"""Failure paths, exercised without faulting, trapping or hanging the GPU.

* Bounded device waits: with pr_set_wait_limit at one microsecond the grid
  barriers of the persistent kernels give up; the call returns PR_ETIMEOUT,
  the kernels have returned, and the next call with the default limit
  succeeds on the same context.
* Host-side fault injection (PRGB_FAULT): a device allocation, a kernel
  launch or a host<->device copy reported as failed gives PR_ENOMEM /
  PR_ECUDA, every buffer of the failed call is
  released (the stream-ordered pool's bytes in use are back where they
  were), and the library keeps working; PRGB_FAULT=noconv gives PR_ENOCONV
  with the partial result.
* PR_CANONICALIZE: unsorted rows with repeated columns give the same graph as
  their canonical CSR.
"""
import ctypes as C
import os

import numpy as np
import pytest

import graphgen as gg

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


@pytest.fixture
def fault():
    """Sets PRGB_FAULT for the body of a test and always clears it."""
    def arm(spec):
        os.environ["PRGB_FAULT"] = spec
    yield arm
    os.environ.pop("PRGB_FAULT", None)


def _pool_used():
    """Bytes in use in the device's default stream-ordered pool (the one the
    library allocates from), through libcuda."""
    import torch
    torch.cuda.synchronize()
    cu = C.CDLL("libcuda.so.1")
    dev = C.c_int(0)
    assert cu.cuCtxGetDevice(C.byref(dev)) == 0
    pool = C.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(C.byref(pool), dev) == 0
    v = C.c_uint64(0)
    assert cu.cuMemPoolGetAttribute(pool, 7, C.byref(v)) == 0  # CU_MEMPOOL_ATTR_USED_MEM_CURRENT
    return v.value


def _graph_data(torch, seed=7, n=100_000):
    g = gg.web_like(seed=seed, n=n, n_small=2_000, layers=10, giant_layer=3)
    return g, torch.from_numpy(g.rowptr).cuda(), torch.from_numpy(g.col).cuda(), torch.from_numpy(g.u).cuda()


def test_wait_limit_times_out_and_recovers(prgb):
    import torch
    g, rp, col, u = _graph_data(torch)
    G = prgb.graph(rp, col)
    P = prgb.partition(G)
    assert P.n_scc_vertices > 16_384  # a grid-wide component: the solve has grid barriers
    prgb.set_wait_limit(1)
    try:
        codes = []
        for _ in range(5):
            try:
                prgb.global_power(G, CC, u, 1e-10)
                codes.append(0)
            except prgb.PrError as e:
                codes.append(e.code)
        assert 5 in codes and set(codes) <= {0, 5}  # PR_ETIMEOUT, never anything else
        with pytest.raises(prgb.PrError) as ei:
            for _ in range(5):
                prgb.solve(P, CC, u, 1e-10)
        assert ei.value.name == "PR_ETIMEOUT"
        with pytest.raises(prgb.PrError) as ei:
            for _ in range(5):
                prgb.partition(G)
        assert ei.value.name == "PR_ETIMEOUT"
    finally:
        prgb.set_wait_limit(0)
    # the context is usable and the default limit is back
    R, k = prgb.global_power(G, CC, u, 1e-10)
    assert prgb.residual_l1(G, CC, u, R) <= CC * 1e-10 * (1 + 1e-6) + 1e-15
    P2 = prgb.partition(G)
    R2 = prgb.solve(P2, CC, u, 1e-10)
    assert torch.equal(prgb.solve(P, CC, u, 1e-10), R2)
    assert prgb.residual_l1(G, CC, u, R2) <= CC * 1e-10 * (1 + 1e-6) + 1e-15


@pytest.mark.parametrize("spec,call,code", [
    ("alloc:1", "graph", 2),
    ("alloc:25", "partition", 2),
    ("launch:1", "graph", 3),
    ("launch:30", "partition", 3),
    ("copy:1", "graph_host", 3),
    ("copy:1", "solve_host", 3),
    ("launch:2", "global", 3),
])
def test_injected_faults_release_everything(prgb, fault, spec, call, code):
    import torch
    g, rp, col, u = _graph_data(torch, seed=9, n=30_000)
    G = prgb.graph(rp, col)
    before = _pool_used()
    fault(spec)
    with pytest.raises(prgb.PrError) as ei:
        if call == "graph":
            prgb.graph(rp, col)
        elif call == "graph_host":
            prgb.graph(g.rowptr, g.col, on_host=True)
        elif call == "partition":
            prgb.partition(G)
        elif call == "global":
            prgb.global_power(G, CC, u, 1e-10)
        else:
            P = prgb.Partition(G)  # device CSR: no host copies, the count stays at 0
            try:
                prgb.solve(P, CC, g.u, 1e-10)
            finally:
                P.close()
    assert ei.value.code == code
    os.environ.pop("PRGB_FAULT", None)
    assert _pool_used() == before
    # the library still works
    P = prgb.partition(G)
    R = prgb.solve(P, CC, u, 1e-10)
    assert prgb.residual_l1(G, CC, u, R) <= CC * 1e-10 * (1 + 1e-6) + 1e-15


def test_noconv_gives_partial_result(prgb, fault):
    import torch
    g, rp, col, u = _graph_data(torch, seed=11, n=30_000)
    G = prgb.graph(rp, col)
    P = prgb.partition(G)
    R_full = prgb.solve(P, CC, u, 1e-10)
    fault("noconv")
    R, st = prgb.solve(P, CC, u, 1e-10, with_stats=True, allow_noconv=True)
    assert st["status"] == 4 and st["iters_max"] == 1
    Rg, k, stg = prgb.global_power(G, CC, u, 1e-10, with_stats=True, allow_noconv=True)
    assert stg["status"] == 4 and k == 1
    os.environ.pop("PRGB_FAULT", None)
    # partial sums of non-negative series: below the converged result
    assert bool((R <= R_full * (1 + 1e-12)).all())
    assert prgb.residual_l1(G, CC, u, R) > 1e-10


def test_canonicalize_matches_the_canonical_csr(prgb):
    import torch
    rng = np.random.default_rng(5)
    g = gg.small_planted(seed=4)
    n = g.n
    src = np.repeat(np.arange(n), np.diff(g.rowptr))
    dst = g.col.astype(np.int64)
    # repeat a third of the edges and shuffle every row
    extra = rng.random(src.shape[0]) < 0.33
    s2 = np.concatenate([src, src[extra]])
    d2 = np.concatenate([dst, dst[extra]])
    order = np.lexsort((rng.random(s2.shape[0]), s2))
    s2, d2 = s2[order], d2[order]
    rp = np.zeros(n + 1, np.int32)
    np.cumsum(np.bincount(s2, minlength=n), out=rp[1:])
    messy = d2.astype(np.int32)
    with pytest.raises(prgb.PrError) as ei:
        prgb.graph(rp, messy)
    assert ei.value.name == "PR_EINVAL"
    G1 = prgb.graph(rp, messy, canonicalize=True)
    G2 = prgb.graph(g.rowptr, g.col)
    P1, P2 = prgb.partition(G1), prgb.partition(G2)
    for a, b in zip(P1.query(), P2.query()):
        assert torch.equal(a, b)
    u = torch.from_numpy(g.u).cuda()
    assert torch.equal(prgb.solve(P1, CC, u, 1e-10), prgb.solve(P2, CC, u, 1e-10))
    # a column out of range is still an error
    bad = messy.copy()
    bad[3] = n
    with pytest.raises(prgb.PrError):
        prgb.graph(rp, bad, canonicalize=True)
