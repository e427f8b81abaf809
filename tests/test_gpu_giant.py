"""The grid-wide SCC series (SCCs above 16,384 vertices) in exact fixed
point: the L-infinity stopping rule against the oracle, and the path for a
component whose light rows are too many for the SELL-32 slices (more than
2^31 / (32 * 64) slices), pinned by the FP64 residual kernel and the global
power series -- two independent computations of the same R."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

C = 0.85
RTOL = 1e-12


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


def test_grid_wide_linf_rule(prgb):
    """The paper's stopping rule (iterate while max P >= tol) on a graph with
    a grid-wide SCC: the GPU's sweep counts replayed by the oracle give the
    same R, and its own decisions are the oracle's within one sweep."""
    import torch
    g = gg.web_like(seed=12, n=60_000, n_small=1_200, layers=12, giant_layer=4)
    G = prgb.graph(g.rowptr, g.col)
    P = prgb.partition(G)
    q = oracle.partition(g.rowptr, g.col)
    sizes = np.bincount(q.comp)
    assert sizes.max() > 16_384
    u = torch.from_numpy(g.u).cuda()
    tol = 1e-13
    R, st = prgb.solve(P, C, u, tol, norm=prgb.NORM_LINF, with_stats=True)
    R = R.cpu().numpy()
    its = st["comp_iters"]
    Ro, its_o = oracle.solve_cw(g.rowptr, g.col, q, C, g.u, tol, norm=oracle.NORM_LINF, replay_iters=its)
    assert np.array_equal(its_o, its)
    assert np.max(np.abs(R - Ro) / np.maximum(np.abs(Ro), 1e-300)) <= RTOL
    _, its_nat = oracle.solve_cw(g.rowptr, g.col, q, C, g.u, tol, norm=oracle.NORM_LINF)
    assert np.all(np.abs(its_nat - its) <= 1)


def test_grid_wide_without_slices(prgb):
    """A random digraph of 37M vertices with three out-edges each: its giant
    SCC (~94% of the vertices, none with more than 64 in-edges) has more
    light rows than the SELL-32 slices can index, so the series walks the
    rows from the in-CSR.  R must meet the L1 residual bound (FP64 residual
    kernel) and agree with the global power series within both stopping
    budgets."""
    import torch
    n, d = 37_000_000, 3
    gen = torch.Generator(device="cuda").manual_seed(5)
    rowptr = torch.arange(0, d * n + 1, d, dtype=torch.int32, device="cuda")
    col = torch.randint(0, n, (d * n,), generator=gen, dtype=torch.int32, device="cuda")
    G = prgb.graph(rowptr, col, canonicalize=True)
    del col
    P = prgb.partition(G)
    assert P.n_scc_vertices > 33_554_432 + 1_000_000  # more light rows than 2^31 / 64 slots
    u = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda")
    tol = 1e-10
    R, st = prgb.solve(P, C, u, tol, with_stats=True)
    assert st["status"] == 0
    floor = 8 * 2.2e-16 * (1.0 + 2 * float(R.sum().item()))
    assert prgb.residual_l1(G, C, u, R) <= C * tol * (1 + 1e-6) + floor
    Rg, _ = prgb.global_power(G, C, u, tol)
    assert float((R - Rg).abs().sum().item()) <= 4 * tol / (1 - C) + 2 * floor / (1 - C)


def test_grid_wide_fp64_gathers(prgb):
    """A giant SCC whose fixed-point sweep does not fit in half the L2 (48 B
    per vertex) but still has SELL slices: z is gathered as FP64 values and
    decoded into the exact sums.  Against the oracle with the GPU's sweep
    counts replayed (1e-12 per entry); by its own rule against the residual
    bound and the global power series."""
    import torch
    rng = np.random.default_rng(17)
    n, d = 1_600_000, 3
    src = np.repeat(np.arange(n), d)
    dst = rng.integers(0, n, d * n)
    rp, col = gg.csr_from_edges(n, src, dst)
    G = prgb.graph(rp, col)
    P = prgb.partition(G)
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    assert P.n_scc_vertices * 48 > l2 // 2  # the giant gathers FP64 values
    q = oracle.partition(rp, col)
    u = np.full(n, 1.0 / n)
    ud = torch.from_numpy(u).cuda()
    tol = 1e-10
    R, st = prgb.solve(P, C, ud, tol, with_stats=True)
    R = R.cpu().numpy()
    its = st["comp_iters"]
    Ro, _ = oracle.solve_cw(rp, col, q, C, u, tol, replay_iters=its)
    assert np.max(np.abs(R - Ro) / np.maximum(np.abs(Ro), 1e-300)) <= RTOL
    floor = 8 * 2.2e-16 * (1.0 + 2 * R.sum())
    assert prgb.residual_l1(G, C, ud, torch.from_numpy(R).cuda()) <= C * tol * (1 + 1e-6) + floor
    Rg, _ = prgb.global_power(G, C, ud, tol)
    assert float(np.abs(R - Rg.cpu().numpy()).sum()) <= 4 * tol / (1 - C) + 2 * floor / (1 - C)
