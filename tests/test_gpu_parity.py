"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Partition: bit-exact (canonical component ids, types, levels).
Solve: the GPU's per-component iteration counts are replayed in the oracle so
both sum the same series; R must then agree within 1e-12 relative (FP64: all
terms are non-negative, so reordering the sums moves the result by a few
ulps per term).  Independently, the FP64 residual of the GPU result must be
within the budget c*tol that the L1 stopping rule guarantees.
"""
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


def gpu_partition(prgb, rowptr, col):
    G = prgb.graph(rowptr, col)
    P = prgb.partition(G)
    comp, typ, lev = P.query()
    return G, P, comp.cpu().numpy(), typ.cpu().numpy(), lev.cpu().numpy()


def assert_partition_equal(prgb, rowptr, col):
    G, P, comp, typ, lev = gpu_partition(prgb, rowptr, col)
    q = oracle.partition(rowptr, col)
    assert P.n_comp == q.n_comp and P.n_levels == q.n_levels
    assert np.array_equal(comp, q.comp)
    assert np.array_equal(typ, q.type)
    assert np.array_equal(lev, q.level)
    return G, P, q


def max_rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.maximum(np.abs(b), 1e-300)
    return float(np.max(np.abs(a - b) / den)) if a.size else 0.0


def assert_solve_parity(prgb, g, G, P, q, tol=1e-10, norm=oracle.NORM_L1, lu=0):
    import torch
    u = torch.from_numpy(g.u).cuda()
    R, st = prgb.solve(P, C, u, tol, norm=norm, with_stats=True, lu_threshold=lu)
    R = R.cpu().numpy()
    its = st["comp_iters"]
    Ro, its_o = oracle.solve_cw(g.rowptr, g.col, q, C, g.u, tol, norm=norm, replay_iters=its, lu_threshold=lu)
    assert np.array_equal(its_o, its)
    assert max_rel(R, Ro) <= RTOL
    if norm == oracle.NORM_L1:
        # c*tol from the stopping rule, plus the rounding floor of evaluating
        # u + cA^T(R/outdeg) - R in FP64 (a few ulps of each term)
        bound = C * tol * (1 + 1e-6) + 8 * 2.2e-16 * (g.u.sum() + 2 * R.sum())
        res = prgb.residual_l1(G, C, u, torch.from_numpy(R).cuda())
        assert res <= bound
        assert oracle.residual_l1(g.rowptr, g.col, C, g.u, R) <= bound
    # the GPU's own stopping decisions agree with the oracle's almost everywhere
    _, its_nat = oracle.solve_cw(g.rowptr, g.col, q, C, g.u, tol, norm=norm, lu_threshold=lu)
    ctype = np.zeros(q.n_comp, np.int64)
    ctype[q.comp] = q.type
    scc = ctype == 1
    if scc.any():
        assert np.mean(np.abs(its_nat[scc] - its[scc]) <= 1) == 1.0
    return R, st


def test_fig1(prgb):
    E = [(0, 1), (0, 2), (1, 3), (3, 1), (2, 4), (2, 5), (1, 5), (4, 5), (6, 7), (7, 6), (1, 6)]
    s, d = zip(*E)
    rp, col = gg.csr_from_edges(8, s, d)
    G, P, comp, typ, lev = gpu_partition(prgb, rp, col)
    assert list(comp) == [0, 1, 2, 1, 2, 2, 3, 3]
    assert list(typ) == [0, 1, 0, 1, 0, 0, 1, 1]
    assert list(lev) == [2, 1, 0, 1, 0, 0, 0, 0]


def test_tiny_random_partitions(prgb):
    rng = np.random.default_rng(5)
    for trial in range(300):
        n = int(rng.integers(1, 14))
        m = rng.random((n, n)) < float(rng.choice([0.1, 0.2, 0.35]))
        if trial % 2:
            m = np.triu(m) | (np.tril(m) & (rng.random((n, n)) < 0.1))
        s, d = np.nonzero(m)
        rp, col = gg.csr_from_edges(n, s, d)
        assert_partition_equal(prgb, rp, col)


@pytest.mark.parametrize("seed", [1, 7])
def test_small_planted(prgb, seed):
    g = gg.small_planted(seed=seed)
    G, P, q = assert_partition_equal(prgb, g.rowptr, g.col)
    assert_solve_parity(prgb, g, G, P, q)


@pytest.mark.parametrize("n,seed", [(300, 0), (3000, 1), (5000, 2)])
def test_random_with_loops_and_dangling(prgb, n, seed):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, 3 * n)
    dst = rng.integers(0, n, 3 * n)
    dang = rng.random(n) < 0.2
    keep = ~dang[src]
    rp, col = gg.csr_from_edges(n, src[keep], dst[keep])  # keeps some self-loops
    u = rng.random(n)
    g = gg.Graph(n, rp, col, u / u.sum(), "random")
    G, P, q = assert_partition_equal(prgb, rp, col)
    assert_solve_parity(prgb, g, G, P, q, tol=1e-12)


def test_web_like_reduced(prgb):
    g = gg.web_like(seed=12, n=60_000, n_small=1_200, layers=12, giant_layer=4)
    G, P, q = assert_partition_equal(prgb, g.rowptr, g.col)
    assert P.n_scc_vertices > 20_000  # a grid-wide SCC is exercised
    assert_solve_parity(prgb, g, G, P, q)


def test_deep_dag_reduced(prgb):
    g = gg.deep_dag(seed=13, n=200_000, levels=40)
    G, P, q = assert_partition_equal(prgb, g.rowptr, g.col)
    assert P.n_levels == 40
    assert_solve_parity(prgb, g, G, P, q)


def test_linf_rule(prgb):
    g = gg.small_planted(seed=3)
    G, P, q = assert_partition_equal(prgb, g.rowptr, g.col)
    assert_solve_parity(prgb, g, G, P, q, tol=1e-13, norm=oracle.NORM_LINF)


def test_global_power_parity(prgb):
    import torch
    for g in [gg.small_planted(seed=2), gg.web_like(seed=14, n=40_000, n_small=800, layers=10, giant_layer=3)]:
        G = prgb.graph(g.rowptr, g.col)
        u = torch.from_numpy(g.u).cuda()
        R, k = prgb.global_power(G, C, u, 1e-10)
        Ro, ko = oracle.solve_global(g.rowptr, g.col, C, g.u, 1e-10, replay_iters=k)
        assert max_rel(R.cpu().numpy(), Ro) <= RTOL
        _, k_nat = oracle.solve_global(g.rowptr, g.col, C, g.u, 1e-10)
        assert abs(k_nat - k) <= 1
        assert prgb.residual_l1(G, C, u, R) <= C * 1e-10 * (1 + 1e-6)


def test_residual_matches_oracle(prgb):
    import torch
    g = gg.small_planted(seed=4)
    G = prgb.graph(g.rowptr, g.col)
    for R in [g.u, g.u * 3.0, np.random.default_rng(0).random(g.n)]:
        r = prgb.residual_l1(G, C, torch.from_numpy(g.u).cuda(), torch.from_numpy(R).cuda())
        ro = oracle.residual_l1(g.rowptr, g.col, C, g.u, R)
        assert r == pytest.approx(ro, rel=1e-12)


def test_edge_cases(prgb):
    import torch
    # no vertices
    G = prgb.graph(np.zeros(1, np.int32), np.zeros(0, np.int32))
    P = prgb.partition(G)
    assert P.n_comp == 0 and P.n_levels == 0
    # one vertex, no edges; one vertex with a self-loop
    for rp, col in [(np.array([0, 0]), np.zeros(0)), (np.array([0, 1]), np.array([0]))]:
        rp = np.asarray(rp, np.int32)
        col = np.asarray(col, np.int32)
        G, P, q = assert_partition_equal(prgb, rp, col)
        R = prgb.solve(P, C, torch.tensor([0.5], dtype=torch.float64, device="cuda"), 1e-10)
        assert R.item() == 0.5
    # all vertices dangling
    n = 1000
    rp, col = np.zeros(n + 1, np.int32), np.zeros(0, np.int32)
    g = gg.Graph(n, rp, col, gg.uniform_u(n), "empty")
    G, P, q = assert_partition_equal(prgb, rp, col)
    R = prgb.solve(P, C, torch.from_numpy(g.u).cuda(), 1e-10).cpu().numpy()
    assert np.array_equal(R, g.u)


def test_single_large_cycle_iterations(prgb):
    import math
    import torch
    k = 50_000
    rp, col = gg.csr_from_edges(k, np.arange(k), (np.arange(k) + 1) % k)
    g = gg.Graph(k, rp, col, gg.uniform_u(k), "cycle")
    G, P, q = assert_partition_equal(prgb, rp, col)
    tol = 3e-9  # ln(tol)/ln(c) = 121.07..., far from an integer
    R, st = prgb.solve(P, C, torch.from_numpy(g.u).cuda(), tol, with_stats=True)
    assert st["comp_iters"][0] == math.ceil(math.log(tol) / math.log(C))
    assert_solve_parity(prgb, g, G, P, q, tol=tol)


def test_long_chain_is_one_grid_wide_cac(prgb):
    k = 20_000
    rp, col = gg.csr_from_edges(k, np.arange(k - 1), np.arange(1, k))
    g = gg.Graph(k, rp, col, np.ones(k), "chain")
    G, P, q = assert_partition_equal(prgb, rp, col)
    import torch
    R = prgb.solve(P, C, torch.from_numpy(g.u).cuda(), 1e-10).cpu().numpy()
    i = np.arange(1, k + 1)
    np.testing.assert_allclose(R, (1 - C ** i) / (1 - C), rtol=1e-13)


def test_invalid_inputs(prgb):
    import torch
    with pytest.raises(prgb.PrError) as e:
        prgb.graph(np.array([0, 2, 2], np.int32), np.array([1, 0], np.int32))  # unsorted row
    assert e.value.code == 1
    with pytest.raises(prgb.PrError):
        prgb.graph(np.array([0, 1, 1], np.int32), np.array([7], np.int32))  # out of range
    with pytest.raises(prgb.PrError):
        prgb.graph(np.array([0, 2, 2], np.int32), np.array([1, 1], np.int32))  # duplicate
    g = gg.small_planted(seed=1)
    G = prgb.graph(g.rowptr, g.col)
    P = prgb.partition(G)
    bad = g.u.copy()
    bad[17] = -1.0
    with pytest.raises(prgb.PrError) as e:
        prgb.solve(P, C, torch.from_numpy(bad).cuda(), 1e-10)
    assert e.value.code == 1
    with pytest.raises(prgb.PrError):
        prgb.solve(P, 1.0, torch.from_numpy(g.u).cuda(), 1e-10)
    with pytest.raises(prgb.PrError):
        prgb.solve(P, C, torch.from_numpy(g.u).cuda(), 0.0)
    # the context is still usable
    R = prgb.solve(P, C, torch.from_numpy(g.u).cuda(), 1e-10)
    assert torch.isfinite(R).all()


def test_not_converged_returns_partial(prgb):
    import torch
    g = gg.small_planted(seed=1)
    G, P, q = assert_partition_equal(prgb, g.rowptr, g.col)
    R, st = prgb.solve(P, C, torch.from_numpy(g.u).cuda(), 1e-10, max_iter=3, with_stats=True,
                       allow_noconv=True)
    assert st["status"] == 4
    its = st["comp_iters"]
    assert its.max() == 3
    Ro, _ = oracle.solve_cw(g.rowptr, g.col, q, C, g.u, 1e-10, replay_iters=its)
    assert max_rel(R.cpu().numpy(), Ro) <= RTOL


def test_host_io_matches_device(prgb):
    import torch
    g = gg.small_planted(seed=9)
    Gh = prgb.graph(g.rowptr, g.col, on_host=True)
    P = prgb.partition(Gh)
    Rh = prgb.solve(P, C, g.u, 1e-10)  # numpy in, numpy out
    Rd = prgb.solve(P, C, torch.from_numpy(g.u).cuda(), 1e-10).cpu().numpy()
    assert isinstance(Rh, np.ndarray) and np.array_equal(Rh, Rd)
    Rg, k = prgb.global_power(Gh, C, g.u, 1e-10)
    Rgd, kd = prgb.global_power(Gh, C, torch.from_numpy(g.u).cuda(), 1e-10)
    assert k == kd and np.array_equal(Rg, Rgd.cpu().numpy())


def test_partition_from_csr(prgb):
    """partition(rowptr, col) prepares the graph itself: same result."""
    import torch
    g = gg.small_planted(seed=5)
    P1 = prgb.partition(g.rowptr, g.col)
    P2 = prgb.partition(prgb.graph(g.rowptr, g.col))
    for a, b in zip(P1.query(), P2.query()):
        assert torch.equal(a, b)


def test_deterministic(prgb):
    import torch
    g = gg.web_like(seed=15, n=30_000, n_small=600, layers=8, giant_layer=3)
    G = prgb.graph(g.rowptr, g.col)
    P1 = prgb.partition(G)
    P2 = prgb.partition(G)
    for a, b in zip(P1.query(), P2.query()):
        assert torch.equal(a, b)
    u = torch.from_numpy(g.u).cuda()
    assert torch.equal(prgb.solve(P1, C, u, 1e-10), prgb.solve(P2, C, u, 1e-10))


def test_web_like_full_size(prgb):
    """The benchmark workload (n = 1,000,000, ~8M edges), full parity."""
    g = gg.web_like()
    G, P, q = assert_partition_equal(prgb, g.rowptr, g.col)
    assert P.n_scc_vertices >= 0.35 * g.n
    assert_solve_parity(prgb, g, G, P, q)


def test_deep_dag_full_size(prgb):
    """n = 4,000,000, ~28M edges, 200 forced levels."""
    g = gg.deep_dag()
    G, P, q = assert_partition_equal(prgb, g.rowptr, g.col)
    assert P.n_levels == 200
    assert_solve_parity(prgb, g, G, P, q)


@pytest.mark.parametrize("k", [20, 200, 5_000, 20_000])
def test_chain_in_every_size_class(prgb, k):
    """A chain is one CAC: warp (<=32), CTA (<=256), cluster (<=16384) and
    grid-wide classes all reproduce R_i = (1 - c^i)/(1 - c)."""
    import torch
    rp, col = gg.csr_from_edges(k, np.arange(k - 1), np.arange(1, k))
    G, P, q = assert_partition_equal(prgb, rp, col)
    R = prgb.solve(P, C, torch.ones(k, dtype=torch.float64, device="cuda"), 1e-10).cpu().numpy()
    i = np.arange(1, k + 1)
    np.testing.assert_allclose(R, (1 - C ** i) / (1 - C), rtol=1e-13)


@pytest.mark.parametrize("n,seed", [(3_000, 31), (40_000, 32)])
def test_random_dags(prgb, n, seed):
    """Acyclic graphs: every component is a CAC (of many sizes, merged
    across levels), solved exactly in one pass."""
    rng = np.random.default_rng(seed)
    m = 3 * n
    a = rng.integers(0, n, m)
    b = rng.integers(0, n, m)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    keep = lo != hi
    rp, col = gg.csr_from_edges(n, hi[keep], lo[keep])
    u = rng.random(n)
    g = gg.Graph(n, rp, col, u / u.sum(), "dag")
    G, P, q = assert_partition_equal(prgb, rp, col)
    assert P.n_scc == 0
    assert_solve_parity(prgb, g, G, P, q)


def test_mid_size_sccs_use_clusters(prgb):
    """SCCs of 300-10000 vertices (cluster class) in a layered graph."""
    g = gg.small_planted(seed=33, n=40_000, n_scc=20, scc_vertices=30_000, n_dangling=4_000, layers=6,
                         target_edges=200_000)
    G, P, q = assert_partition_equal(prgb, g.rowptr, g.col)
    sizes = np.bincount(q.comp[q.type == 1])
    assert np.count_nonzero((sizes > 256) & (sizes <= 16384)) >= 10
    assert_solve_parity(prgb, g, G, P, q)


def test_graph_replay_matches_direct_launches(prgb):
    """pr_solve replays a CUDA graph of the level loop cached in the
    partition; the same kernels launched directly (replaying the graph's
    iteration counts) give bit-identical R.  A cached graph is reused, and
    other parameters rebuild it."""
    import torch
    g = gg.web_like(seed=16, n=40_000, n_small=800, layers=10, giant_layer=3)
    G = prgb.graph(g.rowptr, g.col)
    P = prgb.partition(G)
    u = torch.from_numpy(g.u).cuda()
    R1, st1 = prgb.solve(P, C, u, 1e-10, with_stats=True)
    R2 = prgb.solve(P, C, u, 1e-10, replay_iters=st1["comp_iters"])
    assert torch.equal(R1, R2)
    l0 = prgb.launch_count()
    R3, st3 = prgb.solve(P, C, u, 1e-10, with_stats=True)
    assert torch.equal(R1, R3)
    assert np.array_equal(st1["comp_iters"], st3["comp_iters"])
    assert prgb.launch_count() - l0 == st3["launches"] + 1  # + the edge-count kernel of the stats
    R4, st4 = prgb.solve(P, C, u, 1e-7, with_stats=True)
    assert st4["iters_max"] < st1["iters_max"]
    assert prgb.residual_l1(G, C, u, R4) <= C * 1e-7 * (1 + 1e-6)
    Rm = prgb.solve(P, C, u, 1e-10, precision=prgb.PREC_MIXED)
    assert prgb.residual_l1(G, C, u, Rm) <= 1e-10 * (1 + 1e-6)
    assert torch.equal(prgb.solve(P, C, u, 1e-10), R1)


@pytest.mark.parametrize("lu", [30, 101, 129])
def test_small_scc_dense_solve(prgb, lu):
    """Sec. 4.3 item 3: SCCs below the threshold solved by elimination; the
    rest by the series.  Parity with the oracle run with the same threshold
    (iteration counts replayed for the series components)."""
    g = gg.small_planted(seed=1)
    G, P, q = assert_partition_equal(prgb, g.rowptr, g.col)
    R, st = assert_solve_parity(prgb, g, G, P, q, lu=lu)
    sizes = np.bincount(q.comp, minlength=q.n_comp)
    ctype = np.zeros(q.n_comp, np.int64)
    ctype[q.comp] = q.type
    small = (ctype == 1) & (sizes < lu)
    assert small.any()
    assert np.all(st["comp_iters"][small] == 0)
    assert np.all(st["comp_iters"][(ctype == 1) & ~small] > 0)


def test_dense_solve_closed_forms(prgb):
    import torch
    # complete digraph K_m: R = u / (1 - c); a cycle with non-uniform u
    m = 120
    s, d = np.nonzero(~np.eye(m, dtype=bool))
    rp, col = gg.csr_from_edges(m, s, d)
    G = prgb.graph(rp, col)
    P = prgb.partition(G)
    u = np.full(m, 1.0 / m)
    R, st = prgb.solve(P, C, torch.from_numpy(u).cuda(), 1e-10, lu_threshold=129, with_stats=True)
    np.testing.assert_allclose(R.cpu().numpy(), u / (1 - C), rtol=1e-13)
    assert st["comp_iters"][0] == 0
    k = 50
    rp, col = gg.csr_from_edges(k, np.arange(k), (np.arange(k) + 1) % k)
    G = prgb.graph(rp, col)
    P = prgb.partition(G)
    u = np.random.default_rng(0).random(k)
    R = prgb.solve(P, C, torch.from_numpy(u).cuda(), 1e-10, lu_threshold=k + 1).cpu().numpy()
    # R_i = sum_t c^t u_{i-t} / (1 - c^k) on a cycle
    expect = np.array([sum(C ** t * u[(i - t) % k] for t in range(k)) for i in range(k)]) / (1 - C ** k)
    np.testing.assert_allclose(R, expect, rtol=1e-12)


def test_dense_solve_web_like_and_mixed(prgb):
    import torch
    g = gg.web_like(seed=12, n=60_000, n_small=1_200, layers=12, giant_layer=4)
    G, P, q = assert_partition_equal(prgb, g.rowptr, g.col)
    assert_solve_parity(prgb, g, G, P, q, lu=100)
    u = torch.from_numpy(g.u).cuda()
    Rm = prgb.solve(P, C, u, 1e-10, lu_threshold=100, precision=prgb.PREC_MIXED)
    assert prgb.residual_l1(G, C, u, Rm) <= 1e-10 * (1 + 1e-6)
    with pytest.raises(prgb.PrError):
        prgb.solve(P, C, u, 1e-10, lu_threshold=130)


@pytest.mark.parametrize("cta_max,blocks,balance", [(64, 3, 1), (128, 4, 0), (256, 2, 1)])
def test_launch_shapes_keep_parity(prgb, cta_max, blocks, balance):
    """The autotuner's parameters change which kernel class solves a
    component and the grid of the grid-wide kernels, never the result."""
    g = gg.small_planted(seed=33, n=40_000, n_scc=20, scc_vertices=30_000, n_dangling=4_000, layers=6,
                         target_edges=200_000)
    G, P, q = assert_partition_equal(prgb, g.rowptr, g.col)
    P.set_shape(cta_max, blocks, balance)
    assert_solve_parity(prgb, g, G, P, q)
    g2 = gg.web_like(seed=12, n=60_000, n_small=1_200, layers=12, giant_layer=4)
    G2, P2, q2 = assert_partition_equal(prgb, g2.rowptr, g2.col)
    P2.set_shape(cta_max, blocks, balance)
    assert_solve_parity(prgb, g2, G2, P2, q2)


def test_autotuner(prgb):
    import torch
    g = gg.web_like(seed=12, n=60_000, n_small=1_200, layers=12, giant_layer=4)
    G, P, q = assert_partition_equal(prgb, g.rowptr, g.col)
    choice = P.tune(C, torch.from_numpy(g.u).cuda(), 1e-10)
    assert choice["cta_max"] in (64, 128, 256) and choice["coop_blocks"] in (3, 4) and choice["balance"] in (0, 1)
    assert choice["best_ms"] > 0
    assert_solve_parity(prgb, g, G, P, q)
    # partitions created afterwards start from the tuned shape
    G2, P2, q2 = assert_partition_equal(prgb, g.rowptr, g.col)
    assert_solve_parity(prgb, g, G2, P2, q2)
    with pytest.raises(prgb.PrError):
        P.set_shape(300, 4)
