"""Mixed precision (FP32 SCC series with FP64 residual refinement for the
SCCs of the cluster class, 1,025-16,384 vertices; the others run the exact
fixed-point series as in FP64 mode) against the FP64 oracle.

The FP32 iterates differ from the FP64 ones, so there is no element-wise
1e-12 comparison.  What pins the result instead (the solution of
(I - cA^T)R = u is unique, and ||(I - cA^T)^-1||_1 <= 1/(1 - c)):
  * the FP64 L1 residual of R -- from the GPU's residual kernel and from the
    oracle's -- is within tol plus the FP64 rounding floor of forming it;
  * ||R - R_oracle||_1 <= 2 tol / (1 - c), R_oracle being the FP64 oracle's
    cold-start result (its own residual is at most c tol);
  * closed forms (uniform u on a cycle or a complete digraph: R = u/(1 - c))
    in every kernel class;
  * the largest element-wise relative error, reported and bounded loosely.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

C = 0.85


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


def floor64(u, R):
    # a few ulps of every term of u + cA^T(R/outdeg) - R
    return 8 * 2.2e-16 * (float(np.sum(u)) + 2 * float(np.sum(R)))


def check_mixed(prgb, g, tol=1e-10, max_rel_bound=1e-6):
    import torch
    G = prgb.graph(g.rowptr, g.col)
    P = prgb.partition(G)
    q = oracle.partition(g.rowptr, g.col)
    u = torch.from_numpy(g.u).cuda()
    R, st = prgb.solve(P, C, u, tol, precision=prgb.PREC_MIXED, with_stats=True)
    assert st["status"] == 0
    R = R.cpu().numpy()
    bound = tol + floor64(g.u, R)
    assert prgb.residual_l1(G, C, u, torch.from_numpy(R).cuda()) <= bound
    assert oracle.residual_l1(g.rowptr, g.col, C, g.u, R) <= bound
    Ro, _ = oracle.solve_cw(g.rowptr, g.col, q, C, g.u, tol)
    assert np.abs(R - Ro).sum() <= 2 * tol / (1 - C) + 2 * floor64(g.u, R) / (1 - C)
    rel = float(np.max(np.abs(R - Ro) / np.maximum(np.abs(Ro), 1e-300)))
    assert rel <= max_rel_bound
    sizes = np.bincount(q.comp, minlength=q.n_comp)
    ctype = np.zeros(q.n_comp, np.int64)
    ctype[q.comp] = q.type
    fp32 = (ctype == 1) & (sizes > 1024) & (sizes <= 16384)
    if np.any(fp32):
        # FP32 series refined by FP64 residual sweeps
        assert st["fp64_sweeps_max"] >= 1
        assert 0 < st["fp64_edge_visits"] < st["edge_visits"]
    else:
        # every SCC in the exact fixed-point series: no FP64 sweep
        assert st["fp64_sweeps_max"] == 0 and st["fp64_edge_visits"] == 0
    return R, st, rel


def test_small_planted_mixed(prgb):
    check_mixed(prgb, gg.small_planted(seed=1))


def test_web_like_reduced_mixed(prgb):
    g = gg.web_like(seed=12, n=60_000, n_small=1_200, layers=12, giant_layer=4)
    check_mixed(prgb, g)


def test_cluster_class_mixed(prgb):
    g = gg.small_planted(seed=33, n=40_000, n_scc=20, scc_vertices=30_000, n_dangling=4_000, layers=6,
                         target_edges=200_000)
    check_mixed(prgb, g)


def test_random_with_loops_mixed_tight_tol(prgb):
    rng = np.random.default_rng(2)
    n = 5000
    src = rng.integers(0, n, 3 * n)
    dst = rng.integers(0, n, 3 * n)
    dang = rng.random(n) < 0.2
    keep = ~dang[src]
    rp, col = gg.csr_from_edges(n, src[keep], dst[keep])
    u = rng.random(n)
    check_mixed(prgb, gg.Graph(n, rp, col, u / u.sum(), "random"), tol=1e-12)


def test_loose_tol_needs_one_residual(prgb):
    """With a budget far above the FP32 rounding of the sum (tol*|C|/n
    against ~1e-5 |R_C|), the first FP32 pass of each cluster-class SCC meets
    it and one FP64 residual confirms it."""
    g = gg.small_planted(seed=33, n=40_000, n_scc=20, scc_vertices=30_000, n_dangling=4_000, layers=6,
                         target_edges=200_000)
    _, st, _ = check_mixed(prgb, g, tol=1e-3, max_rel_bound=0.05)
    assert st["fp64_sweeps_max"] == 1


@pytest.mark.parametrize("k", [20, 200, 5_000, 50_000])
def test_cycle_closed_form_every_class(prgb, k):
    """Uniform u on a single cycle: R = u/(1 - c), in the warp, CTA, cluster
    and grid-wide classes."""
    import torch
    rp, col = gg.csr_from_edges(k, np.arange(k), (np.arange(k) + 1) % k)
    G = prgb.graph(rp, col)
    P = prgb.partition(G)
    u = np.full(k, 1.0 / k)
    tol = 1e-10
    R = prgb.solve(P, C, torch.from_numpy(u).cuda(), tol, precision=prgb.PREC_MIXED).cpu().numpy()
    exact = u / (1 - C)
    assert np.abs(R - exact).sum() <= 2 * tol / (1 - C)
    assert np.max(np.abs(R - exact) / exact) <= 1e-6


def test_complete_digraph_closed_form(prgb):
    import torch
    m = 100
    s, d = np.nonzero(~np.eye(m, dtype=bool))
    rp, col = gg.csr_from_edges(m, s, d)
    G = prgb.graph(rp, col)
    P = prgb.partition(G)
    u = np.full(m, 0.01)
    R = prgb.solve(P, C, torch.from_numpy(u).cuda(), 1e-12, precision=prgb.PREC_MIXED).cpu().numpy()
    assert np.abs(R - u / (1 - C)).sum() <= 2e-12 / (1 - C)


def test_web_like_full_size_mixed(prgb):
    """The benchmark workload (n = 1,000,000, ~8M edges)."""
    _, st, rel = check_mixed(prgb, gg.web_like())
    print(f"web_like mixed: sweeps max {st['iters_max']}, FP64 sweeps max {st['fp64_sweeps_max']}, "
          f"FP64 edge share {st['fp64_edge_visits'] / st['edge_visits']:.3f}, max-rel vs oracle {rel:.2e}")


def test_mixed_deterministic(prgb):
    import torch
    g = gg.web_like(seed=15, n=30_000, n_small=600, layers=8, giant_layer=3)
    G = prgb.graph(g.rowptr, g.col)
    P = prgb.partition(G)
    u = torch.from_numpy(g.u).cuda()
    a = prgb.solve(P, C, u, 1e-10, precision=prgb.PREC_MIXED)
    b = prgb.solve(P, C, u, 1e-10, precision=prgb.PREC_MIXED)
    assert torch.equal(a, b)


def test_mixed_invalid_and_noconv(prgb):
    import torch
    g = gg.small_planted(seed=1)
    G = prgb.graph(g.rowptr, g.col)
    P = prgb.partition(G)
    u = torch.from_numpy(g.u).cuda()
    with pytest.raises(prgb.PrError) as e:
        prgb.solve(P, C, u, 1e-10, norm=prgb.NORM_LINF, precision=prgb.PREC_MIXED)
    assert e.value.code == 1
    with pytest.raises(prgb.PrError) as e:
        prgb.solve(P, C, u, 1e-10, replay_iters=np.ones(P.n_comp, np.int32), precision=prgb.PREC_MIXED)
    assert e.value.code == 1
    with pytest.raises(prgb.PrError) as e:
        prgb.solve(P, C, u, 1e-10, precision=7)
    assert e.value.code == 1
    R, st = prgb.solve(P, C, u, 1e-10, max_iter=3, precision=prgb.PREC_MIXED, with_stats=True,
                       allow_noconv=True)
    assert st["status"] == 4
    assert torch.isfinite(R).all()
    # the context is still usable
    R = prgb.solve(P, C, u, 1e-10, precision=prgb.PREC_MIXED)
    assert torch.isfinite(R).all()
