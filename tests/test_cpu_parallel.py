"""The multi-core CPU baseline (cpu_parallel/) against the oracle: the same
componentwise step (Sec. 4.3) and global series (Sec. 4.3.2), so the same
bounds -- residual, distance to the oracle's solution, closed forms -- for
one and several threads, with large components solved one at a time by all
threads or one component per thread."""
import numpy as np
import pytest

import graphgen as gg
import oracle

cp = pytest.importorskip("cpu_parallel")
if not cp.available():
    pytest.skip("gcc with OpenMP is not available", allow_module_level=True)

C = 0.85
TOL = 1e-10


def bounds(g, R, tol, cw=True):
    floor = 8 * 2.2e-16 * (g.u.sum() + 2 * R.sum())
    res = oracle.residual_l1(g.rowptr, g.col, C, g.u, R)
    assert res <= (C * tol if cw else tol) * (1 + 1e-6) + floor


@pytest.mark.parametrize("make", [
    lambda: gg.small_planted(seed=2),
    lambda: gg.web_like(seed=12, n=60_000, n_small=1_200, layers=12, giant_layer=4),
])
def test_matches_oracle(make):
    g = make()
    q = oracle.partition(g.rowptr, g.col)
    plan = cp.Plan(g.rowptr, g.col, q.comp, q.type, q.level)
    Ro, its = oracle.solve_cw(g.rowptr, g.col, q, C, g.u, TOL)
    Rg, git = oracle.solve_global(g.rowptr, g.col, C, g.u, TOL)
    for threads in (1, 4):
        for big in (16_384, 64):  # large components by all threads, or one per thread
            R, it = plan.solve_cw(C, g.u, TOL, threads=threads, big=big)
            bounds(g, R, TOL)
            assert np.abs(R - Ro).sum() <= 1e-12 * Ro.sum()
            assert abs(it - int(its.max())) <= 1  # same stopping rule, sums in another order
        R2, it2 = plan.solve_global(C, g.u, TOL, threads=threads)
        bounds(g, R2, TOL, cw=False)
        assert np.abs(R2 - Rg).sum() <= 1e-12 * Rg.sum()
        assert abs(it2 - git) <= 1


def test_closed_forms():
    # cycle: R = u / (1 - c); chain 0 -> 1 -> ... : R_i = (1 - c^(i+1)) / (1 - c) / n
    k = 500
    rp, col = gg.csr_from_edges(k, np.arange(k), (np.arange(k) + 1) % k)
    q = oracle.partition(rp, col)
    u = np.full(k, 1.0 / k)
    R, _ = cp.Plan(rp, col, q.comp, q.type, q.level).solve_cw(C, u, 1e-12, threads=4, big=100)
    assert np.abs(R - u / (1 - C)).sum() <= 2e-12 / (1 - C)
    rp, col = gg.csr_from_edges(k, np.arange(k - 1), np.arange(1, k))
    q = oracle.partition(rp, col)
    R, _ = cp.Plan(rp, col, q.comp, q.type, q.level).solve_cw(C, u, 1e-12, threads=4)
    expect = (1 - C ** (np.arange(k) + 1)) / (1 - C) / k
    assert np.allclose(R, expect, rtol=1e-13, atol=0)


def test_invalid_arguments():
    g = gg.small_planted(seed=3)
    q = oracle.partition(g.rowptr, g.col)
    plan = cp.Plan(g.rowptr, g.col, q.comp, q.type, q.level)
    for c in (0.0, 1.0):
        with pytest.raises(cp.CpuParallelError):
            plan.solve_cw(c, g.u, TOL)
        with pytest.raises(cp.CpuParallelError):
            plan.solve_global(c, g.u, TOL)
    with pytest.raises(cp.CpuParallelError):
        cp.Plan(g.rowptr, g.col, np.zeros(g.n, np.int32), np.zeros(g.n, np.uint8), np.zeros(g.n, np.int32))
