"""Pins for the oracle's PageRank solves (Sec. 3.1 Def. 3.4-3.5, Sec. 4.3-4.4).

Closed forms (chain, cycle, complete digraph, out-star), exact iteration
counts of a leak-free SCC, the independent dense solve by numpy, the
eigenvector definition R(1) of Def. 3.4 rescaled by Def. 3.5, mass
conservation of the linear system, monotonicity and the tail bound of
Sec. 4.4.
"""
import math

import numpy as np
import pytest

import graphgen as gg
import oracle

C = 0.85


def dense_system(rp, col, c):
    """(I - cA^T) with A_ij = 1/outdeg(i), loops ignored (numpy, independent)."""
    n = len(rp) - 1
    M = np.eye(n)
    for i in range(n):
        row = [int(j) for j in col[rp[i]:rp[i + 1]] if j != i]
        for j in row:
            M[j, i] -= c / len(row)
    return M


def solve_all(rp, col, u, tol, **kw):
    p = oracle.partition(rp, col)
    R, its = oracle.solve_cw(rp, col, p, C, u, tol, **kw)
    return p, R, its


# ---------------------------------------------------------------- closed forms

def test_chain_closed_form():
    k = 40
    rp, col = gg.csr_from_edges(k, np.arange(k - 1), np.arange(1, k))
    u = np.ones(k)
    p, R, _ = solve_all(rp, col, u, 1e-3)  # CAC: exact whatever the tolerance
    i = np.arange(1, k + 1)
    assert p.n_comp == 1 and p.type[0] == 0
    np.testing.assert_allclose(R, (1 - C ** i) / (1 - C), rtol=1e-14)


@pytest.mark.parametrize("k", [2, 3, 7, 50])
def test_cycle_closed_form(k):
    rng = np.random.default_rng(k)
    rp, col = gg.csr_from_edges(k, np.arange(k), (np.arange(k) + 1) % k)
    u = rng.random(k)
    p, R, _ = solve_all(rp, col, u, 1e-15)
    want = np.array([sum(C ** t * u[(i - t) % k] for t in range(k)) for i in range(k)]) / (1 - C ** k)
    assert p.n_comp == 1 and p.type[0] == 1
    np.testing.assert_allclose(R, want, rtol=1e-12)


@pytest.mark.parametrize("m", [2, 5, 30])
def test_complete_digraph(m):
    a, b = np.nonzero(~np.eye(m, dtype=bool))
    rp, col = gg.csr_from_edges(m, a, b)
    u = np.full(m, 0.3)
    _, R, _ = solve_all(rp, col, u, 1e-15)
    np.testing.assert_allclose(R, u / (1 - C), rtol=1e-12)


def test_out_star():
    k = 9
    rp, col = gg.csr_from_edges(k + 1, np.zeros(k, int), np.arange(1, k + 1))
    rng = np.random.default_rng(3)
    u = rng.random(k + 1)
    p, R, _ = solve_all(rp, col, u, 1e-2)
    assert p.n_comp == 1  # centre merges with its dangling leaves
    assert R[0] == u[0]
    np.testing.assert_allclose(R[1:], u[1:] + C * u[0] / k, rtol=1e-15)


def test_leak_free_scc_iteration_count():
    """A sink SCC is stochastic: ||P_k||_1 = c^k ||W||_1 exactly (Sec. 5.2)."""
    k = 12
    rp, col = gg.csr_from_edges(k, np.arange(k), (np.arange(k) + 1) % k)
    u = np.full(k, 1.0 / k)
    for tol in [3e-4, 1e-7, 2e-10]:
        _, _, its = solve_all(rp, col, u, tol)
        # budget tau = tol * |C| / |V| = tol here; smallest k with c^k <= tol
        assert its[0] == math.ceil(math.log(tol) / math.log(C))
        _, kg = oracle.solve_global(rp, col, C, u, tol)
        assert kg == its[0]


def test_linf_rule_on_cycle():
    """The paper's rule: iterate while max(P) >= tol."""
    k = 10
    rp, col = gg.csr_from_edges(k, np.arange(k), (np.arange(k) + 1) % k)
    u = np.full(k, 1.0)
    tol = 1e-6
    _, kg = oracle.solve_global(rp, col, C, u, tol, norm=oracle.NORM_LINF)
    assert kg == math.floor(math.log(tol) / math.log(C)) + 1


# ----------------------------------------------------- against a dense solve

def _random_graph_with_dangling(n, seed):
    rng = np.random.default_rng(seed)
    m = rng.random((n, n)) < rng.uniform(1.5, 4.0) / n
    dangle = rng.random(n) < rng.uniform(0.1, 0.3)
    m[dangle, :] = False
    np.fill_diagonal(m, rng.random(n) < 0.05)
    a, b = np.nonzero(m)
    rp, col = gg.csr_from_edges(n, a, b)
    return rp, col, rng.random(n)


@pytest.mark.parametrize("seed", range(8))
def test_dense_oracle_matches_numpy(seed):
    n = [5, 20, 60, 120, 200, 300, 17, 250][seed]
    rp, col, u = _random_graph_with_dangling(n, seed)
    R = oracle.dense_solve(rp, col, C, u)
    Rn = np.linalg.solve(dense_system(rp, col, C), u)
    np.testing.assert_allclose(R, Rn, rtol=1e-12, atol=0)


@pytest.mark.parametrize("seed", range(8))
def test_componentwise_converges_to_dense(seed):
    n = [30, 80, 150, 300, 300, 220, 64, 128][seed]
    rp, col, u = _random_graph_with_dangling(n, 100 + seed)
    Rn = np.linalg.solve(dense_system(rp, col, C), u)
    _, R, _ = solve_all(rp, col, u, 1e-15)
    np.testing.assert_allclose(R, Rn, rtol=1e-12)
    Rg, _ = oracle.solve_global(rp, col, C, u, 1e-15)
    np.testing.assert_allclose(Rg, Rn, rtol=1e-12)


def test_cac_and_singletons_exact_at_loose_tolerance():
    """Methods (i)-(ii) of Sec. 4.3 do not depend on the tolerance."""
    rng = np.random.default_rng(7)
    n = 250
    a = rng.integers(0, n, 700)
    b = rng.integers(0, n, 700)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    keep = lo != hi
    rp, col = gg.csr_from_edges(n, lo[keep], hi[keep])  # a DAG: no SCC
    u = rng.random(n)
    p, R, _ = solve_all(rp, col, u, 1.0)
    assert p.type.max() == 0
    Rn = np.linalg.solve(dense_system(rp, col, C), u)
    np.testing.assert_allclose(R, Rn, rtol=1e-13)


def test_small_scc_lu_is_exact():
    g = gg.small_planted(seed=4, n=600, n_scc=12, scc_vertices=480, n_dangling=60,
                         layers=5, target_edges=3000)
    Rn = np.linalg.solve(dense_system(g.rowptr, g.col, C), g.u)
    _, R, _ = solve_all(g.rowptr, g.col, g.u, 1.0, lu_threshold=10_000)
    np.testing.assert_allclose(R, Rn, rtol=1e-12)


def test_def35_eigenvector_rescaling():
    """Def. 3.4 R(1) (eigenvector of M) rescaled by Def. 3.5 equals R(3)."""
    n = 80
    rp, col, W = _random_graph_with_dangling(n, 11)
    A = np.zeros((n, n))
    for i in range(n):
        row = [int(j) for j in col[rp[i]:rp[i + 1]] if j != i]
        for j in row:
            A[i, j] = 1.0 / len(row)
    g = (A.sum(axis=1) == 0).astype(float)
    w = W / W.sum()
    M = C * (A + np.outer(g, w)).T + (1 - C) * np.outer(w, np.ones(n))
    vals, vecs = np.linalg.eig(M)
    r1 = np.real(vecs[:, np.argmin(np.abs(vals - 1.0))])
    r1 = r1 / r1.sum()
    d = 1.0 - np.sum(C * A.T @ r1)
    r3 = r1 * W.sum() / d
    _, R, _ = solve_all(rp, col, W, 1e-15)
    np.testing.assert_allclose(R, r3, rtol=1e-10)


# ------------------------------------------------- identities and bounds

def _signed_residual(rp, col, c, u, R):
    n = len(rp) - 1
    r = u - R.copy()
    for i in range(n):
        row = [int(j) for j in col[rp[i]:rp[i + 1]] if j != i]
        for j in row:
            r[j] += c * R[i] / len(row)
    return r


def test_residual_function_closed_form():
    g = gg.small_planted(seed=2)
    outdeg = np.array([np.count_nonzero(g.col[g.rowptr[i]:g.rowptr[i + 1]] != i) for i in range(g.n)])
    # R = u: r = c A^T (u/outdeg), ||r||_1 = c * sum of u over non-dangling vertices
    res = oracle.residual_l1(g.rowptr, g.col, C, g.u, g.u)
    assert res == pytest.approx(C * g.u[outdeg > 0].sum(), rel=1e-13)


def test_mass_conservation_and_budget():
    """With r = u + cA^T(R/outdeg) - R, summing over vertices gives
    (1-c)|R| + c*sum_dangling R = |u| - sum r (column sums of A^T are 1 or 0)."""
    g = gg.small_planted(seed=3)
    for tol in [1e-4, 1e-8, 1e-10]:
        _, R, _ = solve_all(g.rowptr, g.col, g.u, tol)
        r = _signed_residual(g.rowptr, g.col, C, g.u, R)
        outdeg = np.diff(g.rowptr)
        lhs = (1 - C) * R.sum() + C * R[outdeg == 0].sum()
        assert lhs == pytest.approx(g.u.sum() - r.sum(), rel=1e-13)
        # the size-proportional L1 budget bounds the global residual by c*tol
        assert np.abs(r).sum() <= C * tol * (1 + 1e-9)
        assert oracle.residual_l1(g.rowptr, g.col, C, g.u, R) == pytest.approx(np.abs(r).sum(), rel=1e-6, abs=1e-14)


def test_monotone_and_tail_bound():
    """R >= W >= u (series of non-negative terms) and the Sec. 4.4 tail bound."""
    rp, col, u = _random_graph_with_dangling(200, 21)
    Rn = np.linalg.solve(dense_system(rp, col, C), u)
    for tol in [1e-3, 1e-6, 1e-9]:
        Rg, _ = oracle.solve_global(rp, col, C, u, tol)
        assert np.all(Rg >= u)
        assert np.all(Rn - Rg >= -1e-15)
        # ||R_true - R_K||_1 <= c ||p_K||_1 / (1-c) <= c tol / (1-c)
        assert np.abs(Rn - Rg).sum() <= C * tol / (1 - C) * (1 + 1e-9)
        _, Rc, _ = solve_all(rp, col, u, tol)
        assert np.all(Rc >= u)
        assert np.abs(Rn - Rc).sum() <= 2 * tol / (1 - C)


def test_replay_reproduces_iterations():
    g = gg.small_planted(seed=6)
    p, R, its = solve_all(g.rowptr, g.col, g.u, 1e-10)
    R2, its2 = oracle.solve_cw(g.rowptr, g.col, p, C, g.u, 1e-10, replay_iters=its)
    assert np.array_equal(R, R2) and np.array_equal(its, its2)
    # one more iteration everywhere moves R up, by at most the tail bound
    R3, _ = oracle.solve_cw(g.rowptr, g.col, p, C, g.u, 1e-10, replay_iters=its + (its > 0))
    assert np.all(R3 >= R) and np.abs(R3 - R).sum() <= 1e-10


def test_componentwise_agrees_with_global():
    """Both methods solve the same system; at tol 1e-10 (L1) they agree
    within the sum of their tail bounds."""
    g = gg.small_planted(seed=1)
    p, R, its = solve_all(g.rowptr, g.col, g.u, 1e-10)
    Rg, kg = oracle.solve_global(g.rowptr, g.col, C, g.u, 1e-10)
    assert np.abs(R - Rg).sum() <= 2 * 1e-10 / (1 - C)
    ctype = np.zeros(p.n_comp, np.int64)
    ctype[p.comp] = p.type
    assert its[ctype == 0].max(initial=0) == 0 and its[ctype == 1].min() >= 1


def test_invalid_arguments():
    rp, col = gg.csr_from_edges(3, [0, 1], [1, 2])
    p = oracle.partition(rp, col)
    with pytest.raises(oracle.OracleError):
        oracle.solve_cw(rp, col, p, 1.0, np.ones(3), 1e-10)
    with pytest.raises(oracle.OracleError):
        oracle.solve_global(rp, col, 0.85, np.ones(3), 0.0)
    with pytest.raises(oracle.OracleError):
        oracle.partition(np.array([0, 1, 2], np.int32), np.array([1, 5], np.int32))
