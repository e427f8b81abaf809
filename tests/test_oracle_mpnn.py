"""Pins of the warm-start network's reference (oracle/mpnn.py), independent
of the CUDA path: finite differences for the backward pass, hand-set
weights with closed-form outputs for the forward pass and the aggregation
direction, exact features on a cycle, and bfloat16 rounding cases."""
import numpy as np

import graphgen as gg
import oracle
from oracle import mpnn

C = 0.85


def small_case(seed=3):
    g = gg.small_planted(seed=seed, n=600, n_scc=12, scc_vertices=400, n_dangling=60, layers=4,
                         target_edges=3_000)
    q = oracle.partition(g.rowptr, g.col)
    R, _ = oracle.solve_cw(g.rowptr, g.col, q, C, g.u, 1e-13)
    return g, q, R


def test_gradient_matches_central_differences():
    g, q, R = small_case()
    rows, X, ip, isrc, y, mask = mpnn.features(g.rowptr, g.col, q, C, g.u, R)
    assert rows.size > 100
    theta = mpnn.init_params(7).astype(np.float64)
    L, grad = mpnn.loss_and_grad(theta, X, ip, isrc, y, mask)
    rng = np.random.default_rng(0)
    idx = rng.choice(theta.size, 60, replace=False)
    # include every parameter block
    starts = np.cumsum([0] + [int(np.prod(s)) for _, s in mpnn.SHAPES])[:-1]
    idx = np.unique(np.concatenate([idx, starts]))
    h = 1e-6
    for i in idx:
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mpnn.loss(tp, X, ip, isrc, y, mask) - mpnn.loss(tm, X, ip, isrc, y, mask)) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (i, fd, grad[i])


def _set(**kw):
    d = {name: np.zeros(shape) for name, shape in mpnn.SHAPES}
    d.update(kw)
    return mpnn.pack(d)


def test_hand_set_weights_forward():
    # 0 -> 1 -> 2 -> 0 and 0 -> 2: one SCC; internal in-degrees 1, 1, 2
    rp, col = gg.csr_from_edges(3, [0, 1, 2, 0], [1, 2, 0, 2])
    q = oracle.partition(rp, col)
    u = np.full(3, 1 / 3)
    R, _ = oracle.solve_cw(rp, col, q, C, u, 1e-14)
    rows, X, ip, isrc, y, mask = mpnn.features(rp, col, q, C, u, R)
    din = np.array([1, 1, 2])
    assert np.allclose(X[:, 0], np.log1p(din))
    # yhat = x0 of the vertex itself
    A1 = np.zeros((64, 8))
    A1[0, 0] = 1.0
    A2 = np.zeros((64, 64))
    A2[0, 0] = 1.0
    v = np.zeros(64)
    v[0] = 1.0
    yhat, _ = mpnn.forward(_set(A1=A1, A2=A2, v=v), X, ip, isrc)
    assert np.allclose(yhat, np.log1p(din))
    # yhat = mean of x0 over the in-neighbours, through layer 1's aggregation:
    # in(0) = {2}, in(1) = {0}, in(2) = {0, 1}
    B1 = np.zeros((64, 8))
    B1[0, 0] = 1.0
    yhat, _ = mpnn.forward(_set(B1=B1, A2=A2, v=v), X, ip, isrc)
    assert np.allclose(yhat, [np.log1p(2), np.log1p(1), np.log1p(1)])
    # ... and through layer 2's aggregation
    B2 = np.zeros((64, 64))
    B2[0, 0] = 1.0
    yhat, _ = mpnn.forward(_set(A1=A1, B2=B2, v=v, b3=np.array([0.5])), X, ip, isrc)
    assert np.allclose(yhat, 0.5 + np.array([np.log1p(2), np.log1p(1), np.log1p(1)]))
    # both aggregations: two hops, mean over in(i) of the mean over in(j)
    l2, l3 = np.log(2), np.log(3)
    yhat, _ = mpnn.forward(_set(B1=B1, B2=B2, v=v), X, ip, isrc)
    assert np.allclose(yhat, [l2, l3, (l3 + l2) / 2])
    # relu: a negative pre-activation contributes nothing
    yhat, _ = mpnn.forward(_set(A1=-A1, A2=A2, v=v, b3=np.array([2.0])), X, ip, isrc)
    assert np.allclose(yhat, 2.0)


def test_features_on_a_cycle():
    k = 10
    rp, col = gg.csr_from_edges(k, np.arange(k), (np.arange(k) + 1) % k)
    q = oracle.partition(rp, col)
    u = np.full(k, 1.0 / k)
    R = u / (1 - C)
    rows, X, ip, isrc, y, mask = mpnn.features(rp, col, q, C, u, R)
    assert np.array_equal(rows, np.arange(k))
    # in-degree 1, out-degree 1, |C| = k, every out-edge internal, no
    # external in- or out-edge
    expect = np.array([np.log(2), np.log(2), np.log(k), 1.0, 0.0, 0.0, 1, 0])
    assert np.allclose(X, expect[None, :])
    # R = u / (1 - c) and W = u: the amplification is c / (1 - c)
    assert np.allclose(y, np.log(C / (1 - C)))
    assert mask.all()
    # ... and the guess built from it is the solution itself
    assert np.allclose(mpnn.guess(y, u, np.full(k, u.mean())), R)
    # every vertex's in-neighbour is its predecessor on the cycle
    assert np.array_equal(isrc, (np.arange(k) - 1) % k)


def test_target_amplification_sums_to_the_internal_mass():
    """sum_i b_i mean_C(W) = sum_i (R_i - W_i) = ||R_C||_1 - ||W_C||_1 per
    component, and the external in-degree and internal out-degree features
    count what they say (a 2-cycle fed by a source, with a leaving edge)."""
    # 0 -> 1, 1 -> 2, 2 -> 1, 2 -> 3: SCC {1, 2}; 0 and 3 are 1-vertex components
    rp, col = gg.csr_from_edges(4, [0, 1, 2, 2], [1, 2, 1, 3])
    q = oracle.partition(rp, col)
    u = np.array([0.4, 0.1, 0.3, 0.2])
    R, _ = oracle.solve_cw(rp, col, q, C, u, 1e-15)
    rows, X, ip, isrc, y, mask = mpnn.features(rp, col, q, C, u, R)
    assert np.array_equal(rows, [1, 2])
    assert np.allclose(X[:, 3], [1.0, 0.5])           # 1 -> 2 internal; 2 -> 1 of 2 out-edges
    assert np.allclose(X[:, 4], np.log1p([1.0, 0.0]))  # 0 -> 1 enters from outside
    assert np.allclose(X[:, 5], np.log1p([0.0, 1.0]))  # 2 -> 3 leaves
    W = u[rows].copy()
    W[0] += C * R[0]                                   # inflow of vertex 1 from vertex 0
    mw = W.mean()
    b = np.exp(y)
    assert np.isclose((b * mw).sum(), (R[rows] - W).sum())
    assert np.allclose(mpnn.guess(y, W, np.full(2, mw)), R[rows])


def test_bf16_rounding_cases():
    one = np.float32(1.0)
    ulp = np.float32(2.0 ** -7)
    cases = [
        (1.0, 1.0),
        (1.0 + 2.0 ** -8, 1.0),                 # halfway, ties to even (down)
        (1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -6),  # halfway, ties to even (up)
        (1.0 + 2.0 ** -8 + 2.0 ** -20, 1.0 + 2.0 ** -7),
        (-3.0, -3.0),
        (0.0, 0.0),
    ]
    for a, b in cases:
        assert mpnn.bf16_round(np.array([a], np.float32))[0] == np.float32(b), (a, b)
    assert one + ulp == np.float32(1.0078125)
