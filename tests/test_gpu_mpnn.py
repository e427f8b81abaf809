"""The learned warm start on the GPU against its FP64 reference
(oracle/mpnn.py) and against the cold-start solver.

* forward: yhat of every SCC vertex and the loss agree with the reference
  evaluated with the same bfloat16-rounded weights (float32 sums on the GPU);
* backward: the GPU gradient agrees with the reference's analytic gradient,
  itself pinned by finite differences in test_oracle_mpnn.py;
* training with the library's kernels lowers the loss;
* a warm-started solve meets the same bounds as a cold one (residual,
  distance to the oracle's solution, closed forms in every kernel class),
  whatever the network guesses; a trained network needs fewer sweeps.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import mpnn as ref

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


def solved(g, tol=1e-12):
    q = oracle.partition(g.rowptr, g.col)
    R, _ = oracle.solve_cw(g.rowptr, g.col, q, C, g.u, tol)
    return q, R


def small_graph(seed=21):
    return gg.small_planted(seed=seed, n=6_000, n_scc=60, scc_vertices=4_500, n_dangling=500, layers=6,
                            target_edges=40_000)


def test_forward_matches_reference(prgb):
    g = small_graph()
    q, R = solved(g)
    G = prgb.graph(g.rowptr, g.col)
    P = prgb.partition(G)
    M = prgb.Mpnn(seed=5)
    theta = ref.bf16_round(M.get_params())
    y_gpu, loss_gpu = M.predict(P, C, g.u, R)
    y_gpu = y_gpu.cpu().numpy()
    rows, X, ip, isrc, y, mask = ref.features(g.rowptr, g.col, q, C, g.u, R)
    yhat, _ = ref.forward(theta.astype(np.float64), X, ip, isrc)
    assert np.max(np.abs(y_gpu[rows] - yhat)) <= 1e-3 * max(1.0, np.max(np.abs(yhat)))
    others = np.setdiff1d(np.arange(g.n), rows)
    assert np.all(y_gpu[others] == 0.0)
    loss_ref = ref.loss(theta.astype(np.float64), X, ip, isrc, y, mask)
    assert loss_gpu == pytest.approx(loss_ref, rel=1e-3)


def test_gradient_matches_reference(prgb):
    g = small_graph(seed=22)
    q, R = solved(g)
    G = prgb.graph(g.rowptr, g.col)
    P = prgb.partition(G)
    M = prgb.Mpnn(seed=6)
    theta = ref.bf16_round(M.get_params()).astype(np.float64)
    loss_gpu, grad_gpu = M.loss_grad(P, C, g.u, R)
    rows, X, ip, isrc, y, mask = ref.features(g.rowptr, g.col, q, C, g.u, R)
    loss_ref, grad_ref = ref.loss_and_grad(theta, X, ip, isrc, y, mask)
    assert loss_gpu == pytest.approx(loss_ref, rel=1e-3)
    o = 0
    for name, shape in ref.SHAPES:
        k = int(np.prod(shape))
        a, b = grad_gpu[o:o + k].astype(np.float64), grad_ref[o:o + k]
        assert np.linalg.norm(a - b) <= 2e-3 * np.linalg.norm(b) + 1e-6, name
        o += k
    # the gradient call leaves the weights alone
    assert np.array_equal(ref.bf16_round(M.get_params()), theta.astype(np.float32))


def test_params_roundtrip_and_invalid(prgb):
    M = prgb.Mpnn(seed=1)
    th = M.get_params()
    assert th.size == ref.N_PARAMS
    M.set_params(th * 0.5)
    assert np.array_equal(M.get_params(), (th * 0.5).astype(np.float32))
    with pytest.raises(prgb.PrError):
        M.set_params(th[:-1])
    assert np.array_equal(prgb.Mpnn(seed=1).get_params(), th)  # seeded


def train(prgb, M, graphs, epochs, lr=3e-3):
    losses = []
    for ep in range(epochs):
        tot = 0.0
        for P, g, R in graphs:
            tot += M.train_step(P, C, g.u, R, lr=lr)
        losses.append(tot / len(graphs))
    return losses


def deep_graphs(prgb, seeds, n=100_000, levels=20):
    out = []
    for s in seeds:
        g = gg.deep_dag(seed=s, n=n, levels=levels)
        G = prgb.graph(g.rowptr, g.col)
        P = prgb.partition(G)
        R = prgb.solve(P, C, g.u, 1e-12)  # the plain solver's solution (numpy in, numpy out)
        out.append((P, g, R, G))
    return out


@pytest.fixture(scope="module")
def trained(prgb):
    """Trained on plain-solver solutions of seeded deep-DAG graphs (n =
    100,000) with the library's kernels; returns (model, losses, held-out)."""
    data = deep_graphs(prgb, range(100000, 100006))
    M = prgb.Mpnn(seed=3)
    losses = train(prgb, M, [(P, g, R) for P, g, R, _ in data], epochs=60)
    held = deep_graphs(prgb, [200000, 200001])
    return M, losses, held


def test_training_lowers_the_loss(prgb, trained):
    M, losses, held = trained
    assert losses[-1] < 0.5 * losses[0]
    M0 = prgb.Mpnn(seed=3)
    for P, g, R, _ in held:
        _, l_trained = M.predict(P, C, g.u, R)
        _, l_init = M0.predict(P, C, g.u, R)
        assert l_trained < 0.5 * l_init


def check_warm(prgb, g, M, tol=1e-10, precision=0):
    import torch
    G = prgb.graph(g.rowptr, g.col)
    P = prgb.partition(G)
    q = oracle.partition(g.rowptr, g.col)
    u = torch.from_numpy(g.u).cuda()
    R, st = prgb.solve(P, C, u, tol, warm_start=M, with_stats=True, precision=precision)
    assert st["status"] == 0
    R = R.cpu().numpy()
    floor = 8 * 2.2e-16 * (g.u.sum() + 2 * R.sum())
    bound = (C * tol if precision == 0 else tol) * (1 + 1e-6) + floor
    assert prgb.residual_l1(G, C, u, torch.from_numpy(R).cuda()) <= bound
    assert oracle.residual_l1(g.rowptr, g.col, C, g.u, R) <= bound
    Ro, _ = oracle.solve_cw(g.rowptr, g.col, q, C, g.u, tol)
    assert np.abs(R - Ro).sum() <= 2 * tol / (1 - C) + 2 * floor / (1 - C)
    return R, st


def test_warm_start_bounds_with_untrained_network(prgb):
    """Whatever the network guesses, the solve meets the cold start's bounds
    (the plain series from the guess's residual decides)."""
    M = prgb.Mpnn(seed=11)
    for g in [small_graph(23), gg.web_like(seed=12, n=60_000, n_small=1_200, layers=12, giant_layer=4)]:
        check_warm(prgb, g, M)
        check_warm(prgb, g, M, precision=prgb.PREC_MIXED)


def test_cluster_class_warm(prgb):
    g = gg.small_planted(seed=33, n=40_000, n_scc=20, scc_vertices=30_000, n_dangling=4_000, layers=6,
                         target_edges=200_000)
    M = prgb.Mpnn(seed=12)
    check_warm(prgb, g, M)
    check_warm(prgb, g, M, precision=prgb.PREC_MIXED)


@pytest.mark.parametrize("k", [20, 200, 5_000, 50_000])
def test_warm_cycle_closed_form_every_class(prgb, k):
    import torch
    rp, col = gg.csr_from_edges(k, np.arange(k), (np.arange(k) + 1) % k)
    G = prgb.graph(rp, col)
    P = prgb.partition(G)
    u = np.full(k, 1.0 / k)
    M = prgb.Mpnn(seed=13)
    for prec in [prgb.PREC_FP64, prgb.PREC_MIXED]:
        R = prgb.solve(P, C, torch.from_numpy(u).cuda(), 1e-10, warm_start=M, precision=prec).cpu().numpy()
        assert np.abs(R - u / (1 - C)).sum() <= 2e-10 / (1 - C)


def test_trained_warm_start_needs_fewer_sweeps(prgb, trained):
    """Held-out graphs: the trained guess cuts the SCC sweeps (edge visits)
    and the result meets the same bounds.  Training sums its gradients with
    float atomics, so the model -- and the cut, about 10% of the visits --
    varies a little from run to run; at least 5% is asserted."""
    import torch
    M, _, held = trained
    for P, g, _, G in held:
        u = torch.from_numpy(g.u).cuda()
        Rc, sc = prgb.solve(P, C, u, 1e-10, with_stats=True)
        Rw, sw = prgb.solve(P, C, u, 1e-10, with_stats=True, warm_start=M)
        print(f"held-out n={g.n}: edge visits cold {sc['edge_visits']} warm {sw['edge_visits']}, "
              f"max sweeps cold {sc['iters_max']} warm {sw['iters_max']}")
        assert sw["edge_visits"] < 0.95 * sc["edge_visits"]
        assert prgb.residual_l1(G, C, u, Rw) <= C * 1e-10 * (1 + 1e-6)
        assert (Rw - Rc).abs().sum().item() <= 2e-10 / (1 - C)


def test_warm_start_invalid(prgb):
    import torch
    g = small_graph()
    G = prgb.graph(g.rowptr, g.col)
    P = prgb.partition(G)
    M = prgb.Mpnn(seed=1)
    u = torch.from_numpy(g.u).cuda()
    with pytest.raises(prgb.PrError) as e:
        prgb.solve(P, C, u, 1e-10, warm_start=M, replay_iters=np.ones(P.n_comp, np.int32))
    assert e.value.code == 1
