"""Host-side helpers of bench.py that need no GPU: the sweep statistics of
the Sec. 5.2 comparison, on the oracle's partition and solve."""
import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
bench = pytest.importorskip("bench")


def test_sweep_stats_matches_a_direct_count():
    g = gg.small_planted(seed=4)
    q = oracle.partition(g.rowptr, g.col)
    _, its = oracle.solve_cw(g.rowptr, g.col, q, 0.85, g.u, 1e-10)
    _, git = oracle.solve_global(g.rowptr, g.col, 0.85, g.u, 1e-10)
    out = bench.sweep_stats(torch.from_numpy(q.comp), torch.from_numpy(q.type), torch.from_numpy(g.rowptr),
                            torch.from_numpy(g.col), its, git)
    # direct count, one edge at a time
    src = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    scc = np.zeros(q.n_comp, bool)
    scc[q.comp[q.type == 1]] = True
    w = np.zeros(q.n_comp)
    for a, b in zip(src, g.col):
        if a != b and q.comp[a] == q.comp[b]:
            w[q.comp[a]] += 1
    assert out["scc_components"] == int(scc.sum())
    assert out["min"] == its[scc].min() and out["max"] == its[scc].max()
    assert out["scc_internal_edges"] == int(w[scc].sum())
    assert out["edge_weighted_mean"] == pytest.approx((its[scc] * w[scc]).sum() / w[scc].sum(), rel=1e-12)
    assert out["global_sweeps"] == git
    assert out["min"] <= out["median"] <= out["max"]
