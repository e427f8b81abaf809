"""Per-level device times of a solve (pr_solve_stats.level_ms, CUDA events
recorded between the levels of the captured level loop)."""
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu


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


def test_level_times_cover_the_solve(prgb):
    import torch
    g = gg.deep_dag(seed=7, n=200_000, levels=40)
    G = prgb.graph(torch.from_numpy(g.rowptr).cuda(), torch.from_numpy(g.col).cuda())
    P = prgb.partition(G)
    u = torch.from_numpy(g.u).cuda()
    prgb.solve(P, 0.85, u, 1e-10, level_times=True)  # captures the timed graph
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    R, st = prgb.solve(P, 0.85, u, 1e-10, with_stats=True, level_times=True)
    b.record()
    torch.cuda.synchronize()
    lv = st["level_ms"]
    assert lv.shape == (P.n_levels,) and P.n_levels == 40
    assert (lv > 0).all()
    # the levels run back to back inside the call
    assert lv.sum() <= a.elapsed_time(b) * 1.001
    assert lv.sum() >= 0.5 * a.elapsed_time(b)
    # without level timing nothing is reported
    R2, st2 = prgb.solve(P, 0.85, u, 1e-10, with_stats=True)
    assert "level_ms" not in st2
    assert torch.equal(R, R2)
    R3, st3 = prgb.solve(P, 0.85, u, 1e-10, with_stats=True, timing=True)
    assert "level_ms" not in st3 and st3["kernel_ms"] >= 0
    assert torch.equal(R, R3)


def test_partition_phase_times(prgb):
    """PR_PARTITION_TIMING: phase times between CUDA events that add up to
    the call, wave counts of the frontier kernels, and the same partition as
    without the flag."""
    import torch
    g = gg.web_like(seed=12, n=60_000, n_small=1_200, layers=12, giant_layer=4)
    G = prgb.graph(torch.from_numpy(g.rowptr).cuda(), torch.from_numpy(g.col).cuda())
    P0 = prgb.partition(G)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    P1 = prgb.partition(G, timing=True)
    b.record()
    torch.cuda.synchronize()
    t = P1.timing()
    phases = [t[k] for k in ("trim_ms", "giant_ms", "colour_ms", "levels_ms", "layout_ms")]
    assert all(x >= 0 for x in phases) and t["total_ms"] > 0
    assert sum(phases) <= t["total_ms"] * 1.001 + 1e-3
    assert t["total_ms"] <= a.elapsed_time(b) * 1.001 + 1e-3
    assert t["colour_rounds"] >= 1
    w = t["waves"]
    assert w["trim"]["grid"] + w["trim"]["block"] >= 1
    assert w["reach"]["grid"] + w["reach"]["block"] >= 1  # the giant's forward-backward search
    assert w["kahn"]["grid"] + w["kahn"]["block"] >= 1
    for x, y in zip(P0.query(), P1.query()):
        assert torch.equal(x, y)
    with pytest.raises(prgb.PrError) as e:
        P0.timing()
    assert e.value.code == 1


def test_counts_off_reads_back_only_timing(prgb):
    """counts_off: the solve reports its kernel times (and the grid-wide
    components' bytes) without the per-component counts, and R is the same."""
    import torch
    g = gg.web_like(seed=12, n=60_000, n_small=1_200, layers=12, giant_layer=4)
    G = prgb.graph(torch.from_numpy(g.rowptr).cuda(), torch.from_numpy(g.col).cuda())
    P = prgb.partition(G)
    u = torch.from_numpy(g.u).cuda()
    R1, s1 = prgb.solve(P, 0.85, u, 1e-10, with_stats=True, timing=True)
    R2, s2 = prgb.solve(P, 0.85, u, 1e-10, with_stats=True, timing=True, counts=False)
    assert torch.equal(R1, R2)
    assert "comp_iters" in s1 and "comp_iters" not in s2
    assert s2["iters_max"] == 0 and s2["edge_visits"] == 0
    assert s1["kernel_launches"] == s2["kernel_launches"] >= 1
    assert s2["kernel_bytes"] == s1["kernel_bytes"] > 0 and s2["kernel_ms"] > 0
