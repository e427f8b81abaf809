"""A partition written to a file and read back (pr_partition_save /
pr_partition_load): the loaded partition must equal the one the component
search builds -- the same ids, types and levels (checked against the oracle
too) and bit-identical solves -- and a file that does not belong to the
graph, or is damaged, must be refused with PR_EINVAL."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

C = 0.85
HEADER = 64  # bytes before the per-vertex arrays


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


def _round_trip(prgb, rp, col, path, u, tol=1e-10):
    import torch
    G = prgb.graph(rp, col)
    P = prgb.partition(G)
    P.save(path)
    n = len(rp) - 1
    assert path.stat().st_size == HEADER + 13 * n
    L = prgb.load_partition(G, path)
    assert (L.n_comp, L.n_levels, L.n_scc, L.n_scc_vertices) == (P.n_comp, P.n_levels, P.n_scc,
                                                                  P.n_scc_vertices)
    for a, b in zip(P.query(), L.query()):
        assert torch.equal(a, b)
    if n:
        q = oracle.partition(rp, col)
        comp, typ, lev = (x.cpu().numpy() for x in L.query())
        assert np.array_equal(comp, q.comp)
        assert np.array_equal(typ, q.type)
        assert np.array_equal(lev, q.level)
        ud = torch.from_numpy(u).cuda()
        Rp, sp = prgb.solve(P, C, ud, tol, with_stats=True)
        Rl, sl = prgb.solve(L, C, ud, tol, with_stats=True)
        assert torch.equal(Rp, Rl)
        assert np.array_equal(sp["comp_iters"], sl["comp_iters"])
    return G, P, L


@pytest.mark.parametrize("name", ["web_like", "deep_dag", "planted"])
def test_round_trip(prgb, tmp_path, name):
    """Graphs with a grid-wide SCC, with deep CAC chains (many sub-level
    waves), and with many small SCCs."""
    if name == "web_like":
        g = gg.web_like(seed=12, n=60_000, n_small=1_200, layers=12, giant_layer=4)
    elif name == "deep_dag":
        g = gg.deep_dag(seed=5, n=40_000, levels=40, scc_per_level=(5, 10))
    else:
        g = gg.small_planted(seed=3)
    _round_trip(prgb, g.rowptr, g.col, tmp_path / "p.bin", g.u)


def test_round_trip_degenerate(prgb, tmp_path):
    """No vertex; one vertex with a self-loop; all vertices dangling."""
    cases = [(np.zeros(1, np.int32), np.zeros(0, np.int32)),
             (np.array([0, 1], np.int32), np.array([0], np.int32)),
             (np.zeros(1001, np.int32), np.zeros(0, np.int32))]
    for i, (rp, col) in enumerate(cases):
        n = len(rp) - 1
        _round_trip(prgb, rp, col, tmp_path / f"d{i}.bin", np.full(n, 1.0 / max(n, 1)))


def _load_status(prgb, G, path):
    with pytest.raises(prgb.PrError) as e:
        prgb.load_partition(G, path)
    return e.value.name


def test_refuses_other_graphs_and_damage(prgb, tmp_path):
    g = gg.small_planted(seed=4)
    n = g.n
    path = tmp_path / "p.bin"
    G, P, L = _round_trip(prgb, g.rowptr, g.col, path, g.u)
    good = path.read_bytes()
    # the same n and edge count, one edge moved to another target
    rp, col = g.rowptr.copy(), g.col.copy()
    v = int(np.argmax(np.diff(rp) > 0))
    row = set(col[rp[v]:rp[v + 1]].tolist())
    col[rp[v]] = next(w for w in range(n) if w != v and w not in row)
    order = np.argsort(col[rp[v]:rp[v + 1]], kind="stable")
    col[rp[v]:rp[v + 1]] = col[rp[v]:rp[v + 1]][order]
    assert _load_status(prgb, prgb.graph(rp, col), path) == "PR_EINVAL"
    # another vertex count
    rp2 = np.concatenate([g.rowptr, g.rowptr[-1:]])
    assert _load_status(prgb, prgb.graph(rp2, g.col), path) == "PR_EINVAL"
    # damaged files: the magic, a truncated file, a trailing byte, a count
    # (the header's counts sit at bytes 48, 52 and 56; the largest wave made
    # larger passes every range check, so only the digest refuses it); then
    # one level changed to another level in range (the digest refuses it)
    # and out of range both ways; a missing file
    bad = tmp_path / "bad.bin"
    mw = np.frombuffer(good, np.int32, 1, 56)[0]
    grown = good[:56] + np.int32(mw + 1).tobytes() + good[60:]
    for data in (b"XRGB" + good[4:], good[:-1], good + b"\0", grown):
        bad.write_bytes(data)
        assert _load_status(prgb, G, bad) == "PR_EINVAL"
    lev = np.frombuffer(good, np.int32, n, HEADER + 4 * n).copy()
    top = int(lev.max())
    k = int(np.argmin(lev))
    for new in (top if lev[k] != top else 0, -1, top + 1):
        lev2 = lev.copy()
        lev2[k] = new
        bad.write_bytes(good[:HEADER + 4 * n] + lev2.tobytes() + good[HEADER + 8 * n:])
        assert _load_status(prgb, G, bad) == "PR_EINVAL"
    assert _load_status(prgb, G, tmp_path / "missing.bin") == "PR_EINVAL"
    # the good file still loads after the refusals
    L2 = prgb.load_partition(G, path)
    assert L2.n_comp == P.n_comp
