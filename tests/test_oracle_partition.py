"""Pins for the oracle's SCC/CAC partition (Sec. 3 Theorem 3.1, Sec. 4.1).

The oracle is checked against things other than itself: the worked example
of Fig. 1, a literal brute-force application of the Theorem's merge procedure
on every 4-vertex digraph and on random tiny digraphs, relabelling
invariance (the partition is unique, Theorem statement 1), and the
structural invariants of Def. 3.1-3.3 and Corollary 3.1.
"""
import itertools
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.partition_ref import (as_sets, canonical_arrays, closure, edges_of,
                                 theorem_partition)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig1.txt")


def load_fig1():
    spec = {"components": []}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *rest = line.split()
            if key == "n":
                spec["n"] = int(rest[0])
            elif key == "edges":
                spec["edges"] = [tuple(int(x) for x in t.split("-")) for t in rest]
            elif key == "scc_levels":
                spec["scc_levels"] = [int(x) for x in rest]
            elif key == "component":
                members = [int(x) for x in rest[0].split(",")]
                spec["components"].append((members, rest[1], int(rest[2])))
            else:
                spec[key] = int(rest[0])
    return spec


def test_fig1_partition():
    spec = load_fig1()
    s, d = zip(*spec["edges"])
    rp, col = gg.csr_from_edges(spec["n"], s, d)
    p = oracle.partition(rp, col)
    got = as_sets(p.comp, p.type, p.level)
    want = {(frozenset(m), 1 if t == "SCC" else 0, l) for m, t, l in spec["components"]}
    assert got == want
    assert p.n_levels == spec["n_levels"]
    assert p.n_comp == 4
    # canonical ids: level desc, size desc, min id asc
    assert list(p.comp) == [0, 1, 2, 1, 2, 2, 3, 3]


def test_fig1_scc_only_levels():
    spec = load_fig1()
    s, d = zip(*spec["edges"])
    rp, col = gg.csr_from_edges(spec["n"], s, d)
    p = oracle.partition(rp, col, merge=False)
    assert list(p.level) == spec["scc_levels"]
    assert p.n_levels == spec["n_levels_scc_only"]


def _check_against_theorem(n, edges, rng):
    s = [a for a, _ in edges]
    d = [b for _, b in edges]
    rp, col = gg.csr_from_edges(n, s, d) if edges else (np.zeros(n + 1, np.int32), np.zeros(0, np.int32))
    p = oracle.partition(rp, col)
    ref = theorem_partition(n, edges, rng)
    comp, typ, lev = canonical_arrays(n, ref)
    assert np.array_equal(p.comp, comp), (edges, p.comp, comp)
    assert np.array_equal(p.type, typ), (edges, p.type, typ)
    assert np.array_equal(p.level, lev), (edges, p.level, lev)


def test_all_4_vertex_digraphs_match_theorem():
    n = 4
    pairs = [(a, b) for a in range(n) for b in range(n) if a != b]
    rng = np.random.default_rng(0)
    for mask in range(1 << len(pairs)):
        edges = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        _check_against_theorem(n, edges, rng)


def test_random_tiny_digraphs_match_theorem():
    rng = np.random.default_rng(1)
    for trial in range(1500):
        n = int(rng.integers(1, 11))
        p = float(rng.choice([0.08, 0.15, 0.25, 0.4]))
        m = rng.random((n, n)) < p
        np.fill_diagonal(m, rng.random(n) < 0.1)  # a few self-loops, ignored
        edges = [(int(a), int(b)) for a, b in zip(*np.nonzero(m))]
        _check_against_theorem(n, edges, rng)


def test_random_dag_like_digraphs_match_theorem():
    """Mostly-forward edges give deep chains of merges."""
    rng = np.random.default_rng(2)
    for trial in range(800):
        n = int(rng.integers(3, 13))
        edges = set()
        for _ in range(int(rng.integers(n - 1, 3 * n))):
            a, b = sorted(rng.integers(0, n, 2).tolist())
            if a != b:
                edges.add((a, b) if rng.random() < 0.9 else (b, a))
        _check_against_theorem(n, sorted(edges), rng)


def _relabelled(rp, col, perm):
    n = len(rp) - 1
    src = np.repeat(np.arange(n), np.diff(rp))
    return gg.csr_from_edges(n, perm[src], perm[col])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_partition_unique_under_relabelling(seed):
    g = gg.small_planted(seed=10 + seed)
    p = oracle.partition(g.rowptr, g.col)
    perm = np.random.default_rng(seed).permutation(g.n)
    rp2, col2 = _relabelled(g.rowptr, g.col, perm)
    p2 = oracle.partition(rp2, col2)
    back = as_sets(p2.comp[perm], p2.type[perm], p2.level[perm])
    assert back == as_sets(p.comp, p.type, p.level)
    # component sizes per canonical id are label-free too
    assert np.array_equal(np.sort(p.sizes()), np.sort(p2.sizes()))


def check_invariants(rp, col, p):
    n = len(rp) - 1
    src = np.repeat(np.arange(n), np.diff(rp)).astype(np.int64)
    dst = col.astype(np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    cs, cd = p.comp[src], p.comp[dst]
    lev_c = np.zeros(p.n_comp, np.int64)
    lev_c[p.comp] = p.level
    typ_c = np.zeros(p.n_comp, np.int64)
    typ_c[p.comp] = p.type
    size_c = p.sizes()
    # one level and one type per component
    assert np.all(lev_c[p.comp] == p.level) and np.all(typ_c[p.comp] == p.type)
    # Def. 3.3: level = 0 without external out-edges, else 1 + max level of successors
    ext = cs != cd
    best = np.full(p.n_comp, -1, np.int64)
    np.maximum.at(best, cs[ext], lev_c[cd[ext]])
    assert np.array_equal(lev_c, best + 1)
    # edges between components strictly lower the level (so the component graph is a DAG)
    assert np.all(lev_c[cs[ext]] > lev_c[cd[ext]])
    # SCC type means size >= 2; 1-vertex components are CACs (Sec. 3)
    assert np.all(size_c[typ_c == 1] >= 2)
    # CAC vertices lie on no cycle: they are 1-vertex SCCs of the plain split
    q = oracle.partition(rp, col, merge=False)
    qsize = q.sizes()
    assert np.all(qsize[q.comp[p.type == 0]] == 1)
    # SCC components coincide with the plain SCCs of size >= 2
    scc_mask = p.type == 1
    assert np.all(qsize[q.comp[scc_mask]] >= 2)
    # Corollary 3.1: L_SCC/CAC <= L_SCC
    assert p.n_levels <= q.n_levels
    # every CAC is weakly connected through its internal edges
    internal = (cs == cd) & (typ_c[cs] == 0)
    parent = np.arange(n)

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for a, b in zip(src[internal], dst[internal]):
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[ra] = rb
    roots = {}
    for v in np.nonzero(p.type == 0)[0]:
        roots.setdefault(int(p.comp[v]), set()).add(find(v))
    assert all(len(r) == 1 for r in roots.values())
    # canonical order: level desc, then size desc, then smallest vertex asc
    minv = np.full(p.n_comp, n, np.int64)
    np.minimum.at(minv, p.comp, np.arange(n))
    keys = list(zip(-lev_c, -size_c, minv))
    assert keys == sorted(keys)


@pytest.mark.parametrize("seed", [1, 5])
def test_invariants_small_planted(seed):
    g = gg.small_planted(seed=seed)
    p = oracle.partition(g.rowptr, g.col)
    check_invariants(g.rowptr, g.col, p)
    # the planted SCCs are exactly the SCC components
    assert np.array_equal(np.sort(p.sizes()[np.unique(p.comp[p.type == 1])])[::-1],
                          g.planted["scc_sizes"])


def test_invariants_random_sparse():
    for seed in range(6):
        g = gg.random_digraph(300, 1.3 / 300, seed, loops=True)
        p = oracle.partition(g.rowptr, g.col)
        check_invariants(g.rowptr, g.col, p)


def test_closure_helper_matches_definition():
    # guard for the brute force itself: a 3-cycle plus a tail
    r = closure(4, [(0, 1), (1, 2), (2, 0), (2, 3)])
    assert r[0, 2] and r[2, 0] and r[0, 3] and not r[3, 0]


def test_empty_and_trivial_graphs():
    p = oracle.partition(np.zeros(1, np.int32), np.zeros(0, np.int32))
    assert p.n_comp == 0 and p.n_levels == 0
    p = oracle.partition(np.zeros(2, np.int32), np.zeros(0, np.int32))
    assert p.n_comp == 1 and p.level[0] == 0 and p.type[0] == 0
    # a single self-loop is ignored: one CAC at level 0
    p = oracle.partition(np.array([0, 1], np.int32), np.array([0], np.int32))
    assert p.n_comp == 1 and p.type[0] == 0 and p.level[0] == 0
    # two-vertex edge: merged into one CAC of level 0 (Corollary 3.1 example)
    rp, col = gg.csr_from_edges(2, [0], [1])
    p = oracle.partition(rp, col)
    assert p.n_comp == 1 and p.n_levels == 1
    q = oracle.partition(rp, col, merge=False)
    assert q.n_levels == 2


def test_long_chain_is_one_cac():
    n = 20000
    rp, col = gg.csr_from_edges(n, np.arange(n - 1), np.arange(1, n))
    p = oracle.partition(rp, col)
    assert p.n_comp == 1 and p.n_levels == 1 and p.type.max() == 0
