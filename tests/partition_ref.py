"""Brute-force restatements used to pin the oracle's partition.

``theorem_partition`` applies the merge procedure of Theorem 3.1 literally on
a tiny graph: SCCs from a transitive closure (Warshall), levels recomputed as
the longest path in the component DAG after every merge, and heads chosen at
random among the admissible 1-vertex CACs of the current level.  It shares
nothing with the oracle's DFS and is exponential-free only because graphs are
tiny.
"""
from __future__ import annotations

import numpy as np


def closure(n, edges):
    reach = np.eye(n, dtype=bool)
    for a, b in edges:
        reach[a, b] = True
    for k in range(n):
        reach |= reach[:, k:k + 1] & reach[k:k + 1, :]
    return reach


def scc_sets(n, edges):
    reach = closure(n, edges)
    same = reach & reach.T
    seen = [False] * n
    comps = []
    for v in range(n):
        if not seen[v]:
            members = frozenset(int(x) for x in np.nonzero(same[v])[0])
            for x in members:
                seen[x] = True
            comps.append(members)
    return comps


def comp_levels(n, edges, comps):
    """Def. 3.3: longest path (in components) from each component to a sink."""
    owner = {}
    for i, cset in enumerate(comps):
        for v in cset:
            owner[v] = i
    succ = [set() for _ in comps]
    for a, b in edges:
        if owner[a] != owner[b]:
            succ[owner[a]].add(owner[b])
    memo = {}

    def lev(i):
        if i in memo:
            return memo[i]
        memo[i] = -1  # cycle guard: a cycle in the component graph is a bug
        val = 0 if not succ[i] else 1 + max(lev(j) for j in succ[i])
        memo[i] = val
        return val

    return [lev(i) for i in range(len(comps))], succ, owner


def theorem_partition(n, edges, rng, merge=True):
    """Theorem 3.1 literally; returns a list of (members, type, level)."""
    edges = [(a, b) for a, b in edges if a != b]
    comps = scc_sets(n, edges)
    types = ["SCC" if len(cs) > 1 else "CAC" for cs in comps]
    if merge:
        L = 1
        while True:
            levels, succ, owner = comp_levels(n, edges, comps)
            if L > max(levels, default=0):
                break
            while True:
                levels, succ, owner = comp_levels(n, edges, comps)
                heads = []
                for i, cs in enumerate(comps):
                    if len(cs) != 1 or types[i] != "CAC" or levels[i] != L:
                        continue
                    below = [j for j in succ[i] if levels[j] == L - 1]
                    if not below or any(types[j] == "SCC" for j in below):
                        continue
                    heads.append((i, below))
                if not heads:
                    break
                i, below = heads[int(rng.integers(len(heads)))]
                merged = set(comps[i])
                for j in below:
                    merged |= comps[j]
                keep = [k for k in range(len(comps)) if k != i and k not in below]
                comps = [comps[k] for k in keep] + [frozenset(merged)]
                types = [types[k] for k in keep] + ["CAC"]
            L += 1
    levels, _, _ = comp_levels(n, edges, comps)
    return [(cs, t, l) for cs, t, l in zip(comps, types, levels)]


def canonical_arrays(n, parts):
    """Canonical ids: level desc, size desc, smallest vertex asc."""
    order = sorted(range(len(parts)),
                   key=lambda i: (-parts[i][2], -len(parts[i][0]), min(parts[i][0])))
    comp = np.empty(n, np.int32)
    typ = np.empty(n, np.uint8)
    lev = np.empty(n, np.int32)
    for cid, i in enumerate(order):
        cs, t, l = parts[i]
        for v in cs:
            comp[v] = cid
            typ[v] = 1 if t == "SCC" else 0
            lev[v] = l
    return comp, typ, lev


def as_sets(comp, typ, lev):
    """Label-free view of a partition: {(members, type, level)}."""
    out = {}
    for v in range(len(comp)):
        out.setdefault(int(comp[v]), []).append(v)
    return {(frozenset(m), int(typ[m[0]]), int(lev[m[0]])) for m in out.values()}


def edges_of(rowptr, col):
    out = []
    for i in range(len(rowptr) - 1):
        for e in range(rowptr[i], rowptr[i + 1]):
            out.append((i, int(col[e])))
    return out
