"""Seeded synthetic directed graphs for the componentwise PageRank workloads.

This module only draws graphs and weight vectors: it holds none of the
method's arithmetic (no partition, no PageRank).  Both the CPU oracle and the
CUDA path receive the same arrays from here.

Every generator plants a layered structure whose strongly connected
components are known by construction:

* an SCC unit gets a random Hamiltonian cycle plus extra internal edges, so it
  is strongly connected;
* an acyclic unit (chain or in-tree) only has edges towards its own root;
* every edge between two units goes from an earlier layer to a strictly later
  one, so no cycle crosses units.

Vertex ids are shuffled at the end so that the planted order is invisible in
memory.  Graphs come out as CSR (int32 ``rowptr[n+1]``, int32 ``col[nnz]``),
rows sorted, no duplicate edges and no self-loops.

Workloads (the paper's experiments use SNAP web-Google and a Barabasi-Albert
graph, neither of which ships here; these synthetic graphs stand in for their
shapes, Sec. 5.1):

* ``small_planted``  n=10,000,  ~50k edges, 200 SCCs, 2,000 acyclic vertices,
  10 layers, ~10% dangling, u = 1/n.
* ``web_like``       n=1,000,000, mean out-degree 8, Zipf(2.1) out- and
  in-degrees, one giant SCC (~40% of vertices), ~20,000 small SCCs with
  log-normal sizes (median 6, max 2,000), CAC trees and chains, 15% dangling,
  28 layers, u = 1/n.
* ``deep_dag``       n=4,000,000, ~30M edges, 200 forced levels, 200-400 SCCs
  per level (log-normal sizes in [2, 500]) plus CAC chains of length 1-50,
  u ~ U[0,1] normalised.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "Graph", "csr_from_edges", "small_planted", "web_like", "deep_dag",
    "random_digraph", "uniform_u", "random_u", "config", "closed_slice",
]


class Graph:
    """A CSR digraph plus the weight vector u and the planted facts."""

    def __init__(self, n, rowptr, col, u, name, planted=None):
        self.n = int(n)
        self.rowptr = rowptr
        self.col = col
        self.u = u
        self.name = name
        self.planted = planted or {}

    @property
    def nnz(self):
        return int(self.col.shape[0])

    def __repr__(self):
        return f"Graph({self.name}, n={self.n}, nnz={self.nnz})"


def csr_from_edges(n, src, dst, dedupe=True):
    """Sorted-row CSR from edge arrays (self-loops kept if present)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    key = np.sort(src * np.int64(n) + dst)
    if dedupe and key.shape[0] > 1:
        # sorted, then adjacent duplicates dropped: the same array as
        # np.unique, which on recent numpy hashes first and is far slower
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    s = key // n
    d = key - s * n
    counts = np.bincount(s, minlength=n).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("edge count does not fit int32 offsets")
    return rowptr.astype(np.int32), d.astype(np.int32)


def uniform_u(n):
    return np.full(n, 1.0 / n, dtype=np.float64)


def random_u(n, rng):
    u = rng.random(n)
    return u / u.sum()


def _relabel(n, src, dst, rng):
    perm = rng.permutation(n).astype(np.int64)
    return perm[src], perm[dst], perm


def _rescale_sizes(sizes, total, min_size):
    """Scale integer sizes to sum exactly ``total`` (largest remainder)."""
    x = sizes.astype(np.float64) * total / sizes.sum()
    base = np.floor(x).astype(np.int64)
    rem = total - base.sum()
    order = np.argsort(-(x - base), kind="stable")
    base[order[:rem]] += 1
    base = np.maximum(base, min_size)
    while base.sum() > total:
        i = int(np.argmax(base))
        base[i] -= 1
    return base


def _scc_internal_edges(rng, starts, sizes, extra_src_count=None, p=None):
    """Hamiltonian cycle per unit plus extra internal edges.

    Either ``p`` (Bernoulli per ordered pair, small units only) or
    ``extra_src_count`` (per-vertex number of extra internal targets, drawn
    uniformly inside the unit) selects the extra edges.
    """
    srcs, dsts = [], []
    # Hamiltonian cycles: a random cyclic order of each unit's members.
    total = int(sizes.sum())
    unit_of = np.repeat(np.arange(len(sizes)), sizes)
    offs = np.repeat(starts, sizes)
    # random order within each unit: sort by (unit, random key)
    key = unit_of.astype(np.float64) + rng.random(total) * 0.999
    order = np.argsort(key, kind="stable")
    local = np.arange(total) - np.repeat(np.cumsum(sizes) - sizes, sizes)
    member = offs + local  # member vertex ids in unit order
    cyc = member[order]  # unit-grouped, shuffled within unit
    nxt_local = (local + 1) % np.repeat(sizes, sizes)
    nxt = np.repeat(np.cumsum(sizes) - sizes, sizes) + nxt_local
    srcs.append(cyc)
    dsts.append(cyc[nxt])
    if p is not None:
        for st, sz in zip(starts.tolist(), sizes.tolist()):
            m = rng.random((sz, sz)) < p
            np.fill_diagonal(m, False)
            a, b = np.nonzero(m)
            srcs.append(a + st)
            dsts.append(b + st)
    if extra_src_count is not None:
        k = extra_src_count
        s = np.repeat(member, k)
        usz = np.repeat(np.repeat(sizes, sizes), k)
        ust = np.repeat(offs, k)
        t = ust + (rng.random(s.shape[0]) * usz).astype(np.int64)
        keep = t != s
        srcs.append(s[keep])
        dsts.append(t[keep])
    return np.concatenate(srcs), np.concatenate(dsts)


def _acyclic_units(rng, total, max_len, tree_frac):
    """Split ``total`` acyclic vertices into chains and in-trees.

    Returns (sizes, internal_src, internal_dst, tail_local) where node 0 of a
    unit is its root (the one vertex with no internal out-edge); internal
    edges point from child to parent.
    """
    sizes = []
    left = total
    while left > 0:
        s = int(min(left, rng.integers(1, max_len + 1)))
        sizes.append(s)
        left -= s
    sizes = np.array(sizes, dtype=np.int64)
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    is_tree = rng.random(len(sizes)) < tree_frac
    src, dst = [], []
    unit_of = np.repeat(np.arange(len(sizes)), sizes)
    local = np.arange(total) - np.repeat(starts, sizes)
    child = local > 0
    # chain: local i -> i-1 ; tree: local i -> random parent in [0, i)
    par = local - 1
    tree_v = child & is_tree[unit_of]
    par[tree_v] = (rng.random(int(tree_v.sum())) * local[tree_v]).astype(np.int64)
    g = np.arange(total)
    src = g[child]
    dst = (np.repeat(starts, sizes) + par)[child]
    return sizes, starts, src, dst


def small_planted(seed=1, n=10_000, n_scc=200, scc_vertices=8_000,
                  n_dangling=1_000, layers=10, target_edges=50_000):
    """Plain method, small: 200 planted SCCs + 2,000 acyclic vertices.

    SCC sizes are drawn U[5,100] and rescaled to sum 8,000 so that n stays
    10,000 with 2,000 acyclic vertices (U[5,100] alone would average 52.5 and
    overflow n).  Each SCC is a Hamiltonian cycle plus intra-edges with
    p = 0.05.  Acyclic vertices: 1,000 dangling singletons plus chains and
    in-trees.  Every non-bottom unit gets one edge into the next layer; the
    remaining edges go from a random source to a random vertex of a strictly
    later layer until ~50,000 edges.
    """
    rng = np.random.default_rng(seed)
    sizes_scc = _rescale_sizes(rng.integers(5, 101, n_scc), scc_vertices, 5)
    n_acyc = n - scc_vertices
    a_sizes, a_starts, a_src, a_dst = _acyclic_units(rng, n_acyc - n_dangling, 20, 0.5)
    # units: SCCs, acyclic chains/trees, dangling singletons
    kind = np.concatenate([np.zeros(n_scc, np.int8), np.ones(len(a_sizes), np.int8),
                           np.full(n_dangling, 2, np.int8)])
    usize = np.concatenate([sizes_scc, a_sizes, np.ones(n_dangling, np.int64)])
    ulayer = rng.integers(0, layers, len(usize))
    ulayer[kind == 2] = rng.integers(1, layers, n_dangling)
    order = np.lexsort((rng.random(len(usize)), ulayer))
    ustart = np.zeros(len(usize), np.int64)
    ustart[order] = np.concatenate([[0], np.cumsum(usize[order])[:-1]])
    vlayer = np.empty(n, np.int64)
    vunit = np.empty(n, np.int64)
    for_units = np.repeat(np.arange(len(usize)), usize)
    vpos = np.repeat(ustart, usize) + (np.arange(n) - np.repeat(np.cumsum(usize) - usize, usize))
    vlayer[vpos] = ulayer[for_units]
    vunit[vpos] = for_units
    srcs, dsts = [], []
    s_scc, d_scc = _scc_internal_edges(rng, ustart[:n_scc], sizes_scc, p=0.05)
    srcs.append(s_scc); dsts.append(d_scc)
    # acyclic internal edges: map unit-local ids to positions
    a_off = np.repeat(ustart[n_scc:n_scc + len(a_sizes)] - a_starts, a_sizes)
    srcs.append(a_src + a_off[a_src]); dsts.append(a_dst + a_off[a_dst])
    # layer boundaries in position order
    pos_layer = vlayer  # indexed by position
    lay_start = np.searchsorted(pos_layer, np.arange(layers + 1), side="left")
    dangling = np.zeros(n, bool)
    dangling[vpos[kind[for_units] == 2]] = True
    # one edge from every non-bottom, non-dangling unit into the next layer
    for u_i in range(len(usize)):
        if kind[u_i] == 2 or ulayer[u_i] >= layers - 1:
            continue
        L = ulayer[u_i] + 1
        a, b = lay_start[L], lay_start[L + 1]
        if b <= a:
            continue
        s = ustart[u_i] + rng.integers(0, usize[u_i])
        srcs.append(np.array([s])); dsts.append(np.array([rng.integers(a, b)]))
    cur = sum(x.shape[0] for x in srcs)
    need = max(0, target_edges - cur)
    cand = np.nonzero((~dangling) & (pos_layer < layers - 1))[0]
    s = cand[rng.integers(0, len(cand), need)]
    lo = lay_start[pos_layer[s] + 1]
    t = lo + (rng.random(need) * (n - lo)).astype(np.int64)
    srcs.append(s); dsts.append(t)
    src = np.concatenate(srcs); dst = np.concatenate(dsts)
    src, dst, perm = _relabel(n, src, dst, rng)
    rowptr, col = csr_from_edges(n, src, dst)
    planted = {"scc_sizes": np.sort(sizes_scc)[::-1], "layers": layers,
               "n_dangling_planted": n_dangling}
    return Graph(n, rowptr, col, uniform_u(n), f"small_planted(seed={seed})", planted)


def _zipf(rng, a, size, cap):
    return np.minimum(rng.zipf(a, size), cap).astype(np.int64)


def web_like(seed=2, n=1_000_000, mean_deg=8.0, giant_frac=0.40, n_small=20_000,
             dangling_frac=0.15, layers=28, giant_layer=10, zipf_a=2.1,
             small_median=6.0, small_sigma=1.5, small_max=2_000):
    """Web-like mid graph: giant SCC, many small SCCs, CAC trees/chains.

    Out-degrees of the non-dangling vertices follow Zipf(2.1), rescaled so the
    mean over all vertices is ``mean_deg``; targets of edges that leave a unit
    are picked Chung-Lu style with Zipf(2.1) in-weights, in a later layer at a
    geometric layer distance.
    """
    rng = np.random.default_rng(seed)
    n_giant = int(round(giant_frac * n))
    n_dangling = int(round(dangling_frac * n))
    # small SCC sizes: log-normal, median 6, truncated to [2, small_max]
    sz = np.exp(np.log(small_median) + small_sigma * rng.standard_normal(4 * n_small))
    sz = np.round(sz).astype(np.int64)
    sz = sz[(sz >= 2) & (sz <= small_max)][:n_small]
    budget = n - n_giant - n_dangling - max(1, n // 20)  # keep >=5% tree/chain vertices
    if sz.sum() > budget:
        cs = np.cumsum(sz)
        sz = sz[: int(np.searchsorted(cs, budget, side="right"))]
    n_small = len(sz)
    n_tree = n - n_giant - n_dangling - int(sz.sum())
    a_sizes, a_starts, a_src, a_dst = _acyclic_units(rng, n_tree, 12, 0.6)
    n_scc_units = 1 + n_small
    sizes_scc = np.concatenate([[n_giant], sz])
    kind = np.concatenate([np.zeros(n_scc_units, np.int8), np.ones(len(a_sizes), np.int8),
                           np.full(n_dangling, 2, np.int8)])
    usize = np.concatenate([sizes_scc, a_sizes, np.ones(n_dangling, np.int64)])
    nu = len(usize)
    ulayer = rng.integers(0, layers, nu)
    ulayer[0] = giant_layer
    ulayer[kind == 2] = rng.integers(1, layers, n_dangling)
    order = np.lexsort((rng.random(nu), ulayer))
    ustart = np.zeros(nu, np.int64)
    ustart[order] = np.concatenate([[0], np.cumsum(usize[order])[:-1]])
    for_units = np.repeat(np.arange(nu), usize)
    vpos = np.repeat(ustart, usize) + (np.arange(n) - np.repeat(np.cumsum(usize) - usize, usize))
    pos_layer = np.empty(n, np.int64); pos_layer[vpos] = ulayer[for_units]
    pos_unit = np.empty(n, np.int64); pos_unit[vpos] = for_units
    pos_kind = kind[pos_unit]
    lay_start = np.searchsorted(pos_layer, np.arange(layers + 1), side="left")
    # degrees
    nd = pos_kind != 2
    deg = np.zeros(n, np.int64)
    z = _zipf(rng, zipf_a, int(nd.sum()), 20_000).astype(np.float64)
    # duplicate targets (hubs) and the edges of the last layer are lost when
    # the CSR is built; drawing 1.3x the edges lands the mean near mean_deg
    deg[nd] = np.maximum(1, np.round(z * (1.3 * mean_deg * n) / z.sum())).astype(np.int64)
    inw = _zipf(rng, zipf_a, n, 50_000).astype(np.float64)
    srcs, dsts = [], []
    # SCC internal: cycle gives 1; extra internal edges ~ 80% (giant) / 50% (small) of the rest
    scc_v = pos_kind == 0
    p_int = np.where(pos_unit == 0, 0.8, 0.5)
    extra = np.zeros(n, np.int64)
    rest = np.maximum(deg - 1, 0)
    extra[scc_v] = rng.binomial(rest[scc_v], p_int[scc_v])
    small_units = np.arange(1, n_scc_units)
    # giant internal: weighted targets (Chung-Lu inside the giant)
    g0, g1 = ustart[0], ustart[0] + n_giant
    s_cyc, d_cyc = _scc_internal_edges(rng, ustart[:n_scc_units], sizes_scc,
                                       extra_src_count=None)
    srcs.append(s_cyc); dsts.append(d_cyc)
    gsrc = np.repeat(np.arange(g0, g1), extra[g0:g1])
    gcum = np.cumsum(inw[g0:g1]); gcum /= gcum[-1]
    gdst = g0 + np.searchsorted(gcum, rng.random(gsrc.shape[0]), side="right")
    gdst = np.minimum(gdst, g1 - 1)
    srcs.append(gsrc); dsts.append(gdst)
    # small SCC internal: uniform targets in the unit
    sm = scc_v & (pos_unit != 0)
    ssrc = np.repeat(np.nonzero(sm)[0], extra[sm])
    su = pos_unit[ssrc]
    sdst = ustart[su] + (rng.random(ssrc.shape[0]) * usize[su]).astype(np.int64)
    srcs.append(ssrc); dsts.append(sdst)
    # acyclic internal edges (tree/chain)
    a_off = np.repeat(ustart[n_scc_units:n_scc_units + len(a_sizes)] - a_starts, a_sizes)
    srcs.append(a_src + a_off[a_src]); dsts.append(a_dst + a_off[a_dst])
    # external edges: everything not used internally
    ext = deg - extra - scc_v.astype(np.int64)
    tree_child = np.zeros(n, bool); tree_child[a_src + a_off[a_src]] = True
    ext = np.maximum(ext - tree_child.astype(np.int64), 0)
    ext[pos_layer >= layers - 1] = 0
    esrc = np.repeat(np.arange(n), ext)
    step = rng.geometric(0.45, esrc.shape[0])
    tl = np.minimum(pos_layer[esrc] + step, layers - 1)
    lo = lay_start[tl]; hi = lay_start[tl + 1]
    cum = np.concatenate([[0.0], np.cumsum(inw)])
    r = cum[lo] + rng.random(esrc.shape[0]) * (cum[hi] - cum[lo])
    edst = np.searchsorted(cum, r, side="right") - 1
    edst = np.clip(edst, lo, hi - 1)
    ok = hi > lo
    srcs.append(esrc[ok]); dsts.append(edst[ok])
    src = np.concatenate(srcs); dst = np.concatenate(dsts)
    keep = src != dst
    src, dst, perm = _relabel(n, src[keep], dst[keep], rng)
    rowptr, col = csr_from_edges(n, src, dst)
    planted = {"giant_size": n_giant, "n_small_scc": n_small, "layers": layers}
    return Graph(n, rowptr, col, uniform_u(n), f"web_like(seed={seed}, n={n})", planted)


def deep_dag(seed=3, n=4_000_000, levels=200, scc_per_level=(200, 400),
             scc_mu=np.log(18.0), scc_sigma=1.0, scc_max=500, int_deg=15.0,
             inter_per_vertex=1.0):
    """Deep-DAG batching stress: ``levels`` layers forced to distinct levels.

    Each layer holds 200-400 SCCs (log-normal sizes truncated to [2, 500]) and
    CAC chains of length U[1, 50] filling the layer to n/levels vertices.
    Every SCC and every chain tail of a non-bottom layer gets one edge into an
    SCC of the next layer, which forces the component DAG to exactly
    ``levels`` levels.  Extra inter-layer edges go 1-3 layers down.
    """
    rng = np.random.default_rng(seed)
    per_layer = n // levels
    usize, ukind, ulayer = [], [], []
    for L in range(levels):
        k = int(rng.integers(scc_per_level[0], scc_per_level[1] + 1))
        s = np.round(np.exp(scc_mu + scc_sigma * rng.standard_normal(3 * k))).astype(np.int64)
        s = s[(s >= 2) & (s <= scc_max)][:k]
        cap = per_layer if L < levels - 1 else n - (levels - 1) * per_layer
        cs = np.cumsum(s)
        s = s[: int(np.searchsorted(cs, cap - 1, side="right"))]
        left = cap - int(s.sum())
        ch = []
        while left > 0:
            c = int(min(left, rng.integers(1, 51)))
            ch.append(c); left -= c
        usize += s.tolist() + ch
        ukind += [0] * len(s) + [1] * len(ch)
        ulayer += [L] * (len(s) + len(ch))
    usize = np.array(usize, np.int64); ukind = np.array(ukind, np.int8)
    ulayer = np.array(ulayer, np.int64)
    nu = len(usize)
    ustart = np.concatenate([[0], np.cumsum(usize)[:-1]])
    pos_unit = np.repeat(np.arange(nu), usize)
    pos_layer = ulayer[pos_unit]
    lay_start = np.searchsorted(pos_layer, np.arange(levels + 1), side="left")
    srcs, dsts = [], []
    scc_units = np.nonzero(ukind == 0)[0]
    ssz = usize[scc_units]
    member_cnt = np.repeat(ssz, ssz)
    k = np.minimum(rng.poisson(int_deg, int(ssz.sum())), member_cnt - 1)
    s_i, d_i = _scc_internal_edges(rng, ustart[scc_units], ssz, extra_src_count=k)
    srcs.append(s_i); dsts.append(d_i)
    # chains: local i -> i-1, root (local 0) is the tail that leaves the layer
    ch_units = np.nonzero(ukind == 1)[0]
    csz = usize[ch_units]
    cst = ustart[ch_units]
    loc = np.arange(int(csz.sum())) - np.repeat(np.cumsum(csz) - csz, csz)
    g = np.repeat(cst, csz) + loc
    srcs.append(g[loc > 0]); dsts.append(g[loc > 0] - 1)
    # SCC position table per layer for "edge into an SCC of the next layer"
    scc_pos = np.nonzero(ukind[pos_unit] == 0)[0]
    scc_lay = pos_layer[scc_pos]
    sl_start = np.searchsorted(scc_lay, np.arange(levels + 1), side="left")
    forced_units = np.nonzero(ulayer < levels - 1)[0]
    fs = ustart[forced_units] + (rng.random(len(forced_units)) * usize[forced_units]).astype(np.int64)
    fs[ukind[forced_units] == 1] = ustart[forced_units][ukind[forced_units] == 1]  # chain tail
    nl = ulayer[forced_units] + 1
    a, b = sl_start[nl], sl_start[nl + 1]
    ft = scc_pos[a + (rng.random(len(forced_units)) * (b - a)).astype(np.int64)]
    srcs.append(fs); dsts.append(ft)
    # extra inter-layer edges, 1-3 layers down, uniform targets
    m = int(inter_per_vertex * n)
    es = rng.integers(0, lay_start[levels - 1], m)
    step = rng.integers(1, 4, m)
    tl = np.minimum(pos_layer[es] + step, levels - 1)
    lo = lay_start[tl]; hi = lay_start[tl + 1]
    et = lo + (rng.random(m) * (hi - lo)).astype(np.int64)
    srcs.append(es); dsts.append(et)
    src = np.concatenate(srcs); dst = np.concatenate(dsts)
    keep = src != dst
    src, dst, perm = _relabel(n, src[keep], dst[keep], rng)
    rowptr, col = csr_from_edges(n, src, dst)
    planted = {"levels": levels, "n_scc": int(len(scc_units))}
    return Graph(n, rowptr, col, random_u(n, rng), f"deep_dag(seed={seed}, n={n})", planted)


def closed_slice(rowptr, col, u, keep):
    """The sub-CSR induced by the vertices with ``keep`` set, every edge that
    leaves the set redirected to a dangling dummy vertex: the k-th leaving
    edge of a row goes to dummy ns + k (ns = kept vertices), so each kept
    vertex keeps its out-degree and rows stay simple.  When the kept set is
    closed under predecessors (every in-neighbour of a kept vertex is kept),
    the system (I - c A^T) R = u restricted to it is unchanged: each equation
    involves only in-neighbours and their out-degrees.  Dummies get u = 0.
    Returns (rowptr, col, u, kept_ids): the kept vertices are renumbered
    0..ns-1 in ascending original id, listed in kept_ids."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = rowptr.shape[0] - 1
    ids = np.nonzero(np.asarray(keep, dtype=bool))[0]
    ns = ids.shape[0]
    newid = np.full(n, -1, np.int64)
    newid[ids] = np.arange(ns)
    cnt = rowptr[ids + 1] - rowptr[ids]
    first = np.cumsum(cnt) - cnt
    e = np.arange(int(cnt.sum()), dtype=np.int64) - np.repeat(first, cnt) + np.repeat(rowptr[ids], cnt)
    src = np.repeat(np.arange(ns, dtype=np.int64), cnt)
    dst = newid[col[e]]
    leave = dst < 0
    # rank of each leaving edge within its row
    lc = np.cumsum(leave) - leave
    rank = lc - np.repeat(lc[first] if ns else lc[:0], cnt)
    dst[leave] = ns + rank[leave]
    n_dummy = int(rank[leave].max()) + 1 if leave.any() else 0
    rp, cl = csr_from_edges(ns + n_dummy, src, dst)
    us = np.concatenate([np.asarray(u, dtype=np.float64)[ids], np.zeros(n_dummy)])
    return rp, cl, us, ids


def random_digraph(n, p, seed, loops=False):
    """Erdos-Renyi digraph G(n, p); optional self-loops kept in the CSR."""
    rng = np.random.default_rng(seed)
    m = rng.random((n, n)) < p
    if not loops:
        np.fill_diagonal(m, False)
    s, d = np.nonzero(m)
    rowptr, col = csr_from_edges(n, s, d)
    return Graph(n, rowptr, col, uniform_u(n), f"gnp(n={n},p={p},seed={seed})")


def deep_dag_arrays(spec):
    """(rowptr, col, u) of deep_dag(seed, n, levels) for spec = (seed, n,
    levels): a picklable entry point for process pools."""
    seed, n, levels = spec
    g = deep_dag(seed=seed, n=n, levels=levels)
    return g.rowptr, g.col, g.u


def config(name, seed=None, **kw):
    """Named workloads with their default seeds."""
    if name == "small":
        return small_planted(seed=1 if seed is None else seed, **kw)
    if name == "web":
        return web_like(seed=2 if seed is None else seed, **kw)
    if name == "deep":
        return deep_dag(seed=3 if seed is None else seed, **kw)
    raise KeyError(name)
