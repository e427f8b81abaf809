"""Seeded web-like graphs generated on the GPU with torch, for sizes where the
numpy generator would take many minutes (n = 50,000,000, 400,000,000 edges).

Same recipe as ``graphgen.web_like`` (it holds none of the method's
arithmetic): units laid out in layers -- one giant SCC (a Hamiltonian cycle
plus Chung-Lu internal edges), log-normal small SCCs (a cycle plus uniform
internal edges), chains (acyclic) and dangling vertices -- with Zipf(2.1)
out-degrees; edges leaving a unit go to a later layer at a geometric layer
distance, to targets drawn with Zipf(2.1) in-weights.  Vertex ids are
shuffled.  The graph stays on the device: (rowptr, col) int32 CUDA tensors,
rows sorted, no duplicates, no self-loops; u = 1/n.  With ``with_layers``
the planted layer of each vertex comes back too.

The draws come from torch's CUDA generator, so the graph depends on the
torch version as well as the seed.
"""
from __future__ import annotations

import math


def _zipf(torch, gen, a, size, cap, device):
    # continuous Pareto tail, floored: P(X >= x) ~ x^(1-a), truncated at cap
    u = torch.rand(size, generator=gen, device=device, dtype=torch.float64)
    x = torch.floor((1.0 - u).clamp_min(1e-300) ** (-1.0 / (a - 1.0)))
    return x.clamp(1, cap)


def web_like_device(seed=4, n=50_000_000, mean_deg=8.0, giant_frac=0.5, small_frac=0.012,
                    dangling_frac=0.12, layers=28, giant_layer=9, zipf_a=2.1, small_median=6.0,
                    small_sigma=1.5, small_max=2_000, device="cuda", with_layers=False):
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    i64 = torch.int64
    n_giant = int(round(giant_frac * n))
    n_dangling = int(round(dangling_frac * n))
    # small SCC sizes: log-normal, truncated to [2, small_max]
    k = int(small_frac * n)
    sz = torch.exp(math.log(small_median) + small_sigma *
                   torch.randn(2 * k, generator=gen, device=device, dtype=torch.float64)).round().to(i64)
    sz = sz[(sz >= 2) & (sz <= small_max)][:k]
    budget = n - n_giant - n_dangling - max(1, n // 20)
    cs = torch.cumsum(sz, 0)
    sz = sz[cs <= budget]
    n_chain_v = n - n_giant - n_dangling - int(sz.sum())
    # chains of 1..50 vertices
    ch = torch.randint(1, 51, (n_chain_v // 10 + 10,), generator=gen, device=device, dtype=i64)
    ch = ch[torch.cumsum(ch, 0) <= n_chain_v]
    rest = n_chain_v - int(ch.sum())
    if rest > 0:
        ch = torch.cat([ch, torch.tensor([rest], device=device, dtype=i64)])
    usize = torch.cat([torch.tensor([n_giant], device=device, dtype=i64), sz, ch,
                       torch.ones(n_dangling, device=device, dtype=i64)])
    kind = torch.cat([torch.zeros(1 + sz.numel(), device=device, dtype=torch.int8),
                      torch.ones(ch.numel(), device=device, dtype=torch.int8),
                      torch.full((n_dangling,), 2, device=device, dtype=torch.int8)])
    nu = usize.numel()
    ulayer = torch.randint(0, layers, (nu,), generator=gen, device=device, dtype=i64)
    ulayer[0] = giant_layer
    dmask = kind == 2
    ulayer[dmask] = torch.randint(1, layers, (int(dmask.sum()),), generator=gen, device=device, dtype=i64)
    key = ulayer.to(torch.float64) + torch.rand(nu, generator=gen, device=device, dtype=torch.float64) * 0.5
    order = torch.argsort(key)
    ustart = torch.empty(nu, device=device, dtype=i64)
    so = usize[order]
    ustart[order] = torch.cumsum(so, 0) - so
    # per position: unit, layer, kind, offset in unit
    unit_of_pos = torch.repeat_interleave(order, so)
    pos = torch.arange(n, device=device, dtype=i64)
    off = pos - ustart[unit_of_pos]
    pl = ulayer[unit_of_pos]
    pk = kind[unit_of_pos]
    lay_start = torch.searchsorted(pl, torch.arange(layers + 1, device=device, dtype=i64))
    # out-degrees: Zipf over the non-dangling vertices, mean ~ 1.3 * mean_deg
    nd = pk != 2
    z = _zipf(torch, gen, zipf_a, int(nd.sum()), 20_000, device)
    deg = torch.zeros(n, device=device, dtype=i64)
    deg[nd] = torch.clamp((z * (1.3 * mean_deg * n) / z.sum()).round(), min=1).to(i64)
    inw = _zipf(torch, gen, zipf_a, n, 50_000, device)
    srcs, dsts = [], []
    # SCC cycles (giant and small)
    scc = pk == 0
    us = usize[unit_of_pos]
    nxt = torch.where(off + 1 < us, pos + 1, pos - off)
    srcs.append(pos[scc])
    dsts.append(nxt[scc])
    # chains: i -> i + 1 inside the unit
    cm = (pk == 1) & (off + 1 < us)
    srcs.append(pos[cm])
    dsts.append(pos[cm] + 1)
    # internal extra edges: 80% of the rest in the giant, 50% in small SCCs
    restd = torch.clamp(deg - 1, min=0)
    p_int = torch.where(unit_of_pos == 0, 0.8, 0.5).to(torch.float64)
    extra = torch.zeros(n, device=device, dtype=i64)
    extra[scc] = torch.binomial(restd[scc].to(torch.float64), p_int[scc], generator=gen).to(i64)
    g0 = int(ustart[0])
    g1 = g0 + n_giant
    gm = (pos >= g0) & (pos < g1)
    gsrc = torch.repeat_interleave(pos[gm], extra[gm])
    gcum = torch.cumsum(inw[g0:g1], 0)
    gcum = gcum / gcum[-1]
    r = torch.rand(gsrc.numel(), generator=gen, device=device, dtype=torch.float64)
    gdst = torch.clamp(g0 + torch.searchsorted(gcum, r, right=True), max=g1 - 1)
    srcs.append(gsrc)
    dsts.append(gdst)
    sm = scc & ~gm
    ssrc = torch.repeat_interleave(pos[sm], extra[sm])
    r = torch.rand(ssrc.numel(), generator=gen, device=device, dtype=torch.float64)
    sdst = (pos[ssrc] - off[ssrc]) + (r * us[ssrc]).to(i64)
    srcs.append(ssrc)
    dsts.append(sdst)
    # edges to later layers
    ext = torch.clamp(deg - extra - scc.to(i64) - cm.to(i64), min=0)
    ext[pl >= layers - 1] = 0
    esrc = torch.repeat_interleave(pos, ext)
    u01 = torch.rand(esrc.numel(), generator=gen, device=device, dtype=torch.float64).clamp_min(1e-300)
    step = torch.floor(torch.log(u01) / math.log(1.0 - 0.45)).to(i64) + 1
    tl = torch.clamp(pl[esrc] + step, max=layers - 1)
    lo, hi = lay_start[tl], lay_start[tl + 1]
    cum = torch.cat([torch.zeros(1, device=device, dtype=torch.float64), torch.cumsum(inw, 0)])
    r = cum[lo] + torch.rand(esrc.numel(), generator=gen, device=device, dtype=torch.float64) * (cum[hi] - cum[lo])
    edst = torch.clamp(torch.searchsorted(cum, r, right=True) - 1, min=lo, max=hi - 1)
    ok = hi > lo
    srcs.append(esrc[ok])
    dsts.append(edst[ok])
    del esrc, edst, lo, hi, r, u01, step, tl
    src = torch.cat(srcs)
    dst = torch.cat(dsts)
    del srcs, dsts
    keep = src != dst
    src, dst = src[keep], dst[keep]
    # shuffle ids, then sort by (src, dst) and drop duplicates
    perm = torch.randperm(n, generator=gen, device=device)
    key = perm[src] * n + perm[dst]
    del src, dst
    key = torch.unique(key)  # sorted
    s = torch.div(key, n, rounding_mode="floor")
    col = (key - s * n).to(torch.int32)
    del key
    counts = torch.bincount(s, minlength=n)
    rowptr = torch.zeros(n + 1, device=device, dtype=torch.int32)
    rowptr[1:] = torch.cumsum(counts, 0).to(torch.int32)
    u = torch.full((n,), 1.0 / n, device=device, dtype=torch.float64)
    if with_layers:
        # the planted layer of every vertex (after the id shuffle): edges only
        # stay inside a unit or go to a later layer, so the vertices of the
        # first L layers are closed under predecessors for every L
        vlayer = torch.empty(n, device=device, dtype=torch.int8)
        vlayer[perm] = pl.to(torch.int8)
        return rowptr, col, u, vlayer
    return rowptr, col, u
