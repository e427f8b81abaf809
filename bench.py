#!/usr/bin/env python3
"""Benchmark of the componentwise PageRank hot path on GB300.

One step = the whole path on one synthetic graph already resident in HBM:
prepare the graph (validate, drop loops, CSC), partition it into SCCs/CACs
with levels and lay it out, solve level by level to an L1 residual budget of
1e-10, and check the residual.  The global power series (the paper's
baseline) is timed the same way in a second loop.

value = graph edges / time per step (GTEPS: edges of the input solved to
residual 1e-10 per second), summed over ranks.  Each rank solves its own
replica (independent problems, no collective on the data path).

--impl reference times the CPU oracle (the plain C implementation the tests
use) on the machine's host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import graphgen as gg  # noqa: E402

METRIC = "componentwise PageRank GTEPS & time-to-1e-10 vs global power iter, 1 GB300"
UNIT = "GTEPS"
C = 0.85
TOL = 1e-10
FLUSH_BYTES = 256 << 20
# DRAM bytes (read + write) of one launch of the grid-wide SCC kernel, from
# an ncu capture of the current kernel on that workload (the summary under
# profiles/ gives the command); None where no capture was taken
TRAFFIC_BYTES = {"web": 23_820_032 + 1_577_472, "large": 572_180_000_000 + 47_880_000_000}

WORKLOADS = {
    "web": ("web_like: n=1,000,000, mean out-degree 8, Zipf(2.1) degrees, giant SCC 40%, "
            "~18k small log-normal SCCs, CAC trees/chains, 15% dangling, 28 layers, u=1/n, "
            "c=0.85, L1 tol 1e-10, FP64"),
    "small": ("small_planted: n=10,000, ~50k edges, 200 SCCs, 2,000 acyclic, 10 layers, "
              "u=1/n, c=0.85, L1 tol 1e-10, FP64"),
    "deep": ("deep_dag: n=4,000,000, ~28M edges, 200 forced levels, 200-400 SCCs per level, "
             "CAC chains 1-50, u~U[0,1] normalised, c=0.85, L1 tol 1e-10, FP64"),
    "large": ("web_like (generated on the GPU): n=50,000,000, ~400M edges, Zipf(2.1) degrees, giant SCC 50%, "
              "small log-normal SCCs, chains, 12% dangling, 28 layers, u=1/n, c=0.85, L1 tol 1e-10, FP64 "
              "(mixed precision reported beside it)"),
}


class _DeviceGraph:
    """A graph generated on the device (the large workload): numpy-like
    fields for the host copies the end-to-end leg needs."""

    def __init__(self, rowptr, col, u):
        self.rowptr_d, self.col_d, self.u_d = rowptr, col, u
        self.n = int(rowptr.numel() - 1)
        self.nnz = int(col.numel())

    def host(self):
        return self.rowptr_d.cpu().numpy(), self.col_d.cpu().numpy(), self.u_d.cpu().numpy()


def load_workload(name, large_n=50_000_000):
    if name == "large":
        from graphgen.large import web_like_device
        return _DeviceGraph(*web_like_device(seed=4, n=large_n))
    return gg.config(name)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="web")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--breakdown", action="store_true", help="(per-step times always go to stderr)")
    ap.add_argument("--no-warm-start", action="store_true",
                    help="accepted for compatibility: the default run no longer times the warm start (--warm-eval)")
    ap.add_argument("--large-n", type=int, default=50_000_000, help="vertices of the large workload")
    ap.add_argument("--no-blocks", action="store_true",
                    help="skip the deep_dag and 50M-vertex blocks of the default web_like run")
    ap.add_argument("--warm-eval", action="store_true",
                    help="the learned warm start on the deep-DAG generator: train on 1,000 graphs of n=100,000, "
                         "evaluate on 20 held-out graphs of n=4,000,000 against cold start (one JSON line)")
    ap.add_argument("--warm-train", type=int, default=1000, help="training graphs of --warm-eval")
    ap.add_argument("--warm-held", type=int, default=20, help="held-out graphs of --warm-eval")
    ap.add_argument("--profile-solves", type=int, default=0,
                    help="for profilers: prepare and partition the workload, run this many FP64 solves, exit")
    ap.add_argument("--shape", default=None,
                    help="cta_max,coop_blocks,balance of --profile-solves (default: the autotuner's choice)")
    ap.add_argument("--partition-io", action="store_true",
                    help="time pr_partition_create against pr_partition_save and pr_partition_load "
                         "on the web_like, deep_dag and large graphs; one JSON line")
    ap.add_argument("--cpu-parallel-worker", action="store_true",
                    help="internal: time the multi-core CPU baseline and print one JSON line")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def max_over_ranks(dist, x, device):
    """The largest x over the ranks (each rank times its own replica; the job
    takes as long as the slowest)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(edges_per_rank, world, ms):
    """Whole-job throughput in GTEPS: every rank solves its own replica of
    edges_per_rank edges, in ms milliseconds (the max over ranks)."""
    return world * edges_per_rank / (ms * 1e-3) / 1e9


def measured_l2_gbs(reps=40):
    """L2 bandwidth measured live on 64 MiB resident in L2 after a warm-up,
    bytes over CUDA-event time, the larger of: an FP32 sum of a 64 MiB
    vector (reads; FP32 adds run at full rate, so the loads bound it -- an
    FP64 sum would be bound by GB300's slow FP64 pipe instead) and a copy
    between two 32 MiB buffers (read + write bytes).  The denominator of the
    roofline when the dominant kernel's working set stays in L2 (no device
    constant gives it)."""
    import torch
    x = torch.ones(16 << 20, dtype=torch.float32, device="cuda")
    src = torch.ones(4 << 20, dtype=torch.float64, device="cuda")
    dst = torch.empty_like(src)

    def rate(fn, nbytes):
        for _ in range(5):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return nbytes * reps / (a.elapsed_time(b) * 1e-3) / 1e9

    return max(rate(x.sum, x.numel() * 4), rate(lambda: dst.copy_(src), 2 * src.numel() * 8))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clk", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(1.0)  # let the sampler start up before the timed region

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons),
                       samples=len(sm))
        return out


def oracle_step_result(g):
    """One oracle step (partition + componentwise solve): (seconds, R)."""
    import oracle
    t0 = time.perf_counter()
    q = oracle.partition(g.rowptr, g.col)
    R, _ = oracle.solve_cw(g.rowptr, g.col, q, C, g.u, TOL)
    return time.perf_counter() - t0, R


def oracle_step(g):
    return oracle_step_result(g)[0]


def reference_sample(args):
    """The workload itself when K+W oracle steps fit in ~3 minutes, else the
    same generator at a proportionally smaller n (same shape)."""
    if args.workload == "large":
        # the 50M-vertex graph is far beyond a bounded CPU sample: the numpy
        # web-like generator with the same shape at n = 1,000,000
        g = gg.web_like(seed=4, n=1_000_000, giant_frac=0.5, n_small=12_000, dangling_frac=0.12)
        return g, None, "numpy web_like at n=1,000,000 with the large workload's shape (bounded sample)"
    g = gg.config(args.workload)
    t = oracle_step(g)  # also the first warm-up step
    budget = 180.0
    if (args.steps + args.warmup) * t <= budget or args.workload == "small":
        return g, t, "full workload"
    scale = budget / ((args.steps + args.warmup) * t)
    n = max(10_000, int(g.n * scale))
    if args.workload == "web":
        g2 = gg.web_like(n=n, n_small=max(100, int(20_000 * n / 1_000_000)))
    else:
        g2 = gg.deep_dag(n=n, levels=max(10, int(200 * min(1.0, n / 4_000_000))))
    return g2, None, f"same generator at n={n} (bounded sample)"


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    g, first, sample = reference_sample(args)
    for _ in range(max(0, args.warmup - (1 if first is not None else 0))):
        oracle_step(g)
    times = [oracle_step(g) for _ in range(args.steps)]
    t = sum(times) / len(times)
    value = g.nnz / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "n": g.n, "nnz": g.nnz, "c": C, "tol": TOL,
                   "norm": "L1", "parallelism": "single", "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{sample}: oracle partition + componentwise solve, single thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def sweep_stats(comp, ctype, rowptr, col, comp_iters, g_iters):
    """Power-series sweeps per SCC: min / median / max over the SCCs and the
    mean over SCC-internal edges (each edge weighted by its SCC's sweeps),
    next to the global series' sweeps -- the comparison of Sec. 5.2 (sweeps
    per SCC edge, componentwise against the whole graph as one component).
    comp, ctype: per-vertex component id and type (torch, any device);
    rowptr, col: the CSR on the same device; comp_iters: numpy, by
    component id."""
    import torch
    n = comp.numel()
    n_comp = len(comp_iters)
    dev = comp.device
    comp = comp.long()
    deg = (rowptr[1:] - rowptr[:-1]).long()
    src = torch.repeat_interleave(torch.arange(n, device=dev), deg)
    dst = col.long()
    cs = comp[src]
    internal = (cs == comp[dst]) & (src != dst)
    m_c = torch.bincount(cs[internal], minlength=n_comp).double()
    is_scc = torch.zeros(n_comp, dtype=torch.bool, device=dev)
    is_scc[comp[ctype == 1]] = True
    it = torch.as_tensor(np.asarray(comp_iters), device=dev).double()
    its, ms = it[is_scc], m_c[is_scc]
    if its.numel() == 0:
        return {"scc_components": 0, "global_sweeps": int(g_iters)}
    return {"scc_components": int(its.numel()), "min": int(its.min()), "median": float(its.median()),
            "max": int(its.max()), "edge_weighted_mean": float((its * ms).sum() / ms.sum()),
            "scc_internal_edges": int(ms.sum()), "global_sweeps": int(g_iters)}


def cpu_parallel_worker(args):
    """The multi-core CPU baseline on the host cores: the partition from the
    oracle (single thread, timed apart), then the componentwise step and the
    global power series parallelised with OpenMP (cpu_parallel/), one
    warm-up and the median of three timed runs each."""
    import cpu_parallel as cp
    import oracle
    oracle.build()
    g = gg.config(args.workload)
    t0 = time.perf_counter()
    q = oracle.partition(g.rowptr, g.col)
    t_part = time.perf_counter() - t0
    plan = cp.Plan(g.rowptr, g.col, q.comp, q.type, q.level)
    cores = cp.max_threads()

    def timed(fn):
        fn()
        ts, out = [], None
        for _ in range(3):
            t = time.perf_counter()
            out = fn()
            ts.append(time.perf_counter() - t)
        return float(np.median(ts)) * 1e3, out

    cw_ms, (R, cw_it) = timed(lambda: plan.solve_cw(C, g.u, TOL, threads=cores))
    gl_ms, (Rg, gl_it) = timed(lambda: plan.solve_global(C, g.u, TOL, threads=cores))
    print(json.dumps({
        "cores": cores, "kind": "OpenMP componentwise step and global power series (cpu_parallel/)",
        "partition_ms": t_part * 1e3, "partition_kind": "oracle Tarjan DFS, single thread",
        "cw_solve_ms": cw_ms, "cw_iters_max": cw_it,
        "cw_residual_l1": oracle.residual_l1(g.rowptr, g.col, C, g.u, R),
        "global_solve_ms": gl_ms, "global_iters": gl_it,
        "global_residual_l1": oracle.residual_l1(g.rowptr, g.col, C, g.u, Rg)}), flush=True)
    return 0


def cpu_parallel_leg(args):
    """Runs cpu_parallel_worker in a child process (a failure there costs this
    field only); returns its JSON object or {"unavailable": reason}."""
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-parallel-worker", "--workload", args.workload]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=240)
        if r.returncode != 0:
            return {"unavailable": f"worker exited {r.returncode}: {r.stderr.strip()[-300:]}"}
        return json.loads(r.stdout.strip().splitlines()[-1])
    except (subprocess.TimeoutExpired, OSError, ValueError, IndexError) as e:
        return {"unavailable": f"{type(e).__name__}: {str(e)[:300]}"}


def diff_fields(R_gpu, R_ref):
    """L1 difference and largest relative difference of two solutions."""
    d = np.abs(np.asarray(R_gpu) - np.asarray(R_ref))
    return {"l1_diff": float(d.sum()),
            "max_rel": float(np.max(d / np.abs(np.asarray(R_ref)).clip(1e-300))) if d.size else 0.0}


def replay_for(q, gpu_comp, gpu_iters, ids=None):
    """The GPU's sweep count of each SCC, indexed by the oracle's component
    ids: through one member vertex of each component (ids maps the vertices
    of a slice back to the whole graph).  CACs and dummies get 0."""
    K = q.n_comp
    member = np.zeros(K, np.int64)
    member[q.comp] = np.arange(q.comp.shape[0])
    ctype = np.zeros(K, np.uint8)
    ctype[q.comp] = q.type
    scc = ctype == 1
    orig = member if ids is None else ids[np.minimum(member, ids.shape[0] - 1)]
    return np.where(scc, np.asarray(gpu_iters)[np.asarray(gpu_comp)[orig]], 0).astype(np.int32)


def oracle_vs(rowptr, col, u, tol, R_gpu, gpu_comp, gpu_iters, ids=None, tol_scale=1.0):
    """The oracle (partition + componentwise FP64 solve, single thread) on a
    CSR, against the GPU's FP64 result on the same vertices: once with each
    side stopping by its own rule (the difference is then bounded by
    2 tol / (1 - c) in L1), once with the GPU's sweep counts replayed, where
    both compute the same truncated series and the difference is rounding
    (bound 1e-12 relative per entry).  On a slice (ids given) tol is scaled
    so that every component keeps its budget tol |C| / n of the whole graph."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    q = oracle.partition(rowptr, col)
    t_part = time.perf_counter() - t0
    t0 = time.perf_counter()
    R_own, _ = oracle.solve_cw(rowptr, col, q, C, u, tol * tol_scale)
    t_solve = time.perf_counter() - t0
    R_rep, _ = oracle.solve_cw(rowptr, col, q, C, u, tol * tol_scale,
                               replay_iters=replay_for(q, gpu_comp, gpu_iters, ids))
    k = R_gpu.shape[0]
    own = diff_fields(R_gpu, R_own[:k])
    rep = diff_fields(R_gpu, R_rep[:k])
    return {"own_rule": dict(own, l1_bound=2 * TOL / (1 - C)),
            "replayed_sweeps": dict(rep, max_rel_bound=1e-12),
            "oracle_partition_s": t_part, "oracle_solve_s": t_solve}, R_own[:k]


def make_steps(prgb, rowptr, col, u):
    """One componentwise step (graph, partition, solve, residual) and one
    global step (graph, series, residual), each bracketed by CUDA events on
    the current stream."""
    import torch

    def ev():
        return torch.cuda.Event(enable_timing=True)

    def cw_step():
        e = [ev() for _ in range(5)]
        e[0].record()
        G = prgb.graph(rowptr, col)
        e[1].record()
        P = prgb.partition(G)
        e[2].record()
        # kernel events only: the per-component counts are read after the
        # timed region (counted_stats)
        R, st = prgb.solve(P, C, u, TOL, with_stats=True, timing=True, counts=False)
        e[3].record()
        res = prgb.residual_l1(G, C, u, R)
        e[4].record()
        return e, st, res, P

    def global_step():
        e = [ev() for _ in range(4)]
        e[0].record()
        G = prgb.graph(rowptr, col)
        e[1].record()
        R, k, st = prgb.global_power(G, C, u, TOL, with_stats=True, timing=True)
        e[2].record()
        res = prgb.residual_l1(G, C, u, R)
        e[3].record()
        return e, st, res, k

    return cw_step, global_step


def replay_ms(prgb, P, u, flush, steps, precision):
    """Device time of `steps` solves of an already solved partition (its
    CUDA graph replayed), L2 flushed before each, with the grid-wide
    kernels timed: (mean ms, the last solve's stats)."""
    import torch
    prgb.solve(P, C, u, TOL, timing=True, precision=precision)  # the graph for these parameters
    recs = []
    for k in range(steps):
        flush.fill_(k & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        R, st = prgb.solve(P, C, u, TOL, with_stats=True, timing=True, precision=precision, counts=False)
        b.record()
        recs.append((a, b, st, R))
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b, _, _ in recs])), recs


def counted_stats(prgb, P, u, precision=0):
    """The per-component sweep counts and edge visits of a solve of P (one
    extra solve outside the timed regions; the counts are deterministic)."""
    _, st = prgb.solve(P, C, u, TOL, with_stats=True, precision=precision)
    return st


def partition_phases(prgb, rowptr, col, flush):
    """One extra partition (outside the timed regions, L2 flushed before it)
    with PR_PARTITION_TIMING: its phase times and wave counts."""
    try:
        flush.fill_(7)
        G = prgb.graph(rowptr, col)
        return prgb.partition(G, timing=True).timing()
    except Exception as e:  # a report field only: never lose the bench line
        return {"unavailable": f"{type(e).__name__}: {str(e)[:200]}"}


def elapsed(recs, nphase):
    return np.array([[r[0][j].elapsed_time(r[0][j + 1]) for j in range(nphase)] for r in recs])


def config_block(prgb, name, args, flush, local):
    """A second configuration timed like the headline, on the same GPU: the
    componentwise step and the global series (3 warm-ups, then up to 5 or 3
    timed steps, L2 flushed before each), the FP64 solve against the mixed
    one, the grid-wide kernel's roofline and the sweeps per SCC.  Returns the
    report and what the oracle comparison needs."""
    import torch
    t0 = time.time()
    layers = None
    if name == "large":
        from graphgen.large import web_like_device
        rowptr, col, u, layers = web_like_device(seed=4, n=args.large_n, with_layers=True)
    else:
        g = gg.config(name)
        rowptr = torch.from_numpy(g.rowptr).cuda()
        col = torch.from_numpy(g.col).cuda()
        u = torch.from_numpy(g.u).cuda()
    t_gen = time.time() - t0
    n, E = int(rowptr.numel() - 1), int(col.numel())
    tuned = prgb.partition(prgb.graph(rowptr, col)).tune(C, u, TOL)
    cw_step, global_step = make_steps(prgb, rowptr, col, u)
    steps = max(1, min(args.steps, 5 if name == "deep" else 3))
    for _ in range(3):
        cw_step()
        global_step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    recs = []
    for k in range(steps):
        flush.fill_(k & 0xFF)
        r = cw_step()
        if recs:
            recs[-1] = recs[-1][:3] + (None,)  # keep one partition alive
        recs.append(r)
    grecs = []
    for k in range(steps):
        flush.fill_(k & 0xFF)
        grecs.append(global_step())
    torch.cuda.synchronize()
    clk = clocks.stop()
    ph = elapsed(recs, 4)
    gph = elapsed(grecs, 3)
    t_step, t_solve = float(ph.sum(axis=1).mean()), float(ph[:, 2].mean())
    t_global, t_global_solve = float(gph.sum(axis=1).mean()), float(gph[:, 1].mean())
    P = recs[-1][3]
    st = counted_stats(prgb, P, u)
    comp_d, type_d, _ = P.query()
    g_iters = grecs[-1][3]
    sweeps = sweep_stats(comp_d, type_d, rowptr, col, st["comp_iters"], g_iters)
    part_phases = partition_phases(prgb, rowptr, col, flush)
    R64 = prgb.solve(P, C, u, TOL)
    # mixed precision against FP64 on the same partition, both replayed
    t_fp64r, _ = replay_ms(prgb, P, u, flush, steps, prgb.PREC_FP64)
    t_mixed, mts = replay_ms(prgb, P, u, flush, steps, prgb.PREC_MIXED)
    Rm = mts[-1][3]
    stm = counted_stats(prgb, P, u, prgb.PREC_MIXED)
    m_res = prgb.residual_l1(prgb.graph(rowptr, col), C, u, Rm)
    k_ms = float(np.mean([r[1]["kernel_ms"] for r in recs]))
    k_bytes = float(np.mean([r[1]["kernel_bytes"] for r in recs]))
    peaks, peak_kind = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    roof = None
    if k_ms > 0:
        ach = k_bytes / (k_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": TRAFFIC_BYTES.get(name),
                "kernel": ("solve_large_scc_fxd_k (grid-wide SCC power series, fixed point, z gathered as FP64)"
                           if name == "large" else "solve_large_scc_fx_k (grid-wide SCC power series, fixed point)"),
                "peak_kind": f"{peak_kind} copy bandwidth", "kernel_ms_per_step": k_ms,
                "algorithmic_bytes_per_step": k_bytes}
    out = {
        "workload": WORKLOADS[name] if name != "large" or args.large_n == 50_000_000
        else WORKLOADS["large"].replace("n=50,000,000, ~400M edges", f"n={args.large_n:,}"),
        "n": n, "nnz": E, "generate_s": t_gen, "steps": steps, "warmup": 3,
        "value": E / (t_step * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": t_step,
        "breakdown_ms": {"graph_prepare": float(ph[:, 0].mean()), "partition": float(ph[:, 1].mean()),
                         "solve": t_solve, "residual_check": float(ph[:, 3].mean())},
        "partition_phases": part_phases,
        "global_power": {"ms_per_step": t_global, "solve_ms": t_global_solve, "iters": g_iters,
                         "value": E / (t_global * 1e-3) / 1e9},
        "speedup_vs_global": {"step": t_global / t_step, "solve_only": t_global_solve / t_solve},
        "solve": {"iters_max": st["iters_max"], "levels": P.n_levels, "components": P.n_comp,
                  "scc_components": P.n_scc, "edge_visits": st["edge_visits"],
                  "residual_l1": max(r[2] for r in recs), "sweeps": sweeps},
        "mixed_precision": {"solve_ms": t_mixed, "residual_l1": m_res, "iters_max": stm["iters_max"],
                            "fp64_sweeps_max": stm["fp64_sweeps_max"],
                            "fp64_replay_solve_ms": t_fp64r,
                            "solve_speedup_vs_fp64": t_fp64r / t_mixed,
                            "solve_speedup_vs_global": t_global_solve / t_mixed,
                            "l1_diff_vs_fp64": float((Rm - R64).abs().sum().item()),
                            "max_rel_vs_fp64": float(((Rm - R64).abs() / R64.abs().clamp_min(1e-300)).max().item())},
        "roofline": roof, "autotune": tuned,
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
    }
    keep = {"rowptr": rowptr, "col": col, "u": u, "layers": layers, "R64": R64, "Rm": Rm,
            "comp": comp_d, "iters": np.asarray(st["comp_iters"])}
    return out, keep


def block_vs_oracle(name, keep):
    """The block's FP64 and mixed results against the oracle on the host:
    the whole graph for deep_dag; for the 50M-vertex graph (far beyond a
    single-thread oracle run) the vertices of its first planted layers, a set
    closed under predecessors, solved on that slice with every leaving edge
    kept as an edge to a dangling dummy (graphgen.closed_slice), so that
    their solution is that of the whole graph."""
    rowptr = keep["rowptr"].cpu().numpy()
    col = keep["col"].cpu().numpy()
    u = keep["u"].cpu().numpy()
    comp = keep["comp"].cpu().numpy()
    R64 = keep["R64"].cpu().numpy()
    Rm = keep["Rm"].cpu().numpy()
    n = u.shape[0]
    if name == "large":
        lay = keep["layers"].cpu().numpy()
        counts = np.bincount(lay.astype(np.int64), minlength=int(lay.max()) + 1)
        target = min(4_000_000, n // 10)  # about ten seconds of oracle work on the host
        L = max(1, int(np.searchsorted(np.cumsum(counts), target, side="right")))
        rp, cl, us, ids = gg.closed_slice(rowptr, col, u, lay < L)
        del rowptr, col
        rep, R_or = oracle_vs(rp, cl, us, TOL, R64[ids], comp, keep["iters"], ids=ids,
                              tol_scale=us.shape[0] / n)
        Rm_s = Rm[ids]
        sample = (f"the vertices of planted layers 0-{L - 1} ({ids.shape[0]:,} of {n:,}), closed under "
                  f"predecessors; leaving edges kept as edges to {us.shape[0] - ids.shape[0]:,} dangling dummies")
    else:
        rep, R_or = oracle_vs(rowptr, col, u, TOL, R64, comp, keep["iters"])
        Rm_s = Rm
        sample = "whole graph"
    # the mixed-precision result against the oracle's FP64 one (own rules)
    rep["mixed_own_rule"] = dict(diff_fields(Rm_s, R_or), l1_bound=2 * TOL / (1 - C))
    rep["sample"] = sample
    return rep


def run_ours(args):
    import torch

    import paper_1609_09068_gb300 as prgb
    from paper_1609_09068_gb300 import _build

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if not _build.up_to_date():
        _build.build()
    prgb.load_library()

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks_(x):
        return max_over_ranks(dist, x, "cuda")

    g = load_workload(args.workload, args.large_n)
    E = g.nnz
    if isinstance(g, _DeviceGraph):
        rowptr, col, u = g.rowptr_d, g.col_d, g.u_d
    else:
        rowptr = torch.from_numpy(g.rowptr).cuda()
        col = torch.from_numpy(g.col).cuda()
        u = torch.from_numpy(g.u).cuda()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def ev():
        return torch.cuda.Event(enable_timing=True)

    cw_step, global_step = make_steps(prgb, rowptr, col, u)

    # one-time autotuning of the solve's launch shapes (pr_partition_tune);
    # partitions built in the timed steps start from its choice
    tuned = prgb.partition(prgb.graph(rowptr, col)).tune(C, u, TOL)
    for _ in range(args.warmup):
        cw_step()
        global_step()
    torch.cuda.synchronize()

    # ---- componentwise: the timed region -----------------------------------
    clocks = Clocks(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    l0 = prgb.launch_count()
    recs = []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)  # 256 MiB write: the graph leaves L2 before each step
        recs.append(cw_step())
    torch.cuda.synchronize()
    barrier()
    launches = prgb.launch_count() - l0
    clk = clocks.stop()
    phase = np.array([[recs[i][0][j].elapsed_time(recs[i][0][j + 1]) for j in range(4)]
                      for i in range(args.steps)])
    t_step = max_over_ranks_(float(phase.sum(axis=1).mean()))
    stats = [r[1] for r in recs]
    residual = max(r[2] for r in recs)
    P = recs[-1][3]
    value = job_value(E, world, t_step)
    counted = counted_stats(prgb, P, u)  # sweep counts and edge visits, outside the timed region

    # ---- global power series on the same GPU --------------------------------
    grecs = []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        grecs.append(global_step())
    torch.cuda.synchronize()
    gph = np.array([[grecs[i][0][j].elapsed_time(grecs[i][0][j + 1]) for j in range(3)]
                    for i in range(args.steps)])
    t_global = max_over_ranks_(float(gph.sum(axis=1).mean()))
    t_global_solve = float(gph[:, 1].mean())
    g_iters = grecs[-1][3]
    g_res = max(r[2] for r in grecs)
    gk_ms = float(np.mean([r[1]["kernel_ms"] for r in grecs]))
    gk_bytes = float(np.mean([r[1]["kernel_bytes"] for r in grecs]))

    part_phases = partition_phases(prgb, rowptr, col, flush)

    # sweeps per SCC against the global series' (outside the timed regions)
    try:
        comp_d, type_d, _ = P.query()
        sweeps = sweep_stats(comp_d, type_d, rowptr, col, counted["comp_iters"], g_iters)
        del comp_d, type_d
    except Exception as e:  # a report field only: never lose the bench line
        sweeps = {"unavailable": f"{type(e).__name__}: {str(e)[:200]}"}

    # ---- mixed precision (FP32 SCC series + FP64 residual refinement) ------
    # the solve alone, on the partition of the timed steps, against the FP64
    # result of the same partition
    R64 = prgb.solve(P, C, u, TOL)
    # mixed precision against FP64 on the same partition, both replayed from
    # their CUDA graphs (the timed steps' solve is each new partition's first)
    t_fp64r, _ = replay_ms(prgb, P, u, flush, args.steps, prgb.PREC_FP64)
    t_fp64r = max_over_ranks_(t_fp64r)
    t_mixed, mrecs = replay_ms(prgb, P, u, flush, args.steps, prgb.PREC_MIXED)
    t_mixed = max_over_ranks_(t_mixed)
    stm, Rm = counted_stats(prgb, P, u, prgb.PREC_MIXED), mrecs[-1][3]
    m_res = prgb.residual_l1(prgb.graph(rowptr, col), C, u, Rm)
    m_diff = float((Rm - R64).abs().sum().item())
    m_rel = float(((Rm - R64).abs() / R64.abs().clamp_min(1e-300)).max().item())
    mk_ms = float(np.mean([r[2]["kernel_ms"] for r in mrecs]))
    mk_bytes = float(np.mean([r[2]["kernel_bytes"] for r in mrecs]))
    mixed = {"solve_ms": t_mixed, "residual_l1": m_res, "iters_max": stm["iters_max"],
             "fp64_sweeps_max": stm["fp64_sweeps_max"],
             "fp64_edge_share": stm["fp64_edge_visits"] / max(stm["edge_visits"], 1),
             "l1_diff_vs_fp64": m_diff, "max_rel_vs_fp64": m_rel,
             "fp64_replay_solve_ms": t_fp64r,
             "solve_speedup_vs_fp64": t_fp64r / t_mixed,
             "solve_speedup_vs_global": t_global_solve / t_mixed,
             "giant_kernel_ms": mk_ms,
             "giant_kernel_gbs": mk_bytes / (mk_ms * 1e-3) / 1e9 if mk_ms > 0 else None}

    # ---- end to end through the C ABI with host buffers ---------------------
    hr, hc, hu_ = g.host() if isinstance(g, _DeviceGraph) else (g.rowptr, g.col, g.u)
    rp_h = torch.from_numpy(hr).pin_memory().numpy()
    col_h = torch.from_numpy(hc).pin_memory().numpy()
    u_h = torch.from_numpy(hu_).pin_memory().numpy()
    e2e_ms = []
    for k in range(args.warmup + args.steps):  # the first W steps untimed
        flush.fill_(k & 0xFF)
        a, b = ev(), ev()
        a.record()
        Gh = prgb.graph(rp_h, col_h, on_host=True)
        Ph = prgb.partition(Gh)
        Rh = prgb.solve(Ph, C, u_h, TOL)
        b.record()
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e_ms.append(a.elapsed_time(b))
        assert isinstance(Rh, np.ndarray)
    t_e2e = max_over_ranks_(float(np.mean(e2e_ms)))
    h2d = rp_h.nbytes + col_h.nbytes + u_h.nbytes
    d2h = u_h.nbytes

    # ---- roofline of the dominant SpMV kernel --------------------------------
    # The grid-wide power series (the largest share of the solve).  On the
    # web-like graph (n = 1M) its sweep's working set stays in the 126 MB L2
    # (ncu: ~30 MB of DRAM traffic per launch against ~2 GB of algorithmic
    # bytes), so the bound reported is L2 bandwidth, measured live; the
    # fraction of HBM is kept beside it.  The 50M-vertex block reports HBM.
    peaks, peak_kind = measured_peaks()
    k_ms = float(np.mean([s["kernel_ms"] for s in stats]))
    k_bytes = float(np.mean([s["kernel_bytes"] for s in stats]))
    achieved = k_bytes / (k_ms * 1e-3) / 1e9 if k_ms > 0 else 0.0
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    l2 = measured_l2_gbs()
    in_l2 = args.workload in ("web", "small")
    peak = l2 if in_l2 else hbm
    roofline = {"bound": "l2" if in_l2 else "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": TRAFFIC_BYTES.get(args.workload),
                "kernel": "solve_large_scc_fx_k (grid-wide SCC power series, fixed point)",
                "peak_kind": ("L2 bandwidth measured live (64 MiB resident: FP32 sum or 32 MiB copy, the larger)"
                              if in_l2 else f"{peak_kind} copy bandwidth"),
                "hbm_peak": hbm, "hbm_frac": achieved / hbm, "hbm_peak_kind": f"{peak_kind} copy bandwidth",
                "kernel_ms_per_step": k_ms, "algorithmic_bytes_per_step": k_bytes,
                "launches_per_step": float(np.mean([s["kernel_launches"] for s in stats]))}

    # ---- CPU oracle on the host cores ---------------------------------------
    # one full oracle step (partition + componentwise solve, single thread)
    # timed, and the GPU's FP64 result compared with it: each side stopping by
    # its own rule (L1 bound 2 tol / (1 - c)) and with the GPU's sweep counts
    # replayed (rounding only: 1e-12 per entry)
    cpu = None
    vs_oracle = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload != "large":
        try:
            comp_h, _, _ = P.query()
            vs_oracle, _ = oracle_vs(g.rowptr, g.col, g.u, TOL, R64.double().cpu().numpy(), comp_h.cpu().numpy(),
                                     np.asarray(counted["comp_iters"]))
            t_cpu = vs_oracle["oracle_partition_s"] + vs_oracle["oracle_solve_s"]
            cpu = {"value": E / t_cpu / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": "one full step of the same workload: oracle partition (Tarjan DFS) + "
                             f"componentwise solve, single thread, {t_cpu:.1f} s"}
        except Exception as e:  # a report field only: never lose the bench line
            vs_oracle = {"unavailable": f"{type(e).__name__}: {str(e)[:200]}"}
    # ---- multi-core CPU baseline (OpenMP) on the host cores ------------------
    cpu_par = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload != "large":
        cpu_par = cpu_parallel_leg(args)
        if "cw_solve_ms" in cpu_par:
            cpu_par["gpu_speedup"] = {"cw_solve": cpu_par["cw_solve_ms"] / float(np.mean(phase[:, 2])),
                                      "global_solve": cpu_par["global_solve_ms"] / t_global_solve}

    ph = phase.mean(axis=0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload] if args.workload != "large" or args.large_n == 50_000_000
                   else WORKLOADS["large"].replace("n=50,000,000, ~400M edges", f"n={args.large_n:,}"),
                   "n": g.n, "nnz": E, "c": C, "tol": TOL,
                   "norm": "L1", "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed before each step by a 256 MiB device write outside the timed events"},
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
        "e2e": {"value": job_value(E, world, t_e2e), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": t_e2e},
        "gpu_launches": launches,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "cpu_parallel": cpu_par,
        "breakdown_ms": {"graph_prepare": float(ph[0]), "partition": float(ph[1]),
                         "solve": float(ph[2]), "residual_check": float(ph[3])},
        "partition_phases": part_phases,
        "solve": {"iters_max": counted["iters_max"], "levels": P.n_levels,
                  "components": P.n_comp, "scc_components": P.n_scc,
                  "edge_visits": counted["edge_visits"],
                  "traversed_gteps": counted["edge_visits"] / (ph[2] * 1e-3) / 1e9,
                  "equivalent_gteps": E * g_iters / (ph[2] * 1e-3) / 1e9,
                  "sweeps": sweeps,
                  "residual_l1": residual, "vs_oracle": vs_oracle},
        "global_power": {"ms_per_step": t_global, "solve_ms": t_global_solve, "iters": g_iters,
                         "value": job_value(E, world, t_global), "residual_l1": g_res,
                         "kernel_gbs": gk_bytes / (gk_ms * 1e-3) / 1e9 if gk_ms > 0 else None},
        "speedup_vs_global": {"step": t_global / t_step, "solve_only": t_global_solve / float(ph[2])},
        "autotune": tuned,
        "mixed_precision": mixed,
    }
    # ---- the other configurations, each timed the same way ------------------
    # deep_dag (n = 4M, 200 levels) and the 50M-vertex web-like graph (FP64
    # and mixed precision), after the headline's timed regions
    if world == 1 and args.workload == "web" and not args.no_blocks:
        del recs, grecs, mrecs
        for name, key in (("deep", "deep_dag"), ("large", "large")):
            try:
                blk, kept = config_block(prgb, name, args, flush, local)
                if not args.no_cpu_baseline:
                    try:
                        blk["vs_oracle"] = block_vs_oracle(name, kept)
                    except Exception as e:  # a report field only
                        blk["vs_oracle"] = {"unavailable": f"{type(e).__name__}: {str(e)[:200]}"}
                del kept
            except Exception as e:  # a report block only: never lose the bench line
                blk = {"unavailable": f"{type(e).__name__}: {str(e)[:300]}"}
            line[key] = blk
            torch.cuda.empty_cache()
    if rank == 0:
        print(json.dumps(line), flush=True)
        print(json.dumps({"phase_ms_per_step": np.round(phase, 3).tolist(),
                          "global_ms_per_step": np.round(gph, 3).tolist(),
                          "e2e_ms": np.round(e2e_ms, 3).tolist()}), file=sys.stderr)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def warm_eval(args):
    """The learned warm start as the deep-DAG warm-start setting specifies it:
    a 2-layer message-passing net (hidden 64, bf16 weights, FP32 sums) is
    trained with the library's kernels on plain-solver PageRank (L1 residual
    1e-12) of seeded deep_dag graphs with n = 100,000, then each held-out
    deep_dag graph with n = 4,000,000 (200 levels) is solved to 1e-10 cold and
    warm.  The training graphs keep the held-out graphs' layer size (n / levels
    = 20,000 vertices, so 5 levels), hence the same per-level mix of SCCs and
    chains.  Graphs are generated on the host cores by a process pool started
    before any CUDA work.  One JSON line: solve time and sweeps, cold vs warm,
    per held-out seed and summarised; the warm results are judged by their
    residual."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    n_train, n_held = 100_000, 4_000_000
    train_specs = [(100_000 + i, n_train, n_train // 20_000) for i in range(args.warm_train)]
    held_specs = [(200_000 + i, n_held, 200) for i in range(args.warm_held)]
    t_all = time.time()
    with ctx.Pool(max(1, min(16, (os.cpu_count() or 2) - 1))) as pool:
        train_it = pool.imap(gg.deep_dag_arrays, train_specs, chunksize=4)
        held_it = pool.imap(gg.deep_dag_arrays, held_specs, chunksize=1)
        import torch
        import paper_1609_09068_gb300 as prgb
        prgb.load_library()
        model = prgb.Mpnn(seed=3)
        t0 = time.time()
        losses = []
        for i, (rp, cl, u) in enumerate(train_it):
            G = prgb.graph(torch.from_numpy(rp).cuda(), torch.from_numpy(cl).cuda())
            P = prgb.partition(G)
            ud = torch.from_numpy(u).cuda()
            R = prgb.solve(P, C, ud, 1e-12)
            lr = 3e-3 if i < len(train_specs) // 2 else 1e-3
            for _ in range(2):
                losses.append(model.train_step(P, C, ud, R, lr=lr))
            P.close()
            G.close()
        t_train = time.time() - t0
        ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
        seeds = []
        for (sd, _, _), (rp, cl, u) in zip(held_specs, held_it):
            G = prgb.graph(torch.from_numpy(rp).cuda(), torch.from_numpy(cl).cuda())
            P = prgb.partition(G)
            ud = torch.from_numpy(u).cuda()
            rec = {"seed": sd}
            for mode in ("cold", "warm"):
                wm = model if mode == "warm" else None
                R, st = prgb.solve(P, C, ud, TOL, with_stats=True, warm_start=wm)  # builds the graph, untimed
                ts = []
                for _ in range(3):
                    a, b = ev(), ev()
                    a.record()
                    R, st = prgb.solve(P, C, ud, TOL, with_stats=True, warm_start=wm)
                    b.record()
                    torch.cuda.synchronize()
                    ts.append(a.elapsed_time(b))
                rec[mode] = {"solve_ms": statistics.median(ts), "iters_max": st["iters_max"],
                             "edge_visits": st["edge_visits"], "residual_l1": prgb.residual_l1(G, C, ud, R)}
            # the guess is computed once per partition and model version;
            # re-setting the weights forces it, so this solve pays for it
            model.set_params(model.get_params())
            a, b = ev(), ev()
            a.record()
            prgb.solve(P, C, ud, TOL, warm_start=model)
            b.record()
            torch.cuda.synchronize()
            rec["warm"]["solve_ms_with_guess"] = a.elapsed_time(b)
            rec["speedup"] = rec["cold"]["solve_ms"] / rec["warm"]["solve_ms"]
            rec["speedup_with_guess"] = rec["cold"]["solve_ms"] / rec["warm"]["solve_ms_with_guess"]
            seeds.append(rec)
            P.close()
            G.close()
    sp = [r["speedup"] for r in seeds]
    spg = [r["speedup_with_guess"] for r in seeds]
    line = {
        "metric": "learned warm start: solve time to L1 residual 1e-10, cold / warm (deep_dag, 1 GB300)",
        "value": statistics.mean(spg) if spg else None, "unit": "x (cold ms / warm ms incl. the guess)",
        "higher_is_better": True, "speedup_guess_cached": statistics.mean(sp) if sp else None,
        "data": "synthetic", "dtype": "f64",
        "config": {"workload": "deep_dag warm start: train %d graphs n=100,000 (5 levels of 20,000), held-out %d "
                               "graphs n=4,000,000 (200 levels), c=0.85, L1 tol 1e-10, FP64" %
                               (len(train_specs), len(held_specs)),
                   "model": "2-layer MPNN, hidden 64, bf16 weights, FP32 sums, Adam, 2 steps per graph"},
        "train": {"graphs": len(train_specs), "seconds": t_train, "loss_first": losses[0] if losses else None,
                  "loss_last_100_mean": float(np.mean(losses[-100:])) if losses else None},
        "held_out": {"graphs": len(seeds), "speedup_min": min(sp) if sp else None,
                     "speedup_max": max(sp) if sp else None,
                     "solve_ms_cold_mean": statistics.mean(r["cold"]["solve_ms"] for r in seeds),
                     "solve_ms_warm_mean": statistics.mean(r["warm"]["solve_ms"] for r in seeds),
                     "solve_ms_warm_with_guess_mean": statistics.mean(r["warm"]["solve_ms_with_guess"]
                                                                      for r in seeds),
                     "iters_max_cold_mean": statistics.mean(r["cold"]["iters_max"] for r in seeds),
                     "iters_max_warm_mean": statistics.mean(r["warm"]["iters_max"] for r in seeds),
                     "edge_visits_ratio_mean": statistics.mean(r["warm"]["edge_visits"] / r["cold"]["edge_visits"]
                                                               for r in seeds),
                     "residual_l1_warm_max": max(r["warm"]["residual_l1"] for r in seeds)},
        "per_seed": seeds, "total_seconds": time.time() - t_all,
    }
    print(json.dumps(line), flush=True)
    return 0


def profile_solves(args):
    """A short run for profilers: graph, partition, the launch shape, then
    --profile-solves FP64 solves (one launch of the grid-wide SCC kernel per
    large SCC and one level-kernel launch per level each); one line out."""
    import torch
    import paper_1609_09068_gb300 as prgb
    prgb.load_library()
    g = load_workload(args.workload, args.large_n)
    if isinstance(g, _DeviceGraph):
        rp, cl, u = g.rowptr_d, g.col_d, g.u_d
    else:
        rp, cl, u = (torch.from_numpy(x).cuda() for x in (g.rowptr, g.col, g.u))
    G = prgb.graph(rp, cl)
    P = prgb.partition(G)
    if args.shape:
        cm, cb, bl = (int(x) for x in args.shape.split(","))
        P.set_shape(cm, cb, bl)
        shape = {"cta_max": cm, "coop_blocks": cb, "balance": bl}
    else:
        shape = P.tune(C, u, TOL)
    for _ in range(args.profile_solves):
        R = prgb.solve(P, C, u, TOL)
    # one more, timed (it comes after the launches a profiler captures with -s/-c)
    R, st = prgb.solve(P, C, u, TOL, with_stats=True, timing=True)
    torch.cuda.synchronize()
    print(json.dumps({"workload": args.workload, "solves": args.profile_solves, "shape": shape,
                      "levels": P.n_levels, "residual_l1": prgb.residual_l1(G, C, u, R),
                      "grid_scc_kernel": {"launches": st["kernel_launches"], "ms": st["kernel_ms"],
                                          "algorithmic_bytes": st["kernel_bytes"]}}), flush=True)
    return 0


def partition_io(args):
    """Partition files: for each graph, the wall time of pr_partition_create
    against pr_partition_save and pr_partition_load of the same partition
    (each call synchronises; medians of 5 calls, 3 for the large graph, after
    one untimed call of each), the file's size, and whether the loaded
    partition equals the created one."""
    import torch
    import paper_1609_09068_gb300 as prgb
    prgb.load_library()

    def med(f, k):
        ts = []
        for _ in range(k):
            torch.cuda.synchronize()
            t = time.perf_counter()
            r = f()
            ts.append((time.perf_counter() - t) * 1e3)
        return statistics.median(ts), r

    out = {}
    for name in ("web", "deep", "large"):
        try:
            if name == "large":
                from graphgen.large import web_like_device
                rowptr, col, _ = web_like_device(seed=4, n=args.large_n)
            else:
                g = gg.config(name)
                rowptr, col = torch.from_numpy(g.rowptr).cuda(), torch.from_numpy(g.col).cuda()
            G = prgb.graph(rowptr, col)
            k = 3 if name == "large" else 5
            with tempfile.TemporaryDirectory() as d:
                path = os.path.join(d, "part.bin")
                P = prgb.partition(G)
                create_ms, P = med(lambda: prgb.partition(G), k)
                P.save(path)
                save_ms, _ = med(lambda: P.save(path), k)
                prgb.load_partition(G, path)
                load_ms, L = med(lambda: prgb.load_partition(G, path), k)
                same = all(bool(torch.equal(a, b)) for a, b in zip(P.query(), L.query()))
                out[name] = {"n": int(rowptr.numel() - 1), "edges": int(col.numel()),
                             "create_ms": round(create_ms, 2), "save_ms": round(save_ms, 2),
                             "load_ms": round(load_ms, 2), "file_bytes": os.path.getsize(path),
                             "loaded_equals_created": same}
            del G, P, L, rowptr, col
            torch.cuda.empty_cache()
        except Exception as e:  # report the failure, keep the other graphs
            out[name] = {"unavailable": f"{type(e).__name__}: {str(e)[:200]}"}
    print(json.dumps({"metric": "partition_io", "unit": "ms", "graphs": out}), flush=True)
    return 0


def main():
    args = parse()
    if args.partition_io:
        return partition_io(args)
    if args.profile_solves > 0:
        return profile_solves(args)
    if args.cpu_parallel_worker:
        return cpu_parallel_worker(args)
    if args.warm_eval:
        return warm_eval(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
