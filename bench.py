#!/usr/bin/env python3
"""Benchmark of the batched AGP push on one GB300 (or N replicas).

Workload (the batched Katz / transition-probability configuration): Chung-Lu power-law graph,
exponent 2.1, 4,000,000 nodes, 120,000,000 distinct undirected edges (a synthetic stand-in for the
paper's Orkut/YouTube-class social graphs). One step = one launch of 256 Katz queries
(a = b = 0, w_i = beta^i, beta = 0.85 / lambda_1 with lambda_1 from the library's FP64 power
iteration, L = 20) plus one launch of 256 L-hop transition-probability queries (a = 0, b = 1,
w_4 = 1, L = 4), eps = 1e-8, from 256 degree-weighted random sources each (fresh sources every
step, fixed seeds). Metric: queries per second, whole job.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl agp|reference] [--small]
Prints one JSON line (rank 0). Under torchrun (N > 1) every rank runs the same workload on its own
GPU (replicas, weak scaling) and the timing is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import graphs as SG  # noqa: E402

S = 20210603
HBM_FALLBACK_GBS = 6800.0

# Algorithmic bytes per unit of work (roofline numerator), per level-loop step:
#   compaction:             two reads of every active lane's residue vector (4 B per node each) +
#                           per frontier item: item id 4 + r value 4 + clearing 4
#   frontier item (expand): item id 4 + r value 4 + reserve RMW 8 + degree 4 + row start 8
#   deterministic push:     colidx 4 + residue atomic RMW 8 (+ neighbour degree 4 when a > 0)
#   sampler trial:          colidx 4 (+ neighbour degree 4 when a > 0)
#   accepted sample:        residue atomic RMW 8
B_ITEM, B_DET, B_TRIAL, B_ACC, B_DEG, B_COMPACT_ITEM, B_SCAN = 28, 12, 4, 8, 4, 12, 8

# DRAM traffic of k_push per L2 reduction, from one ncu capture with warm caches
# (dram__bytes_read.sum + dram__bytes_write.sum over lts__t_sectors_srcunit_tex_op_red.sum, three
# k_push launches of a step of 64 Katz + 64 transition sources at four lanes per wave; see
# profiles/launch_list_katz_transition_4M.md). It scales a launch of the bench step by its
# reductions, for a four-lane wave only. Per launch it ranged from 16.4 to 26.6 B, so the scaled
# figure is an estimate. It must be re-measured whenever the push kernel changes.
PUSH_DRAM_BYTES_PER_RED, PUSH_TRAFFIC_LANES = 18.3, 4


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------------------------- workload
def workload(small: bool):
    if small:
        return dict(name="rmat-2^14 ppr+transition (small)", n=16384, m=131072, kind="rmat", Q=64, L_katz=20,
                    eps=1e-7, seed_graph=S + 1, seed_src=S + 101)
    return dict(name="chung-lu-2.1 n=4M m=120M katz(L=20)+transition(L=4) x256 sources, eps=1e-8",
                n=4_000_000, m=120_000_000, kind="chung_lu", Q=256, L_katz=20, eps=1e-8,
                seed_graph=S + 2, seed_src=S + 102)


def make_edges(wl):
    if wl["kind"] == "rmat":
        return SG.cached("rmat", SG.rmat_edges, wl["n"], wl["m"], wl["seed_graph"])
    return SG.cached("chunglu", SG.chung_lu_edges, wl["n"], wl["m"], 2.1, wl["seed_graph"])


def atomic_ceiling(g, lanes, n, count=1 << 27, reps=5):
    """Random FP32 atomic-add throughput (adds/s) into a buffer the size of one wave's residue
    vectors (lanes x n floats, which fit in L2), measured with torch's index_add_ (a library scatter
    kernel: one atomic add per element). Two target laws: uniform, and endpoints of uniformly drawn
    edges (probability proportional to degree, as the pushes of a propagation land)."""
    import torch
    _, colidx, _ = g.csr()
    lanes = max(int(lanes), 1)
    size = lanes * n
    buf = torch.zeros(size, dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(S + 300)
    vals = torch.full((count,), 1e-8, dtype=torch.float32, device="cuda")
    targets = {"uniform": torch.randint(0, size, (count,), generator=gen, device="cuda")}
    pos = torch.randint(0, colidx.numel(), (count,), generator=gen, device="cuda")
    lane_of = torch.randint(0, lanes, (count,), generator=gen, device="cuda")
    targets["degree_weighted"] = colidx[pos].long() + lane_of * n
    del pos, lane_of
    out = {}
    for name, idx in targets.items():
        for _ in range(2):
            buf.index_add_(0, idx, vals)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            buf.index_add_(0, idx, vals)
        e1.record()
        e1.synchronize()
        out[name] = count * reps / (e0.elapsed_time(e1) / 1e3)
    return out


def degree_weighted_sources(n, u, v, count, seed):
    deg = np.bincount(u, minlength=n) + np.bincount(v, minlength=n)
    p = deg / deg.sum()
    rng = np.random.default_rng(seed)
    return rng.choice(n, size=count, p=p).astype(np.int32)


# ------------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="agp_clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = [l.split(",") for l in open(self.path) if l.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------- host description
def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the CPU baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ------------------------------------------------------------------------------- oracle baseline
def oracle_sample(og, n, sources, eps, L=4, threads=None):
    """Time the FP64 oracle (Algorithm 2, as it stands) on transition queries in parallel threads."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    w, Y = oracle.tail_sums(oracle.TRANSITION, L)
    threads = threads or min(len(sources), host_cores())

    def one(s):
        x = np.zeros(n)
        x[s] = 1.0
        return oracle.randomized(og, 0, 1, L, w, Y, eps, x, int(s))

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(one, [int(s) for s in sources[:threads]]))
    dt = time.perf_counter() - t0
    return threads, dt


def run_reference(args, wl, rank):
    """Reference arm: the FP64 oracle on the host cores, same workload, bounded sample per step."""
    if rank != 0:
        return
    u, v = make_edges(wl)
    n = wl["n"]
    srcs = degree_weighted_sources(n, u, v, wl["Q"] * 2 * (args.warmup + args.steps), wl["seed_src"])
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    og = oracle.build_csr(n, u, v)
    w, Y = oracle.tail_sums(oracle.TRANSITION, 4)
    threads = host_cores()

    def one(s):
        x = np.zeros(n)
        x[s] = 1.0
        oracle.randomized(og, 0, 1, 4, w, Y, wl["eps"], x, int(s))

    def step(k, count):
        base = k * 2 * wl["Q"] + wl["Q"]  # the transition half of step k's sources
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(one, [int(s) for s in srcs[base:base + count]]))

    for k in range(args.warmup):
        step(k, 1)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        step(args.warmup + k, threads)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = threads * args.steps / total
    sample = (f"{threads} of the {wl['Q']} L=4 transition queries of each step, one per host thread on all "
              f"{threads} cores ({cpu_model()}); the oracle runs per-neighbour Bernoulli trials, and its eps=1e-8 "
              f"Katz queries take minutes each and are left out")
    line = {"impl": "reference", "metric": "queries/s", "value": value, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "l2": "not applicable (CPU)"},
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------- accuracy
def row_accuracy(og, kind, a, b, L, w, Y, eps, s_, row):
    """One GPU result row against the exact FP64 propagation of x = e_s (the oracle's Algorithm 1)."""
    import oracle
    x = np.zeros(og.n)
    x[s_] = 1.0
    exact = oracle.basic(og, a, b, L, w, Y, x)
    res = {"kind": kind, "source": int(s_), "eps": float(eps), "L": int(L)}
    rel = np.abs(row.astype(np.float64) - exact) / np.maximum(exact, 1e-300)
    for name, delta in (("paper", eps * L * (L + 1) / 2 * Y[0]), ("chebyshev", 5000 * L * (L + 1) * eps * Y[0])):
        big = exact >= delta
        res[f"delta_{name}"] = float(delta)
        res[f"nodes_{name}"] = int(big.sum())
        res[f"frac_ok_{name}"] = float(np.mean(rel[big] <= 0.1)) if big.any() else None
    res["rel_l1"] = float(np.abs(row - exact).sum() / np.abs(exact).sum())
    # the paper's measures (appendix, Katz experiments): MaxError = max_v |pi(v) - pi_hat(v)| and
    # Precision@50 = overlap of the 50 largest entries (ties by id)
    res["max_error"] = float(np.abs(row.astype(np.float64) - exact).max())
    top = lambda x: set(np.lexsort((np.arange(x.size), -x))[:50].tolist())
    res["precision_at_50"] = len(top(row.astype(np.float64)) & top(exact)) / 50.0
    # the smallest delta at which >= 99% of the nodes with pi >= delta have relative error <= 0.1
    order = np.argsort(-exact)
    order = order[exact[order] > 0]
    ok = np.cumsum(rel[order] <= 0.1) / np.arange(1, order.size + 1)
    good = np.flatnonzero(ok >= 0.99)
    res["delta_99"] = float(exact[order[good[-1]]]) if good.size else None
    return res


def accuracy_vs_oracle(og, checks, eps, beta, L_katz, threads):
    """Relative error of GPU results against the exact FP64 propagation (the oracle's Algorithm 1).
    checks: list of (kind, source, gpu_row). Reported per query: the fraction of nodes with
    pi(v) >= delta whose relative error is <= 0.1, at the paper's experimental delta = eps L(L+1)/2
    (times Y_0) and at the Chebyshev delta 5000 L(L+1) eps Y_0 of Lemma 4.2, and the relative L1
    error. The oracle runs on the host outside the timed region."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    n = og.n
    tables = {"katz": (0.0, 0.0, L_katz) + oracle.tail_sums(oracle.KATZ, L_katz, beta),
              "transition": (0.0, 1.0, 4) + oracle.tail_sums(oracle.TRANSITION, 4)}

    def one(item):
        kind, s_, row = item
        a, b, L, w, Y = tables[kind]
        return row_accuracy(og, kind, a, b, L, w, Y, eps, s_, row)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=max(1, min(threads, len(checks)))) as ex:
        per = list(ex.map(one, checks))
    secs = time.perf_counter() - t0
    summ = {}
    for name in ("paper", "chebyshev"):
        vals = [r[f"frac_ok_{name}"] for r in per if r[f"frac_ok_{name}"] is not None]
        summ[f"frac_ok_at_delta_{name}"] = {"min": float(min(vals)) if vals else None,
                                           "mean": float(np.mean(vals)) if vals else None,
                                           "queries": len(vals)}
    summ["rel_l1_max"] = float(max(r["rel_l1"] for r in per))
    summ["max_error_max"] = float(max(r["max_error"] for r in per))
    summ["precision_at_50_min"] = float(min(r["precision_at_50"] for r in per))
    for kind in ("katz", "transition"):
        d99 = [r["delta_99"] for r in per if r["kind"] == kind and r["delta_99"] is not None]
        summ[f"delta_99_{kind}"] = {"max": float(max(d99)) if d99 else None,
                                    "median": float(np.median(d99)) if d99 else None}
    summ["queries_checked"] = len(per)
    summ["oracle_s"] = secs
    summ["per_query"] = per
    return summ


def latency_summary(ms):
    ms = np.asarray(ms, np.float64)
    return {"p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
            "max_ms": float(ms.max()), "queries": int(ms.size)}


# ------------------------------------------------------------------------------- multi-rank
def rank_reduce(x: float, op: str, world: int, device: str = "cpu") -> float:
    """max / sum of a scalar over all ranks (identity for a single process)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(local_ms: float, local_units: float, world: int, device: str = "cpu"):
    """Whole-job rate: units summed over ranks / the slowest rank's time. Returns (ms, units, rate)."""
    ms = rank_reduce(local_ms, "max", world, device)
    units = rank_reduce(local_units, "sum", world, device)
    return ms, units, units / (ms / 1e3)


def end_to_end(agp, g, args, all_params, srcs, Q, n, world, dev):
    """The same steps through host buffers: H2D of the sources and D2H of all results timed."""
    import torch
    h_srcs = srcs.copy()
    h_off = np.arange(Q + 1, dtype=np.int64)
    h_out_k = torch.empty((Q, n), dtype=torch.float32, pin_memory=True)
    h_out_t = torch.empty((Q, n), dtype=torch.float32, pin_memory=True)
    e2e_times = []
    # one untimed step through the host path first (its staging buffers are allocated on first use)
    pk, pt = all_params[max(args.warmup - 1, 0)]
    base = max(args.warmup - 1, 0) * 2 * Q
    agp.query_batch(g, pk, h_off, h_srcs[base:base + Q], None, h_out_k, n, 0)
    agp.query_batch(g, pt, h_off, h_srcs[base + Q:base + 2 * Q], None, h_out_t, n, 0)
    torch.cuda.synchronize()
    for k in range(args.steps):
        pk, pt = all_params[args.warmup + k]
        base = (args.warmup + k) * 2 * Q
        t0 = time.perf_counter()
        agp.query_batch(g, pk, h_off, h_srcs[base:base + Q], None, h_out_k, n, 0)
        agp.query_batch(g, pt, h_off, h_srcs[base + Q:base + 2 * Q], None, h_out_t, n, 0)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    _, _, e2e_value = job_throughput(1e3 * sum(e2e_times), 2 * Q * args.steps, world, dev)
    h2d = 2 * (h_off.nbytes + Q * 4)
    d2h = 2 * Q * n * 4

    return e2e_value, h2d, d2h


# ------------------------------------------------------------------------------- features
def run_features(args):
    """GNN feature propagation: every column of a BF16 feature matrix is a graph signal."""
    import torch
    import paper_2106_03058_gb300 as agp
    n, m, d = 2_500_000, 60_000_000, 128
    if args.small:
        n, m, d = 16384, 131072, 32
    u, v = SG.cached("rmat", SG.rmat_edges, n, m, S + 3)
    g = agp.build_graph(n, u, v, add_self_loops=True)
    X = torch.randn(n, d, generator=torch.Generator().manual_seed(S + 203)).to(torch.bfloat16).cuda()
    Z = torch.empty((n, d), dtype=torch.float32, device="cuda")
    eps = args.eps if args.eps > 0 else 1e-6
    models = {"appnp": agp._params(0.5, 0.5, 10, agp.W_PPR, 0.1, eps=eps, seed=S + 7),
              "sgc": agp._params(0.5, 0.5, 4, agp.W_TRANSITION, eps=eps, seed=S + 8)}
    # the accuracy / time trade-off of eps (the configuration's eps plus tighter ones and exact)
    sweep_eps = [eps, eps / 10, eps / 100, 0.0] if not args.small else [eps, 0.0]
    for name in ("appnp", "sgc"):
        base = models[name]
        for e in sweep_eps[1:]:
            models[f"{name}_eps{e:g}"] = agp._params(0.5, 0.5, base.L, base.kind, base.param, eps=e, seed=base.seed)
    out = {}
    for name, p in models.items():
        for _ in range(args.warmup):
            agp.feature_propagate(g, p, X, Z)
        torch.cuda.synchronize()
        times = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            agp.feature_propagate(g, p, X, Z)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = float(np.median(times))
        out[name] = {"ms_per_matrix": ms, "columns_per_s": d / (ms / 1e3), "L": p.L}
    # CPU baseline: the FP64 oracle (Algorithm 1, exact) on two columns of each weight sequence, one
    # host thread, timed without caching; the same run gives the GPU's error on those columns
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        og = oracle.build_csr(n, u, v, add_self_loops=True)
        Xh = X[:, :2].float().cpu().numpy().astype(np.float64)
        exact_of, secs = {}, 0.0
        for kind, L, param in ((oracle.PPR, models["appnp"].L, models["appnp"].param),
                               (oracle.TRANSITION, models["sgc"].L, 0.0)):
            w, Y = oracle.tail_sums(kind, L, param)
            for c in range(2):
                t0 = time.perf_counter()
                exact_of[(kind, L, c)] = oracle.basic(og, 0.5, 0.5, L, w, Y, Xh[:, c])
                secs += time.perf_counter() - t0
        errors = {}
        for name, p in models.items():
            agp.feature_propagate(g, p, X, Z)
            Zh = Z[:, :2].cpu().numpy().astype(np.float64)
            kind = oracle.PPR if p.kind == agp.W_PPR else oracle.TRANSITION
            errs = []
            for c in range(2):
                exact = exact_of[(kind, p.L, c)]
                errs.append({"rel_l1": float(np.abs(Zh[:, c] - exact).sum() / np.abs(exact).sum()),
                             "max_abs_over_max": float(np.abs(Zh[:, c] - exact).max() / np.abs(exact).max())})
            out[name]["error_vs_fp64_oracle"] = errs
            errors[name] = errs
        cpu = {"value": 4 / secs, "unit": "columns/s", "cores": 1, "kind": "oracle",
               "sample": "2 columns x (APPNP L=10, SGC L=4), FP64 Algorithm 1 (exact) on one host thread "
                         f"({secs:.1f}s; CSR build excluded)"}
    total_cols = 2 * d  # headline: the configuration's two models at the configuration's eps
    total_ms = out["appnp"]["ms_per_matrix"] + out["sgc"]["ms_per_matrix"]
    line = {"metric": "feature columns/s", "value": total_cols / (total_ms / 1e3), "unit": "columns/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "bf16-in/f32", "data": "synthetic",
            "config": {"workload": f"rmat n={n} m={m} + self-loops, X {n}x{d} bf16 N(0,1), eps={eps} per column part",
                       "models": {k: {"a": 0.5, "b": 0.5, "L": models[k].L, "eps": models[k].eps} for k in models}},
            "models": out, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    g.destroy()


# ------------------------------------------------------------------------------- large graph
def run_large(args):
    """Large single-source PPR and heat-kernel PPR: Chung-Lu exponent 2.0, 65M nodes, 1.8B edges
    (a synthetic stand-in for Friendster), 64 uniform sources, eps = 1e-8, L = 30."""
    import torch
    import paper_2106_03058_gb300 as agp
    n, m, Q = 65_000_000, 1_800_000_000, 64
    if args.small:
        n, m, Q = 1_000_000, 20_000_000, 16
    t0 = time.perf_counter()
    log(f"[large] drawing a Chung-Lu graph n={n} m={m} on the GPU")
    u, v = SG.chung_lu_edges_cuda(n, m, 2.0, S + 4, log=log)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    torch.cuda.empty_cache()  # the builder allocates with cudaMalloc, outside torch's cache
    deg_expected = torch.zeros(n, dtype=torch.int64, device="cuda")
    for s0 in range(0, m, 1 << 28):  # chunks below 2^31 elements
        deg_expected += torch.bincount(u[s0:s0 + (1 << 28)].long(), minlength=n)
        deg_expected += torch.bincount(v[s0:s0 + (1 << 28)].long(), minlength=n)
    log(f"[large] generated in {t_gen:.1f}s; building the CSR")
    u_h, v_h = u.cpu().numpy(), v.cpu().numpy()  # the edge list on the host, for the oracle check
    t0 = time.perf_counter()
    g = agp.build_graph(n, u, v)
    t_build = time.perf_counter() - t0
    del u, v
    torch.cuda.empty_cache()
    log(f"[large] generated {m} edges in {t_gen:.1f}s, built the CSR (nnz={g.nnz}) in {t_build:.1f}s")
    # structural checks at full size: degrees, row order by (degree, id), symmetry on sampled edges
    rowptr, colidx, deg = g.csr()
    checks = {"degrees_match_edge_list": bool(torch.equal(deg.long(), deg_expected)),
              "rowptr_matches_degrees": bool(torch.equal(rowptr[1:] - rowptr[:-1], deg.long()))}
    gen = torch.Generator().manual_seed(S + 104)
    live = torch.nonzero(deg > 0).flatten().cpu()
    rows = live[torch.randint(live.numel(), (512,), generator=gen)]
    ok_sorted, ok_sym = True, True
    for s_ in rows.tolist():
        a, b = int(rowptr[s_]), int(rowptr[s_ + 1])
        nb = colidx[a:b].long()
        key = deg[nb].long() * n + nb
        ok_sorted &= bool((key[1:] > key[:-1]).all()) and not bool((nb == s_).any())
        t = int(nb[torch.randint(nb.numel(), (1,), generator=gen)].item())
        ta, tb = int(rowptr[t]), int(rowptr[t + 1])
        ok_sym &= bool((colidx[ta:tb] == s_).any())
    checks["sampled_rows_sorted_no_loops"] = ok_sorted
    checks["sampled_edges_symmetric"] = ok_sym
    del rowptr, colidx, deg, deg_expected
    torch.cuda.empty_cache()
    srcs = live[torch.randint(live.numel(), (Q * (args.warmup + args.steps),), generator=gen)].to(torch.int32)
    d_srcs = srcs.cuda()
    off = torch.arange(Q + 1, dtype=torch.int64, device="cuda")
    out = torch.empty((Q, n), dtype=torch.float32, device="cuda")
    w_ppr = 1.0 - 0.8 ** 31
    w_hk = float(sum(math.exp(-5.0 + i * math.log(5.0) - math.lgamma(i + 1.0)) for i in range(31)))
    flags = agp.INPUT_ON_DEVICE | agp.OUTPUT_ON_DEVICE
    # wave width by timing on the first 32 PPR queries (or as given)
    qs = min(Q, 32)
    if args.lanes > 0:
        g.set_wave_lanes(args.lanes)
        g.set_group_width(args.width)
        lanes, width, tuned_ms = args.lanes, args.width, None
    else:
        lanes, width, tuned_ms = agp.autotune(g, [agp.ppr(0.2, 30, 1e-8, seed=S + q) for q in range(qs)],
                                              off[:qs + 1], d_srcs[:qs], None, out, n, candidates=[1, 2, 4, 8, 16])
        log(f"[large] autotuned wave width {lanes} lanes, group width {width}")
    res = {}
    for name, mk, mass in (("ppr", lambda sd: agp.ppr(0.2, 30, 1e-8, seed=sd), w_ppr),
                           ("hkpr", lambda sd: agp.hkpr(5.0, 30, 1e-8, seed=sd), w_hk)):
        times, masses = [], []
        agp.profile_read(g, reset=True)
        for k in range(args.warmup + args.steps):
            params = [mk(S + 10000 * k + q) for q in range(Q)]
            if k == args.warmup:
                agp.profile_read(g, reset=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            agp.query_batch(g, params, off, d_srcs[k * Q:(k + 1) * Q], None, out, n,
                            flags | (agp.PROFILE if k >= args.warmup else 0))
            e1.record()
            e1.synchronize()
            if k >= args.warmup:
                times.append(e0.elapsed_time(e1))
                masses.append(np.array([float(out[q].sum(dtype=torch.float64)) for q in range(Q)]))
        kern_ms, kern_launches, _ = agp.profile_read(g, reset=True)
        # work of one launch (same sources and seeds, counted in a separate pass)
        k = args.warmup
        st = agp.query_batch(g, [mk(S + 10000 * k + q) for q in range(Q)], off, d_srcs[k * Q:(k + 1) * Q], None,
                             out, n, flags | agp.COLLECT_STATS)
        work = np.zeros((3, 4))
        items = 0
        for s_ in st:
            work += np.array([list(r) for r in s_.by_kernel], dtype=np.float64)
            items += sum(s_.frontier[: s_.levels])
        ms = float(np.mean(times))
        mm = np.concatenate(masses)
        log(f"[large] {name}: {ms:.1f} ms per launch of {Q} queries; kernel ms {kern_ms}")
        res[name] = {"ms_per_launch": ms, "queries_per_s": Q / (ms / 1e3),
                     "mass_expected": mass, "mass_mean": float(mm.mean()), "mass_std": float(mm.std()),
                     "kernel_ms_per_launch": {k_: v_ / args.steps for k_, v_ in kern_ms.items()},
                     "work_per_launch": {"frontier_items": float(items),
                                         "deterministic_pushes": float(work[:, 0].sum()),
                                         "sampler_trials": float(work[:, 1].sum()),
                                         "samples_accepted": float(work[:, 2].sum())}}
    oracle_check = None if args.no_accuracy else large_oracle_check(agp, g, n, u_h, v_h, srcs[:4].numpy())
    del u_h, v_h
    line = {"metric": "queries/s", "value": 2 * Q / ((res["ppr"]["ms_per_launch"] + res["hkpr"]["ms_per_launch"]) / 1e3),
            "unit": "queries/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"chung-lu-2.0 n={n} m={m} ppr(0.2)+hkpr(5), L=30, eps=1e-8, {Q} uniform sources per launch",
                       "generate_s": t_gen, "build_s": t_build, "wave_lanes": lanes, "group_width": width,
                       "autotune_ms": tuned_ms},
            "checks": checks, "models": res, "oracle_check": oracle_check,
            "note": "a = 0, b = 1 keeps mass: E[sum pi] = sum_{i<=L} w_i for every source with degree >= 1"}
    print(json.dumps(line), flush=True)
    g.destroy()


def large_oracle_check(agp, g, n, u_h, v_h, srcs):
    """Exact PPR (alpha = 0.2, L = 2, eps = 0) of a few sources on the full graph against the FP64
    oracle, entry by entry. With L = 2, a = 0 and b = 1, pi depends only on x, the degrees of the
    source and of its neighbours, and the rows of those nodes: the oracle runs on the subgraph of
    every edge incident to a source or a neighbour of one (the generator's edges are distinct and
    loop-free, so each such node keeps its full degree there), built by the oracle's own CSR builder
    from the host edge list. Every entry outside that subgraph must be exactly zero."""
    import torch
    import oracle
    L, alpha = 2, 0.2
    t0 = time.perf_counter()
    pi_gpu, _ = agp.query_sources(g, [agp.ppr(alpha, L, 0.0) for _ in srcs], srcs)
    pi_gpu = pi_gpu.cpu().numpy()
    # the nodes whose rows matter: the sources and their neighbours
    mark = np.zeros(n, bool)
    mark[srcs] = True
    hit = mark[u_h] | mark[v_h]
    mark[u_h[hit]] = True
    mark[v_h[hit]] = True
    sel = mark[u_h] | mark[v_h]
    su, sv = u_h[sel], v_h[sel]
    nodes = np.unique(np.concatenate([su, sv]))
    local = np.full(n, -1, np.int64)
    local[nodes] = np.arange(nodes.size)
    og = oracle.build_csr(int(nodes.size), local[su].astype(np.int32), local[sv].astype(np.int32))
    w, Y = oracle.tail_sums(oracle.PPR, L, alpha)
    t_sub = time.perf_counter() - t0
    per = []
    for q, s_ in enumerate(srcs):
        x = np.zeros(og.n)
        x[local[s_]] = 1.0
        want_local = oracle.basic(og, 0.0, 1.0, L, w, Y, x)
        want = np.zeros(n)
        want[nodes] = want_local
        got = pi_gpu[q].astype(np.float64)
        nz = want != 0
        rel = np.abs(got[nz] - want[nz]) / np.abs(want[nz])
        per.append({"source": int(s_), "degree": int(og.deg[local[s_]]), "support": int(nz.sum()),
                    "max_rel_err": float(rel.max()) if rel.size else 0.0,
                    "entries_beyond_1e-5": int((rel > 1e-5).sum()),
                    "nonzero_outside_support": int((got[~nz] != 0).sum())})
    return {"what": f"exact PPR alpha={alpha} L={L} (eps = 0) vs the FP64 oracle, every entry",
            "subgraph_edges": int(su.size), "subgraph_nodes": int(nodes.size),
            "seconds": time.perf_counter() - t0, "subgraph_s": t_sub, "per_source": per}


# ------------------------------------------------------------------------------- serving
def serve_trace(n, u, v, rate, duration, seed, beta):
    """Seeded Poisson trace of the serving mix: PPR / Katz / HKPR / transition (22.5% each) and
    BF16 feature blocks of 1-64 columns (10%, log-uniform); eps in {1e-6, 1e-7, 1e-8, 1e-9};
    L uniform in 5..40; sources uniform over nodes with edges (50%) or degree-weighted (50%)."""
    rng = np.random.default_rng(seed)
    deg = np.bincount(u, minlength=n) + np.bincount(v, minlength=n)
    live = np.flatnonzero(deg > 0)
    cdf = np.cumsum(deg, dtype=np.float64)
    cdf /= cdf[-1]
    gaps = rng.exponential(1.0 / rate, size=int(rate * duration * 1.2) + 64)
    t = np.cumsum(gaps)
    while t[-1] < duration:  # extend in the rare case the draw fell short
        t = np.concatenate([t, t[-1] + np.cumsum(rng.exponential(1.0 / rate, size=1024))])
    t = t[t < duration]
    k = len(t)
    r = rng.random(k)
    kinds = np.where(r < 0.10, 4, np.minimum(3, ((r - 0.10) / 0.225).astype(np.int64)))
    names = ("ppr", "katz", "hkpr", "transition", "features")
    eps = rng.choice([1e-6, 1e-7, 1e-8, 1e-9], size=k)
    L = rng.integers(5, 41, size=k)
    uniform_src = live[rng.integers(0, len(live), size=k)]
    weighted_src = np.minimum(np.searchsorted(cdf, rng.random(k), side="right"), n - 1)
    src = np.where(rng.random(k) < 0.5, uniform_src, weighted_src)
    cols = np.clip(np.round(np.exp(rng.uniform(0, np.log(64), size=k))), 1, 64).astype(np.int64)
    seeds = rng.integers(0, 2**62, size=k)
    return [(float(t[i]), names[kinds[i]], float(eps[i]), int(L[i]), int(src[i]), int(cols[i]), int(seeds[i]))
            for i in range(k)]


def run_serve(args, wl):
    import torch
    import paper_2106_03058_gb300 as agp
    u, v = make_edges(wl)
    n = wl["n"]
    g = agp.build_graph(n, u, v)
    beta, lam = agp.katz_beta(g, 0.85, iters=1000, tol=1e-12)
    # the trace spans the warm-up and the measured window; only requests arriving in the window count
    trace = serve_trace(n, u, v, args.rate, args.serve_warmup + args.duration, S + 500, beta)
    X = torch.randn(n, 64, generator=torch.Generator().manual_seed(S + 200)).to(torch.bfloat16).cuda()

    def params_of(kind, eps, L, seed):
        if kind == "ppr":
            return agp.ppr(0.2, L, eps, seed=seed)
        if kind == "katz":
            return agp.katz(beta, L, eps, seed=seed)
        if kind == "hkpr":
            return agp.hkpr(5.0, L, eps, seed=seed)
        if kind == "transition":
            return agp.transition(L, eps, seed=seed)
        return agp._params(0.5, 0.5, L, agp.W_PPR, 0.1, eps=eps, seed=seed)

    def replay(mode, admission=agp.ADMIT_COST, check=False):
        """Submit the trace in real time while a consumer thread takes results in completion order
        (agp_serve_next) and releases each at once, as a serving client does."""
        import threading
        srv = agp.Server(g, mode=mode, max_lanes=args.lanes if args.lanes > 0 else 0, admission=admission)
        arrival = {}
        lock = threading.Lock()
        stop = threading.Event()
        finished = []  # (arrival s, latency s, status)
        kept = []      # (trace index, result row) of a few single-source results, for the oracle check

        def consume():
            while True:
                r = srv.next(timeout_us=20_000)
                if r is None:
                    if stop.is_set():
                        return
                    continue
                tk, res = r
                while True:  # the submitting thread records the arrival right after submit returns
                    with lock:
                        ta = arrival.get(tk)
                    if ta is not None:
                        break
                    time.sleep(1e-4)
                ta, i_tr = ta
                finished.append((ta, res.latency_us / 1e6, res.status))
                tr = trace[i_tr]
                if (check and res.status == 0 and len(kept) < 8 and tr[1] != "features" and tr[3] <= 12
                        and ta >= args.serve_warmup):
                    kept.append((i_tr, srv.result_array(res).cpu().numpy().copy()))
                srv.release(tk)

        th = threading.Thread(target=consume, daemon=True)
        th.start()
        tickets = []
        log(f"[serve] mode {mode}: replaying {len(trace)} requests over {args.serve_warmup + args.duration}s")
        t0 = time.perf_counter()
        for i_tr, (ta, kind, eps, L, src, cols, seed) in enumerate(trace):
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            p = params_of(kind, eps, L, seed)
            tk = srv.submit(p, X=X[:, :cols]) if kind == "features" else srv.submit(p, source=src)
            with lock:
                arrival[tk] = (ta, i_tr)
            tickets.append(tk)
        submitted_by = time.perf_counter() - t0
        # the window closes at warm-up + duration + drain; a request counts when it completes inside
        # the measured window (after the warm-up), whenever it arrived: under overload the oldest
        # waiting requests are the ones that finish
        end_s = args.serve_warmup + args.duration + args.drain
        time.sleep(max(0.0, t0 + end_s - time.perf_counter()))
        stop.set()
        th.join()
        lat, done, done_arrived = [], 0, 0
        for ta, latency, status in finished:
            t_end = ta + latency
            if status == 0 and args.serve_warmup <= t_end <= end_s:
                done += 1
                done_arrived += ta >= args.serve_warmup
                lat.append(latency * 1e3)
        elapsed = end_s - args.serve_warmup
        st = srv.stats()
        log(f"[serve] mode {mode}: {done} done in {elapsed:.1f}s, stats {st}; stopping the server")
        for tk in tickets:  # requests still queued are dropped, the running ones end their sweep
            try:
                srv.cancel(tk)
            except Exception:
                pass
        srv.destroy()
        log(f"[serve] mode {mode}: stopped after {time.perf_counter() - t0:.1f}s")
        lat = np.array(lat) if lat else np.array([np.nan])
        offered = sum(1 for tr in trace if tr[0] >= args.serve_warmup)
        out = {"offered": offered, "completed": done, "completed_arrived_in_window": done_arrived,
               "queries_per_s": done / elapsed,
               "p50_ms": float(np.nanpercentile(lat, 50)), "p99_ms": float(np.nanpercentile(lat, 99)),
               "elapsed_s": elapsed, "submit_s": submitted_by, "sweeps": st["sweeps"]}
        if check:
            out["accuracy"] = serve_accuracy(kept)
        return out

    og_cache = []

    def serve_accuracy(kept):
        """Served single-source results (L <= 12, arrived in the window) against the exact FP64
        propagation: the same measures as the batched step's accuracy."""
        import oracle
        from concurrent.futures import ThreadPoolExecutor
        if not kept:
            return None
        if not og_cache:
            og_cache.append(oracle.build_csr(n, u, v))
        og = og_cache[0]
        weights = {"ppr": (oracle.PPR, 0.2), "katz": (oracle.KATZ, beta), "hkpr": (oracle.HKPR, 5.0),
                   "transition": (oracle.TRANSITION, 0.0)}

        def one(item):
            i_tr, row = item
            _, kind, eps, L, src, _, _ = trace[i_tr]
            wk, prm = weights[kind]
            w, Y = oracle.tail_sums(wk, L, prm)
            return row_accuracy(og, kind, 0.0, 1.0 if kind != "katz" else 0.0, L, w, Y, eps, src, row)

        t0_ = time.perf_counter()
        with ThreadPoolExecutor(max_workers=max(1, min(host_cores(), len(kept)))) as ex:
            per = list(ex.map(one, kept))
        summ = {}
        for name in ("paper", "chebyshev"):
            vals = [r[f"frac_ok_{name}"] for r in per if r[f"frac_ok_{name}"] is not None]
            summ[f"frac_ok_at_delta_{name}"] = {"min": float(min(vals)) if vals else None,
                                               "mean": float(np.mean(vals)) if vals else None, "queries": len(vals)}
        summ["rel_l1_max"] = float(max(r["rel_l1"] for r in per))
        summ["max_error_max"] = float(max(r["max_error"] for r in per))
        summ["precision_at_50_min"] = float(min(r["precision_at_50"] for r in per))
        d99 = [r["delta_99"] for r in per if r["delta_99"] is not None]
        summ["delta_99"] = {"max": float(max(d99)) if d99 else None, "median": float(np.median(d99)) if d99 else None}
        summ["queries_checked"] = len(per)
        summ["oracle_s"] = time.perf_counter() - t0_
        summ["per_query"] = per
        return summ

    batched = replay(agp.SERVE_BATCHED, check=not args.no_accuracy)
    batched_fifo = replay(agp.SERVE_BATCHED, agp.ADMIT_FIFO)
    fifo = replay(agp.SERVE_FIFO_PLAIN) if not args.no_fifo else None
    line = {"metric": "served queries/s (continuous batching)", "value": batched["queries_per_s"], "unit": "queries/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["name"] + " | serving trace", "rate": args.rate, "duration_s": args.duration,
                       "warmup_s": args.serve_warmup, "drain_s": args.drain, "lambda_1": lam},
            "batched": batched, "batched_fifo_admission": batched_fifo, "fifo_plain": fifo,
            "note": "completed = requests finishing inside the measured window (after the warm-up); latency "
                    "percentiles over those; offered = arrivals inside the window; a consumer thread takes "
                    "results in completion order (agp_serve_next) and releases each at once"}
    print(json.dumps(line), flush=True)
    g.destroy()


# ------------------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="agp", choices=["agp", "reference"])
    ap.add_argument("--small", action="store_true", help="small R-MAT workload (quick check)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the oracle check of timed queries")
    ap.add_argument("--plain-queries", type=int, default=64)
    ap.add_argument("--queries", type=int, default=0, help="sources per launch (default: the workload's 256)")
    ap.add_argument("--lanes", type=int, default=0, help="wave width; 0 = autotune (with the group width)")
    ap.add_argument("--width", type=int, default=0, help="group width with --lanes (1, 2, 4; 0 = automatic)")
    ap.add_argument("--pull", type=int, default=None,
                    help="pull a level when the lane's frontier volume is >= nnz >> PULL (-1 = never; default: the "
                         "library's)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serve", action="store_true", help="serving trace instead of the batched step")
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--duration", type=float, default=10.0)
    ap.add_argument("--drain", type=float, default=20.0)
    ap.add_argument("--no-fifo", action="store_true")
    ap.add_argument("--serve-warmup", type=float, default=0.0,
                    help="seconds of trace before the measured window (its requests are served, not counted)")
    ap.add_argument("--features", action="store_true", help="GNN feature propagation workload")
    ap.add_argument("--large", action="store_true", help="65M-node, 1.8B-edge PPR / HKPR workload")
    ap.add_argument("--eps", type=float, default=0.0)
    args = ap.parse_args()
    wl = workload(args.small)
    if args.queries:
        wl["Q"] = args.queries
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # N GPUs asked for outside torchrun: launch the N ranks here (one process per GPU)
        import socket
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
               "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__)] + sys.argv[1:]
        sys.exit(subprocess.call(cmd))
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world != args.gpus and rank == 0:
        log(f"[bench] --gpus {args.gpus} but WORLD_SIZE {world}: running {world} rank(s)")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, wl, rank)
    if args.serve:
        return run_serve(args, wl)
    if args.features:
        return run_features(args)
    if args.large:
        return run_large(args)

    import torch
    import torch.distributed as dist
    import paper_2106_03058_gb300 as agp

    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    if world > 1:
        dist.init_process_group("nccl")

    def barrier_sync():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    t0 = time.perf_counter()
    u, v = make_edges(wl)
    n, Q = wl["n"], wl["Q"]
    log(f"[bench] edges ready in {time.perf_counter() - t0:.1f}s")
    agp.lib()
    t0 = time.perf_counter()
    g = agp.build_graph(n, u, v, device=local)
    log(f"[bench] graph built on GPU in {time.perf_counter() - t0:.2f}s (nnz={g.nnz})")
    beta, lam = agp.katz_beta(g, 0.85, iters=1000, tol=1e-12)
    log(f"[bench] lambda_1={lam:.6f} beta={beta:.6e}")
    if args.pull is not None:
        g.set_pull_threshold(args.pull)

    steps_total = args.warmup + args.steps
    srcs = degree_weighted_sources(n, u, v, Q * 2 * steps_total, wl["seed_src"])
    d_srcs = torch.as_tensor(srcs, device=dev)
    off = torch.arange(Q + 1, dtype=torch.int64, device=dev)
    out_k = torch.empty((Q, n), dtype=torch.float32, device=dev)
    out_t = torch.empty((Q, n), dtype=torch.float32, device=dev)
    eps = wl["eps"]

    def params_for(step):
        pk = [agp.katz(beta, wl["L_katz"], eps, seed=S + step * 4096 + q) for q in range(Q)]
        pt = [agp.transition(4, eps, seed=S + step * 4096 + 2048 + q) for q in range(Q)]
        return pk, pt

    all_params = [params_for(k) for k in range(steps_total)]
    flags = agp.INPUT_ON_DEVICE | agp.OUTPUT_ON_DEVICE

    def run_step(k, extra=0, stats=False):
        pk, pt = all_params[k]
        base = k * 2 * Q
        f = flags | extra | (agp.COLLECT_STATS if stats else 0)
        sk = agp.query_batch(g, pk, off, d_srcs[base:base + Q], None, out_k, n, f)
        st = agp.query_batch(g, pt, off, d_srcs[base + Q:base + 2 * Q], None, out_t, n, f)
        return sk, st

    # accuracy sample: 4 Katz and 4 transition queries of each of the first two timed steps, their
    # rows copied to the host after the step (outside the timed region), checked against the oracle
    acc_steps = min(2, args.steps) if not args.no_accuracy else 0
    acc_rows = []

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2

    # wave width: given, or tuned on a sample of the first step's Katz launch (cached)
    tuned_ms = None
    width = args.width
    if args.lanes > 0:
        g.set_wave_lanes(args.lanes)
        g.set_group_width(args.width)
        lanes = args.lanes
    else:
        # the sample has the step's mix: half Katz, half transition queries of the first step
        h = min(Q, 16)
        qs = 2 * h
        pk, pt = all_params[0]
        t0 = time.perf_counter()
        sample_src = torch.cat([d_srcs[:h], d_srcs[Q:Q + h]])
        lanes, width, tuned_ms = agp.autotune(g, list(pk[:h]) + list(pt[:h]), off[:qs + 1], sample_src, None, out_k,
                                              n, candidates=[c for c in (1, 2, 4, 8, 16, 32) if c <= 2 * qs])
        log(f"[bench] autotuned wave width {lanes} lanes, group width {width} ({tuned_ms:.1f} ms for {h} Katz + "
            f"{h} transition queries, {time.perf_counter() - t0:.1f}s)")

    for k in range(args.warmup):
        run_step(k)
    barrier_sync()
    agp.profile_read(g, reset=True)
    stream = torch.cuda.current_stream()
    step_ms = []
    lat_k, lat_t = [], []
    with ClockSampler(local) as clocks:
        barrier_sync()
        for k in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sk, st = run_step(args.warmup + k, agp.PROFILE | agp.QUERY_TIMES)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            lat_k += [x.done_ms for x in sk]
            lat_t += [x.done_ms for x in st]
            if k < acc_steps:
                base = (args.warmup + k) * 2 * Q
                for j in range(4):
                    q = j * (Q // 4)
                    acc_rows.append(("katz", int(srcs[base + q]), out_k[q].cpu().numpy()))
                    acc_rows.append(("transition", int(srcs[base + Q + q]), out_t[q].cpu().numpy()))
        barrier_sync()
    clk = clocks.summary()
    kern_ms, kern_launches, total_launches = agp.profile_read(g, reset=True)
    total_ms, queries, value = job_throughput(sum(step_ms), 2 * Q * args.steps, world, dev)

    # per-kernel work of the timed steps (same sources and seeds, counted in a separate pass)
    work = np.zeros((3, 4))
    items = 0
    for k in range(args.steps):
        sk, st = run_step(args.warmup + k, 0, stats=True)
        for s_ in list(sk) + list(st):
            work += np.array([list(r) for r in s_.by_kernel], dtype=np.float64)
            items += sum(s_.frontier[: s_.levels])
    # a = 0 for both query types: no neighbour-degree gathers
    scanned = args.steps * Q * n * ((wl["L_katz"] + 1) + (4 + 1))  # lane-levels x nodes
    bytes_k = {
        "compact": items * B_COMPACT_ITEM + scanned * B_SCAN,
        "expand": items * B_ITEM + work[0, 0] * B_DET + work[0, 1] * B_TRIAL + work[0, 2] * B_ACC,
        "push": work[1, 0] * B_DET + work[1, 1] * B_TRIAL + work[1, 2] * B_ACC,
        "sample": work[2, 1] * B_TRIAL + work[2, 2] * B_ACC,
    }
    # The dominant kernel is the push: the largest share of the step in the serialised launch list
    # (profiles/launch_list_katz_transition_4M.md: push 37%, expansion 34%, sampler 16%). The live
    # event times below overlap with the other wave's kernels, which inflates the latency-bound
    # expansion most, so they do not rank the kernels. Every kernel's figure is reported as well.
    dom = "push"

    def kernel_roofline(k_):
        n_l = max(kern_launches[k_], 1)
        ms = kern_ms[k_] / n_l
        return (bytes_k[k_] / n_l) / (ms / 1e3) / 1e9 if ms > 0 else 0.0, n_l, ms

    achieved, launches, avg_ms = kernel_roofline(dom)
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        peak = float(json.load(open(peaks_path))["hbm_gbs"])
        peak_src = "measured"
    else:
        peak, peak_src = HBM_FALLBACK_GBS, "fallback"
    edge_ops = work[:, 0].sum() + work[:, 2].sum()
    traffic = None
    if dom == "push" and lanes == PUSH_TRAFFIC_LANES and PUSH_DRAM_BYTES_PER_RED is not None:
        traffic = PUSH_DRAM_BYTES_PER_RED * (work[1, 0] + work[1, 2]) / launches
    # k_push is bound by random FP32 atomic adds into residue vectors that stay in L2, not by HBM:
    # its adds per second against a library scatter-add of the same shape on this GPU
    atomics = None
    if rank == 0 and kern_ms["push"] > 0:
        ceil = atomic_ceiling(g, lanes, n)
        push_adds = (work[1, 0] + work[1, 2]) / args.steps
        rate = push_adds / (kern_ms["push"] / args.steps / 1e3)
        # the same rate for one wave alone (the step's first `lanes` Katz queries as a call of their
        # own: one wave, so no second wave shares the GPU with its pushes)
        pk0, _ = all_params[args.warmup]
        one_off = off[:lanes + 1]
        agp.profile_read(g, reset=True)
        agp.query_batch(g, pk0[:lanes], one_off, d_srcs[args.warmup * 2 * Q:args.warmup * 2 * Q + lanes], None,
                        out_k, n, flags | agp.PROFILE)
        one_ms, _, _ = agp.profile_read(g, reset=True)
        st1 = agp.query_batch(g, pk0[:lanes], one_off, d_srcs[args.warmup * 2 * Q:args.warmup * 2 * Q + lanes],
                              None, out_k, n, flags | agp.COLLECT_STATS)
        w1 = sum(np.array([list(r) for r in s_.by_kernel], dtype=np.float64) for s_ in st1)
        one_rate = (w1[1, 0] + w1[1, 2]) / (one_ms["push"] / 1e3) if one_ms["push"] > 0 else None
        atomics = {"push_adds_per_step": push_adds, "push_adds_per_s": rate,
                   "ceiling_adds_per_s": ceil, "frac_of_degree_weighted": rate / ceil["degree_weighted"],
                   "one_wave_alone": {"push_adds_per_s": one_rate,
                                      "frac_of_degree_weighted": (one_rate / ceil["degree_weighted"]
                                                                  if one_rate else None),
                                      "queries": int(lanes), "kind": "katz"},
                   "note": "push time from CUDA events around every k_push of the timed steps, which "
                           "include the other wave's kernels sharing the GPU (an upper bound on its time); "
                           "one_wave_alone times the pushes of one Katz wave run by itself"}

    # ---- plain path: one query per launch sequence, host-synchronised frontier sizes. The same
    # queries run on both paths after a warm-up of each; a query's latency is its completion time
    # from the start of its launch (one CUDA event per wave), and throughput is queries over the
    # host wall time of both launches.
    plain_qps = None
    if args.plain_queries > 0 and rank == 0:
        k = args.warmup
        pk, pt = all_params[k]
        base = k * 2 * Q
        half = min(args.plain_queries // 2, Q)

        def both(fl):
            a_ = agp.query_batch(g, pk[:half], off[:half + 1], d_srcs[base:base + half], None, out_k, n,
                                 fl | agp.QUERY_TIMES)
            b_ = agp.query_batch(g, pt[:half], off[:half + 1], d_srcs[base + Q:base + Q + half], None, out_t, n,
                                 fl | agp.QUERY_TIMES)
            return [x.done_ms for x in a_] + [x.done_ms for x in b_]

        res = {}
        for name, fl in (("plain", flags | agp.PLAIN), ("batched", flags)):
            both(fl)  # warm-up (captured graphs, workspaces)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lat = both(fl)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            res[name] = {"queries_per_s": 2 * half / dt, **latency_summary(lat)}
        plain_qps = {"queries": 2 * half, "plain": res["plain"], "batched": res["batched"],
                     "speedup_queries_per_s": res["batched"]["queries_per_s"] / res["plain"]["queries_per_s"],
                     "note": "same Katz + transition queries on both paths, each after one untimed run"}

    # ---- end to end through host buffers (pinned), copies inside the timed region
    e2e_value, h2d, d2h = None, 0, 0
    if not args.no_e2e:
        e2e_value, h2d, d2h = end_to_end(agp, g, args, all_params, srcs, Q, n, world, dev)

    # ---- the oracle's CSR (host), for the accuracy check and the CPU baseline
    og, t_csr = None, 0.0
    need_oracle = rank == 0 and (acc_rows or (not args.no_cpu_baseline and world == 1))
    if need_oracle:
        import oracle
        t0 = time.perf_counter()
        og = oracle.build_csr(n, u, v)
        t_csr = time.perf_counter() - t0

    # ---- accuracy of the timed queries against the exact FP64 propagation
    accuracy = None
    if acc_rows and rank == 0:
        accuracy = accuracy_vs_oracle(og, acc_rows, eps, beta, wl["L_katz"], host_cores())
        log(f"[bench] accuracy vs oracle: {json.dumps({k_: v_ for k_, v_ in accuracy.items() if k_ != 'per_query'})}")

    # ---- CPU baseline: the oracle on the host cores, bounded sample (rank 0, N = 1 only)
    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        base = args.warmup * 2 * Q + Q
        threads = host_cores()
        used, dt = oracle_sample(og, n, srcs[base:base + threads], eps, 4, threads)
        cpu = {"value": used / dt, "unit": "queries/s", "cores": used, "nproc": host_cores(), "cpu_model": cpu_model(),
               "kind": "oracle",
               "sample": f"{used} of the {Q} L=4 transition queries of one step, one per host thread on all "
                         f"{used} cores, FP64 Algorithm 2 with per-neighbour Bernoulli trials ({dt:.1f}s; CSR build "
                         f"{t_csr:.1f}s excluded; Katz queries at eps=1e-8 take minutes each in the oracle and are "
                         f"left out)"}

    if rank == 0:
        line = {
            "metric": "queries/s", "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["name"], "parallelism": f"replicas{world}", "queries_per_step": 2 * Q,
                       "wave_lanes": lanes, "group_width": width, "autotune_ms": tuned_ms,
                       "pull_threshold_shift": args.pull if args.pull is not None else "default (-1: pull levels off)",
                       "lambda_1": lam, "beta": beta,
                       "l2": "flushed before every timed step (256 MB write); CSR 0.96 GB and 8 GB of residues exceed L2"},
            "latency_ms": {"per_query": latency_summary(lat_k + lat_t), "katz": latency_summary(lat_k),
                           "transition": latency_summary(lat_t),
                           "p50_step": float(np.percentile(step_ms, 50)), "p99_step": float(np.percentile(step_ms, 99)),
                           "note": "a query's latency is the end of the wave that finished it, from the start of its "
                                   "launch (CUDA events, timed steps)"},
            "accuracy": accuracy,
            "edges_pushed_per_s": rank_reduce(edge_ops, "sum", world, dev) / (total_ms / 1e3),
            "work_per_step": {"frontier_items": items / args.steps,
                              "deterministic_pushes": float(work[:, 0].sum()) / args.steps,
                              "sampler_trials": float(work[:, 1].sum()) / args.steps,
                              "samples_accepted": float(work[:, 2].sum()) / args.steps,
                              "by_kernel_det_trials_accepted": {k_: [float(x) / args.steps for x in work[i_, :3]]
                                                                for i_, k_ in enumerate(("expand", "push", "sample"))}},
            "plain_path": plain_qps,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                         "algorithmic_bytes_per_launch": bytes_k[dom] / launches, "avg_launch_ms": avg_ms,
                         "by_kernel": {k_: {"achieved": kernel_roofline(k_)[0], "frac": kernel_roofline(k_)[0] / peak,
                                            "avg_launch_ms": kernel_roofline(k_)[2]}
                                       for k_ in ("compact", "expand", "push", "sample")}},
            "l2_atomics": atomics,
            "kernel_ms": kern_ms, "kernel_launches_profiled": kern_launches,
            "gpu_launches": int(total_launches),
            "clocks": clk,
            "cpu_baseline": cpu,
            "e2e": None if e2e_value is None else {"value": e2e_value, "unit": "queries/s", "h2d_bytes_per_step": h2d,
                                                   "d2h_bytes_per_step": d2h},
        }
        print(json.dumps(line), flush=True)
    g.destroy()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
