#!/usr/bin/env python3
"""Exact betweenness-centrality throughput on one GB300 (GTEPS = sources * m / s).

Workload (default): batched multi-source BC on an undirected R-MAT graph, scale 20
(1,048,576 vertices), edge factor 16, a/b/c/d = 0.57/0.19/0.19/0.05, seed 3; 4096 sources
drawn uniformly from the largest component (seed 4); tiles of 32..256 sources per
launch, tile width chosen by the autotuner.  One step = one bc_sources call over the
4096 sources (forward sigma counting + backward dependency sweep + BC accumulation).

Also reported beside the headline: the same step end to end through the C ABI with host
buffers (e2e), the tile kernel's roofline, the per-source path on the same graph and GPU (a
sample of its sources), each tile width, the all-sources runs of the R-MAT scale-12
graph, the leaf-rich graph pruned vs unpruned, the 1024 x 1024 grid's level-loop modes,
the serving sweep (p50/p99 latency per arrival rate), and the oracle on the host cores
(cpu_baseline).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       python bench.py --study deg1|deg2|scan     (one study, one JSON line)
       python bench.py --profile-case SPEC         (one small call for a profiler)
Multi-GPU (torchrun): each rank runs the graph on its own GPU with its own 4096 seeded
sources (weak scaling) and, once per step inside the timed region, the ranks sum their BC
vectors with one NCCL all-reduce (BC is additive over sources).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402

METRIC = "BC GTEPS (sources·m/s) batched vs per-source on 1 GB300; serving p50/p99 latency"
# what the path computes in: path counts as 64-bit integers (modulo 2^64, extended range past
# it), dependency sums as float-float pairs (two f32, about 48 significant bits), the BC
# accumulation in f64
DTYPE = "u64+ff32x2+f64"
WORKLOAD = {
    "workload": "rmat-s20-ef16 batched exact BC, 4096 LCC sources",
    "graph": "R-MAT scale 20, edge factor 16, a/b/c/d .57/.19/.19/.05, seed 3",
    "sources": "4096 uniform from the largest component, seed 4",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sources", type=int, default=4096)
    ap.add_argument("--quick", action="store_true", help="skip the side measurements")
    ap.add_argument("--study", default=None, choices=["deg1", "deg2", "scan"],
                    help="deg1: the 1-degree removal study on R-MAT scale 20, EF 4 / 16 / 32; "
                         "deg2: the heuristics H0-H3 on road-like graphs; scan: the degree-prefix "
                         "reuse of the per-source path on and off (one JSON line, instead of the "
                         "benchmark)")
    ap.add_argument("--profile-case", default=None,
                    help="run one small case for a profiler and exit: 'tile:T:K' (one bc_sources "
                         "call of K sources in tiles of T) or 'plain:K' on the R-MAT scale-20 graph")
    return ap.parse_args()


def profile_case(spec: str):
    """One bc_sources call, for ncu captures of a single kernel: on the R-MAT scale-20 graph
    ('tile:T:K', 'plain:K') or on the 1024 x 1024 deleted-edge grid ('grid:T:K'; its
    sigma needs the extended range, so the tile runs twice when it starts in 64-bit mode),
    or the per-source path on R-MAT scale 12 with its first K non-isolated sources
    ('small:K', one source per CTA), or one source per CTA on the grid ('gridcta:K')."""
    import paper_1602_00963_gb300 as bc
    parts = spec.split(":")
    if parts[0] == "grid":
        g = gg.cached("grid", gg.grid2d, 1024, 1024, 5, 0.1)
        src = gg.sample_sources(g, 1024, seed=6)
    elif parts[0] == "small":
        g = gg.rmat(12, 16, 1)
        src = np.flatnonzero(g.degrees() > 0).astype(np.int32)
    elif parts[0] == "gridcta":
        g = gg.cached("grid", gg.grid2d, 1024, 1024, 5, 0.1)
        src = gg.sample_sources(g, 1024, seed=6)
    else:
        g, src = load_workload(4096, 0)
    # gridcta: a 2.5 GB budget keeps the per-CTA workspace (and what a profiler saves
    # between its passes) small; the kernel then runs fewer CTAs
    ctx = bc.bc_ctx_create(0, (5 << 29) if parts[0] == "gridcta" else 0)
    h = bc.bc_graph_create(ctx, g.n, g.row_ptr, g.col_idx, g.nnz, 0)
    if parts[0] in ("tile", "grid"):
        T, k = int(parts[1]), int(parts[2])
        flags = bc.BC_PATH_TILED | bc.BC_TILE(T)
    else:
        k = int(parts[1])
        flags = bc.BC_PATH_PLAIN | (bc.BC_PLAIN_CTA if parts[0] == "gridcta" else 0)
    if parts[0] in ("small", "gridcta"):
        bc.bc_sources(h, g.n, src[:k], flags)  # warm-up: workspace and shared-memory setup
    _, st = bc.bc_sources(h, g.n, src[:k], flags)
    print(json.dumps({"profile_case": spec, "seconds": st["seconds"], "gteps": st["gteps"],
                      "kernel_launches": st["kernel_launches"],
                      "reached_vertices": st["reached_vertices"], "reached_arcs": st["reached_arcs"]}))
    bc.bc_destroy(h)
    bc.bc_destroy(ctx)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_sources(g, nsrc: int, rank: int):
    """Rank r's sources: nsrc uniform from the largest component, seed 4 + 1000 r (rank 0
    draws the workload's own list; other ranks draw their own, so per-rank work is fixed)."""
    return gg.sample_sources(g, nsrc, seed=4 + 1000 * rank)


def load_workload(nsrc: int, rank: int):
    g = gg.cached("rmat", gg.rmat, 20, 16, 3)
    return g, rank_sources(g, nsrc, rank)


def reduce_bc(bc_vec, dist):
    """Sources are split over the ranks and BC is additive over sources (Alg. 1 sums each
    source's dependencies), so the job's BC is the sum of the ranks' vectors: one sum
    all-reduce of the FP64 BC vector per step (the paper's coarse-grained mode with every
    rank on its own source shard, Sec. 3.3).  No-op on one rank."""
    if dist is not None:
        dist.all_reduce(bc_vec)
    return bc_vec


def max_over_ranks(x: float, dist, device="cpu") -> float:
    """The largest of the ranks' values of x (a time): the job ends with its slowest rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks sampler
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) > 8 for i in range(4)
                          if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------------ roofline model
def algorithmic_bytes(stats: dict, tile_width: int) -> float:
    """Compulsory bytes of one call, per source from its reached vertices n_r and arcs a_r:
    per-source path 8 a_r + 84 n_r; a tile of width T (CSR shared by the tile)
    (8 a_r + 16 n_r) / T + 68 n_r + n_r / 4 (each datum moved once per pass, perfect reuse;
    the last term is the T-bit level masks, read and written once per vertex and level:
    2 T / 8 bytes shared by the tile's T sources)."""
    nr = stats["reached_vertices"]
    ar = stats["reached_arcs"]
    if tile_width <= 1:
        return 8.0 * ar + 84.0 * nr
    return (8.0 * ar + 16.0 * nr) / tile_width + 68.0 * nr + 0.25 * nr


def code_sha1(path: str) -> str:
    """sha1 of a C/CUDA source with its comments and blank lines removed: it changes when
    the code changes, not when a comment does."""
    import hashlib
    import re
    with open(path) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    lines = [ln.rstrip() for ln in text.splitlines()]
    return hashlib.sha1("\n".join(ln for ln in lines if ln.strip()).encode()).hexdigest()


def ncu_traffic(T: int, tiles_bytes: float):
    """DRAM bytes (read + write) per launch of the tile kernel from the committed ncu
    summary, if it was taken on the current kernel code and this tile width."""
    path = os.path.join(ROOT, "profiles", f"tile_rmat20_dram_T{T}.json")
    src = os.path.join(ROOT, "paper_1602_00963_gb300", "csrc", "bc_tile.cu")
    try:
        with open(path) as f:
            j = json.load(f)
        if j.get("kernel_code_sha1") != code_sha1(src) or int(j.get("tile_width", 0)) != T:
            return None
        return float(j["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------ CPU oracle
SOFT_FLOAT = ("the oracle keeps sigma and delta in C long double: binary128 done in software "
              "on aarch64 (Grace), 80-bit x87 on x86-64")


def cpu_baseline(g, src, budget_s: float = 15.0, single_s: float = 8.0):
    """The oracle as it stands (plain sequential Brandes built -O3, one thread per host core
    over sources), timed on a bounded sample of the workload's sources; and on one core, on
    a smaller sample (each timing a labelled sample of the same sources, as the paper's
    totals are)."""
    import oracle
    nth = os.cpu_count() or 1
    t = time.perf_counter()
    oracle.bc(g, src[:1], nthreads=1)
    one = max(time.perf_counter() - t, 1e-3)
    k = int(max(1, min(len(src), budget_s * nth / one)))
    k = max(nth, (k // nth) * nth) if k >= nth else k
    sample = src[:k]
    t = time.perf_counter()
    oracle.bc(g, sample, nthreads=min(nth, k))
    dt = time.perf_counter() - t
    k1 = int(max(1, min(len(src), single_s / one)))
    t = time.perf_counter()
    oracle.bc(g, src[:k1], nthreads=1)
    dt1 = time.perf_counter() - t
    return {"value": k * g.m / dt / 1e9, "unit": "GTEPS", "cores": min(nth, k), "kind": "oracle",
            "sample": f"{k} of the {len(src)} sources, one thread per core, {dt:.1f} s; {SOFT_FLOAT}",
            "single_core": {"value": k1 * g.m / dt1 / 1e9, "unit": "GTEPS", "cores": 1,
                            "sample": f"{k1} of the {len(src)} sources on one core, {dt1:.1f} s"}}, dt / k


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    """The oracle on the host cores as the reference arm: the same workload, metric and
    unit; each step runs a bounded sample of the workload's sources (about 4 s), after W
    warm-up steps of the same sample."""
    if rank != 0:
        return
    g, src = load_workload(args.sources, 0)
    cb, per_src = cpu_baseline(g, src, budget_s=6.0, single_s=4.0)
    import oracle
    nth = os.cpu_count() or 1
    k = max(min(nth, len(src)), int(4.0 / max(per_src, 1e-6)))
    k = min(k, len(src))
    for _ in range(args.warmup):
        oracle.bc(g, src[:k], nthreads=min(nth, k))
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.bc(g, src[:k], nthreads=min(nth, k))
        times.append(time.perf_counter() - t)
    dt = statistics.median(times)
    value = k * g.m / dt / 1e9
    line = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64+f128",
            "data": "synthetic", "impl": "reference", "config": dict(WORKLOAD),
            "cpu_baseline": {"kind": "oracle", "cores": min(nth, k), "value": value,
                             "sample": f"{k} of the {len(src)} sources per step (median of "
                                       f"{args.steps} steps); {SOFT_FLOAT}",
                             "single_core": cb["single_core"]},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ serving load
def serving_pool():
    """Resident pool: Erdos-Renyi n = 1K / 16K / 256K (average degree 8), R-MAT scale 12 /
    16 / 20 (EF 16), grids 256^2 / 1024^2 (10% of edges deleted, largest component);
    seeds 10..17 in that order."""
    return [
        ("er-1k", gg.cached("er", gg.erdos_renyi, 1 << 10, 4 << 10, 10)),
        ("er-16k", gg.cached("er", gg.erdos_renyi, 1 << 14, 4 << 14, 11)),
        ("er-256k", gg.cached("er", gg.erdos_renyi, 1 << 18, 4 << 18, 12)),
        ("rmat-s12", gg.cached("rmat", gg.rmat, 12, 16, 13)),
        ("rmat-s16", gg.cached("rmat", gg.rmat, 16, 16, 14)),
        ("rmat-s20", gg.cached("rmat", gg.rmat, 20, 16, 15)),
        ("grid-256", gg.cached("grid", gg.grid2d, 256, 256, 16, 0.1)),
        ("grid-1024", gg.cached("grid", gg.grid2d, 1024, 1024, 17, 0.1)),
    ]


def serving_bench(bc, ctx, per_rate=300, lam0=8.0, lam_max=1024.0, seed=100):
    """Poisson arrivals of BC requests over the resident pool: graph uniform, k =
    floor(exp(U(0, ln 1024))) sources, exact list or sampled with probability 1/2; per_rate
    requests at each rate, the rate doubling from lam0 until completions fall behind
    arrivals (served rate below 0.8 lambda: throughput saturation).  Reports p50 / p99 of
    the latency (submit -> result), the served rate and the delivered GTEPS per rate; the
    latency knee (the first rate whose p99 is above 10 x the first rate's);
    capacity_gteps, the largest delivered GTEPS of the sweep; and offline_mix_gteps, the
    bound the same graph mix reaches when each graph runs its sources offline in batches of
    512."""
    pool = serving_pool()
    handles = [bc.bc_graph_create(ctx, g.n, g.row_ptr, g.col_idx, g.nnz, 0) for _, g in pool]
    for (_, g), h in zip(pool, handles):  # kernel choice per graph (not timed)
        if g.n > 4096:
            bc.bc_autotune(h, 64, 7)
    nonisolated = [np.flatnonzero(g.degrees() > 0).astype(np.int32) for _, g in pool]
    for gi, (_, g) in enumerate(pool):  # workspaces set up before the sweep
        buf = np.zeros(g.n, np.float64)
        rid = bc.bc_stream_submit(ctx, handles[gi], buf, bc.BC_REQ_EXACT_LIST, src=nonisolated[gi][:8])
        bc.bc_stream_poll(ctx, rid, -1)
    # the same graph mix run offline: each graph's throughput on 512 of its sources in one
    # bc_sources call (its tuned kernel), combined with the sweep's weights (graph uniform,
    # the same source count on average): total work over total time
    offline = {}
    for gi, (name, g) in enumerate(pool):
        src = np.random.Generator(np.random.PCG64(seed + gi)).choice(
            nonisolated[gi], size=min(512, nonisolated[gi].size), replace=False).astype(np.int32)
        bc.bc_sources(handles[gi], g.n, src[:8])
        _, st = bc.bc_sources(handles[gi], g.n, src)
        offline[name] = st["gteps"]
    mix_gteps = sum(g.m for _, g in pool) / sum(g.m / offline[name] for name, g in pool)
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    lam, p99_low, saturated, knee_lam = lam0, None, False, None
    while lam <= lam_max and not saturated:
        reqs = []
        t0 = time.perf_counter()
        t_next = 0.0
        for _ in range(per_rate):
            t_next += rng.exponential(1.0 / lam)
            gi = int(rng.integers(0, len(pool)))
            k = int(min(1024, max(1, np.floor(np.exp(rng.uniform(0.0, np.log(1024.0)))))))
            k = min(k, nonisolated[gi].size)
            exact = bool(rng.integers(0, 2))
            now = time.perf_counter() - t0
            if t_next > now:
                time.sleep(t_next - now)
            buf = np.zeros(pool[gi][1].n, np.float64)
            if exact:
                src = rng.choice(nonisolated[gi], size=k, replace=False).astype(np.int32)
                rid = bc.bc_stream_submit(ctx, handles[gi], buf, bc.BC_REQ_EXACT_LIST, src=src)
            else:
                rid = bc.bc_stream_submit(ctx, handles[gi], buf, bc.BC_REQ_SAMPLED, k=k,
                                          seed=int(rng.integers(0, 2**40)))
            reqs.append((rid, gi, k, buf))
        offered_s = time.perf_counter() - t0
        lat, edges_done = [], 0.0
        for rid, gi, k, buf in reqs:
            st, res = bc.bc_stream_poll(ctx, rid, -1)
            if res["status"] != bc.BC_OK:
                raise RuntimeError(f"serving request failed with status {res['status']}")
            lat.append(res["latency_seconds"])
            edges_done += k * pool[gi][1].m
        wall = time.perf_counter() - t0
        p50, p99 = float(np.percentile(lat, 50) * 1e3), float(np.percentile(lat, 99) * 1e3)
        served = per_rate / wall
        p99_low = p99 if p99_low is None else p99_low
        saturated = served < 0.8 * lam
        if knee_lam is None and p99 > 10.0 * p99_low:
            knee_lam = lam
        out.append({"lambda_per_s": lam, "requests": len(reqs), "p50_ms": p50, "p99_ms": p99,
                    "served_per_s": served, "gteps": edges_done / wall / 1e9, "wall_s": wall,
                    "offered_s": offered_s, "saturated": saturated,
                    "p99_above_10x_low_load": p99 > 10.0 * p99_low})
        lam *= 2.0
    for h in handles:
        bc.bc_destroy(h)
    knee = max(out, key=lambda r: r["gteps"])
    return {"pool": [name for name, _ in pool], "requests_per_rate": per_rate, "rates": out,
            "capacity_gteps": knee["gteps"], "capacity_lambda_per_s": knee["lambda_per_s"],
            "offline_mix_gteps": mix_gteps, "offline_gteps_per_graph": offline,
            "saturated_at_lambda_per_s": out[-1]["lambda_per_s"] if out[-1]["saturated"] else None,
            "latency_knee_lambda_per_s": knee_lam,
            "requests": "graph uniform; k = floor(exp(U(0, ln 1024))); exact list or sampled 1:1; "
                        "request-stream seed 100; rates doubling until the served rate < 0.8 lambda; "
                        "latency knee: first rate with p99 > 10x the first rate's"}


# ------------------------------------------------------------------ side configurations
def ba_pruning_bench(bc, ctx):
    """Leaf-rich preferential-attachment graph, n = 262144 (40% of arrivals attach once,
    the rest 8 times), seed 2: exact BC over all sources with and without the 1-degree
    removal (Eq. 3 / Eq. 4), tile width from the autotuner; GTEPS counts every
    non-isolated vertex as a source and the original m in both runs."""
    g = gg.cached("ba", gg.ba_pref_attach, 262144, 2)
    h = bc.bc_graph_create(ctx, g.n, g.row_ptr, g.col_idx, g.nnz, 0)
    tune = bc.bc_autotune(h, 0, 7)
    T = int(tune["tile_width"]) or 128
    flags = bc.BC_PATH_TILED | bc.BC_TILE(T)
    bc.bc_exact(h, g.n, flags | bc.BC_PRUNE_DEG1)  # warm-up (builds the residual graph)
    pruned, stp = bc.bc_exact(h, g.n, flags | bc.BC_PRUNE_DEG1)
    full, stf = bc.bc_exact(h, g.n, flags)
    bc.bc_destroy(h)
    err = np.abs(pruned - full) / np.maximum(np.abs(full), 1.0)
    return {"n": g.n, "m": g.m, "leaves": int(np.sum(g.degrees() == 1)), "tile_width": T,
            "pruned_gteps": stp["gteps"], "pruned_s": stp["seconds"], "pruned_sources": stp["sources"],
            "unpruned_gteps": stf["gteps"], "unpruned_s": stf["seconds"], "unpruned_sources": stf["sources"],
            "speedup": stf["seconds"] / stp["seconds"], "max_rel_diff": float(err.max())}


def grid_loop_bench(bc, ctx, T: int = 64):
    """2-D 1024 x 1024 grid, 10% of its edges deleted (seed 5), largest component; 1024
    sources uniform from it (seed 6), tiles of T: the level loop as one persistent
    cooperative kernel, as one launch per phase, and as CUDA-graph chunks of launches; and
    the per-source path with one source per CTA (the autotuner's choice on this graph)."""
    g = gg.cached("grid", gg.grid2d, 1024, 1024, 5, 0.1)
    src = gg.sample_sources(g, 1024, seed=6)
    h = bc.bc_graph_create(ctx, g.n, g.row_ptr, g.col_idx, g.nnz, 0)
    out = {"n": g.n, "m": g.m, "sources": int(src.size), "tile_width": T}
    modes = {"persistent": bc.BC_PATH_TILED | bc.BC_TILE(T),
             "per_level_launches": bc.BC_PATH_TILED | bc.BC_TILE(T) | bc.BC_LOOP_LAUNCH,
             "cuda_graph": bc.BC_PATH_TILED | bc.BC_TILE(T) | bc.BC_LOOP_GRAPH,
             "per_source_one_per_cta": bc.BC_PATH_PLAIN | bc.BC_PLAIN_CTA}
    for name, flags in modes.items():
        bc.bc_sources(h, g.n, src[:T], flags)
        _, st = bc.bc_sources(h, g.n, src, flags)
        out[name] = {"gteps": st["gteps"], "seconds": st["seconds"], "levels": st["levels"],
                     "kernel_launches": st["kernel_launches"]}
    bc.bc_destroy(h)
    return out


# ------------------------------------------------------------------ 1-degree study
def deg1_study(scale: int = 20, efs=(4, 16, 32), k: int = 1024, T: int = 64):
    """1-degree removal (Eq. 3 / Eq. 4, Alg. 6) on R-MAT graphs of one scale and several edge
    factors (seed 3): preprocessing time (device pruning plus the copies of omega and the
    residual CSR to the host), then the mean time per source of the tile path on the original
    graph (k sources drawn from the non-isolated vertices) and on the residual graph (k
    drawn from the residual vertices), and totals extrapolated to every source of each run,
    as the paper's totals are (the pruned run has fewer sources and fewer edges)."""
    import paper_1602_00963_gb300 as bc
    ctx = bc.bc_ctx_create(0)
    flags = bc.BC_PATH_TILED | bc.BC_TILE(T)
    rows = []
    for ef in efs:
        g = gg.cached("rmat", gg.rmat, scale, ef, 3)
        h = bc.bc_graph_create(ctx, g.n, g.row_ptr, g.col_idx, g.nnz, 0)
        bc.bc_prune(h, g.n, g.nnz)  # warm-up
        t = time.perf_counter()
        om, rem, rrp, rci = bc.bc_prune(h, g.n, g.nnz)
        t_pre = time.perf_counter() - t
        hr = bc.bc_graph_create(ctx, g.n, rrp, rci, rci.size, 0)
        deg = g.degrees()
        all_src = np.flatnonzero(deg > 0)
        res_src = np.flatnonzero((deg > 0) & (rem == 0))
        rng = np.random.Generator(np.random.PCG64(5))
        su = rng.choice(all_src, size=min(k, all_src.size), replace=False).astype(np.int32)
        sp = rng.choice(res_src, size=min(k, res_src.size), replace=False).astype(np.int32)
        bc.bc_sources(h, g.n, su[:T], flags)
        bc.bc_sources(hr, g.n, sp[:T], flags)
        _, stu = bc.bc_sources(h, g.n, su, flags)
        _, stp = bc.bc_sources(hr, g.n, sp, flags)
        per_u, per_p = stu["seconds"] / su.size, stp["seconds"] / sp.size
        tot_u, tot_p = per_u * all_src.size, per_p * res_src.size + t_pre
        rows.append({"edge_factor": ef, "n": g.n, "m": g.m, "leaves_removed": int(rem.sum()),
                     "sources_unpruned": int(all_src.size), "sources_pruned": int(res_src.size),
                     "residual_m": int(rci.size // 2), "preprocessing_s": t_pre,
                     "mean_ms_per_source_unpruned": per_u * 1e3, "mean_ms_per_source_pruned": per_p * 1e3,
                     "total_s_unpruned": tot_u, "total_s_pruned": tot_p, "speedup": tot_u / tot_p})
        bc.bc_destroy(hr)
        bc.bc_destroy(h)
    bc.bc_destroy(ctx)
    print(json.dumps({"study": "1-degree removal, R-MAT scale %d (seed 3), tiles of %d, %d sampled sources" % (scale, T, k),
                      "rows": rows}), flush=True)


def deg2_triples(g) -> int:
    """How many degree-2 runs the library derives: degree-2 vertices c taken in vertex
    order while c and both neighbours are unused (the rule of BC_DEG2)."""
    used = np.zeros(g.n, bool)
    cnt = 0
    for c in np.flatnonzero(g.degrees() == 2):
        a, b = g.col_idx[g.row_ptr[c]:g.row_ptr[c] + 2]
        if used[c] or used[a] or used[b]:
            continue
        used[[a, b, c]] = True
        cnt += 1
    return cnt


def deg2_study():
    """The two heuristics of Sec. 3.4 on road-network stand-ins small enough for the
    per-source CTA kernel, all sources, exact BC: H0 plain, H1 1-degree reduction, H2 the
    2-degree heuristic, H3 both (device time of the call), the degree-2 runs derived, and
    the largest relative difference of each result from H0."""
    import paper_1602_00963_gb300 as bc
    ctx = bc.bc_ctx_create(0)
    sub = gg.subdivide_edges(gg.grid2d(160, 160, seed=18, delete_frac=0.1), 0.4, 19)
    graphs = [("grid 256x256, 10% deleted, LCC", gg.cached("grid", gg.grid2d, 256, 256, 16, 0.1)),
              ("grid 160x160, 10% deleted, LCC, 40% of edges subdivided", sub),
              ("the same with 1-2 dead ends on 15% of the vertices", gg.attach_leaves(sub, 0.15, 20, 2))]
    P = bc.BC_PATH_PLAIN
    variants = {"H0": P, "H1": P | bc.BC_PRUNE_DEG1, "H2": P | bc.BC_DEG2,
                "H3": P | bc.BC_DEG2 | bc.BC_PRUNE_DEG1}
    rows = []
    for name, g in graphs:
        h = bc.bc_graph_create(ctx, g.n, g.row_ptr, g.col_idx, g.nnz, 0)
        bc.bc_sources(h, g.n, gg.sample_sources(g, 64, seed=1), P)  # workspace set-up
        res = {}
        for key, fl in variants.items():
            bc.bc_exact(h, g.n, fl)  # warm-up (and the 1-degree preprocessing, cached)
            res[key] = bc.bc_exact(h, g.n, fl)
        b0, s0 = res["H0"]
        deg = g.degrees()
        omega, removed, rrp, rci = bc.bc_prune(h, g.n, g.nnz)
        resg = gg.Graph(g.n, rrp, rci, g.name + "-res")
        row = {"graph": name, "n": g.n, "m": g.m, "degree1_vertices": int((deg == 1).sum()),
               "leaves_removed": int(removed.sum()), "degree2_vertices": int((deg == 2).sum()),
               "derived_runs_H2": deg2_triples(g), "derived_runs_H3": deg2_triples(resg),
               "sources_H0": int((deg > 0).sum()), "seconds_H0": s0["seconds"]}
        for key in ("H1", "H2", "H3"):
            bk, sk = res[key]
            row[f"seconds_{key}"] = sk["seconds"]
            row[f"speedup_{key}"] = s0["seconds"] / sk["seconds"]
            row[f"max_rel_diff_{key}"] = float((np.abs(bk - b0) / np.maximum(np.abs(b0), 1.0)).max())
        rows.append(row)
        bc.bc_destroy(h)
    bc.bc_destroy(ctx)
    print(json.dumps({"study": "heuristics H0-H3, per-source path (one source per CTA), all sources",
                      "rows": rows}), flush=True)


def scan_study():
    """Sec. 3.1's reuse of the forward sweep's degree prefix CD in the backward sweep,
    measured on the grid-wide per-source kernel: the same sources with the reuse and with
    CD scanned again per backward level (BC_NO_CD_REUSE), device time of the call, on a
    short-diameter R-MAT and on long-diameter grids (the paper's comparison of Sec. 4)."""
    import paper_1602_00963_gb300 as bc
    ctx = bc.bc_ctx_create(0)
    cases = [("R-MAT scale 16, EF 16, seed 5", gg.rmat(16, 16, 5), 256),
             ("grid 256x256, 10% deleted, LCC", gg.cached("grid", gg.grid2d, 256, 256, 16, 0.1), 64),
             ("grid 1024x1024, 10% deleted, LCC", gg.cached("grid", gg.grid2d, 1024, 1024, 5, 0.1), 16)]
    G = bc.BC_PATH_PLAIN | bc.BC_PLAIN_GRID
    rows = []
    for name, g, k in cases:
        src = gg.sample_sources(g, k, seed=7)
        h = bc.bc_graph_create(ctx, g.n, g.row_ptr, g.col_idx, g.nnz, 0)
        res = {}
        for key, fl in (("reuse", G), ("rescan", G | bc.BC_NO_CD_REUSE)):
            bc.bc_sources(h, g.n, src[:4], fl)
            res[key] = bc.bc_sources(h, g.n, src, fl)
        (b0, s0), (b1, s1) = res["reuse"], res["rescan"]
        rows.append({"graph": name, "n": g.n, "m": g.m, "sources": k,
                     "levels_per_source": s0["levels"] / k,
                     "seconds_reuse": s0["seconds"], "seconds_rescan": s1["seconds"],
                     "gain_of_reuse": s1["seconds"] / s0["seconds"] - 1.0,
                     "gteps_reuse": s0["gteps"], "gteps_rescan": s1["gteps"],
                     "max_rel_diff": float((np.abs(b1 - b0) / np.maximum(np.abs(b0), 1.0)).max())})
        bc.bc_destroy(h)
    bc.bc_destroy(ctx)
    print(json.dumps({"study": "degree-prefix reuse (Sec. 3.1), grid-wide per-source kernel",
                      "rows": rows}), flush=True)


# ------------------------------------------------------------------ our arm
def main():
    args = parse()
    rank, world, local = dist_env()
    if args.profile_case:
        profile_case(args.profile_case)
        return
    if args.study == "deg1":
        deg1_study()
        return
    if args.study == "deg2":
        deg2_study()
        return
    if args.study == "scan":
        scan_study()
        return
    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, rank, world)
        return
    import torch
    import paper_1602_00963_gb300 as bc
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    g, src = load_workload(args.sources, rank)
    ctx = bc.bc_ctx_create(local)
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    h = bc.bc_graph_create(ctx, g.n, rp, ci, g.nnz, bc.BC_VALIDATE)
    dsrc = torch.from_numpy(src).cuda()
    dbc = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    # tile width (and direction-switch threshold) from the autotuner
    tune = None
    try:
        tune = bc.bc_autotune(h, 0, 7)
    except bc.BCError:
        tune = None
    sweep = {}
    if tune is None or not args.quick:
        for T in (32, 64, 128, 256):
            s512 = dsrc[:512]
            bc.bc_sources(h, g.n, s512, bc.BC_PATH_TILED | bc.BC_TILE(T), bc_out=dbc, stream=stream)
            _, st = bc.bc_sources(h, g.n, s512, bc.BC_PATH_TILED | bc.BC_TILE(T), bc_out=dbc, stream=stream)
            sweep[T] = st["gteps"]
    if tune is not None and tune["tile_width"] > 0:
        T = int(tune["tile_width"])
    else:
        T = max(sweep, key=sweep.get)
    flags = bc.BC_PATH_TILED | bc.BC_TILE(T)

    for _ in range(args.warmup):
        bc.bc_sources(h, g.n, dsrc, flags, bc_out=dbc, stream=stream)
        reduce_bc(dbc, dist)
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    stats = []
    with ClockSampler(local) as clk:
        barrier()
        ev0.record()
        for _ in range(args.steps):
            _, st = bc.bc_sources(h, g.n, dsrc, flags, bc_out=dbc, stream=stream)
            reduce_bc(dbc, dist)  # the job's BC over every rank's sources (N > 1)
            stats.append(st)
        ev1.record()
        barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    per_step_ms = ms / args.steps
    total_sources = args.sources * world
    value = total_sources * g.m / (per_step_ms * 1e-3) / 1e9

    # roofline of the dominant kernel (the tile kernel: one launch per tile)
    st0 = stats[-1]
    launches = sum(s["kernel_launches"] for s in stats)
    tiles = (args.sources + T - 1) // T
    kernel_s = sum(s["seconds"] for s in stats)  # CUDA events around each tile, library stream
    avg_launch_s = kernel_s / (tiles * args.steps)
    bytes_per_launch = algorithmic_bytes(st0, T) / tiles
    peak, peak_kind = measured_peaks()
    achieved = bytes_per_launch / avg_launch_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": ncu_traffic(T, tiles_bytes=bytes_per_launch),
                "peak_kind": peak_kind,
                "kernel": f"tile_persistent (T={T}), one launch per tile of {T} sources",
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "avg_launch_ms": avg_launch_s * 1e3}

    # end to end through the public API with host (pinned) buffers: graph upload, sources
    # in, BC out, inside the timed region (numpy views of pinned tensors: no staging copy)
    hrp = torch.from_numpy(g.row_ptr).pin_memory().numpy()
    hci = torch.from_numpy(g.col_idx).pin_memory().numpy()
    hsrc = torch.from_numpy(src).pin_memory().numpy()
    hbc = torch.zeros(g.n, dtype=torch.float64).pin_memory().numpy()
    times = []
    for _ in range(args.steps):
        barrier()
        t = time.perf_counter()
        gh = bc.bc_graph_create(ctx, g.n, hrp, hci, g.nnz, 0)
        bc.bc_sources(gh, g.n, hsrc, flags, bc_out=hbc)
        times.append(time.perf_counter() - t)
        bc.bc_destroy(gh)
    e_dt = max_over_ranks(statistics.median(times), dist, "cuda")
    e2e = {"value": total_sources * g.m / e_dt / 1e9, "unit": "GTEPS",
           "h2d_bytes_per_step": int(g.row_ptr.nbytes + g.col_idx.nbytes + src.nbytes),
           "d2h_bytes_per_step": int(g.n * 8), "seconds_per_step": e_dt,
           "steps": args.steps, "statistic": "median over steps",
           "includes": "graph upload (CSR), sources, BC download; untuned thresholds"
                       + ("; the ranks' BC not summed (host buffers)" if world > 1 else "")}

    side = {}
    if not args.quick and rank == 0:
        # per-source path on a sample of the same sources
        s_plain = dsrc[:128]
        bc.bc_sources(h, g.n, s_plain[:8], bc.BC_PATH_PLAIN, bc_out=dbc, stream=stream)
        _, stp = bc.bc_sources(h, g.n, s_plain, bc.BC_PATH_PLAIN, bc_out=dbc, stream=stream)
        side["per_source_path_gteps"] = stp["gteps"]
        side["per_source_path_sample"] = "128 of the 4096 sources"
        side["per_source_roofline_frac"] = (algorithmic_bytes(stp, 1) / stp["seconds"] / 1e9) / peak
        side["tile_sweep_gteps_512_sources"] = sweep
        # the same step with the sources in the given order (no locality grouping)
        bc.bc_sources(h, g.n, dsrc, flags | bc.BC_KEEP_ORDER, bc_out=dbc, stream=stream)
        _, sk = bc.bc_sources(h, g.n, dsrc, flags | bc.BC_KEEP_ORDER, bc_out=dbc, stream=stream)
        side["given_order_gteps"] = sk["gteps"]
        # R-MAT scale 12, all sources: per-source path vs tiles
        g12 = gg.rmat(12, 16, 1)
        h12 = bc.bc_graph_create(ctx, g12.n, g12.row_ptr, g12.col_idx, g12.nnz, 0)
        bc.bc_exact(h12, g12.n, bc.BC_PATH_PLAIN)
        _, sp = bc.bc_exact(h12, g12.n, bc.BC_PATH_PLAIN)
        _, stl = bc.bc_exact(h12, g12.n, bc.BC_PATH_TILED | bc.BC_TILE(256))
        side["rmat12_all_sources_gteps"] = {"per_source": sp["gteps"], "tile256": stl["gteps"]}
        bc.bc_destroy(h12)
        side["ba262144_all_sources"] = ba_pruning_bench(bc, ctx)
        side["grid1024_loop_modes"] = grid_loop_bench(bc, ctx)
        side["serving"] = serving_bench(bc, ctx)

    cpu = None
    if rank == 0:
        cpu, _ = cpu_baseline(g, src, budget_s=15.0)

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per_step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE, "data": "synthetic",
            "config": dict(WORKLOAD, tile_width=T, autotuned=tune is not None,
                           l2="inputs larger than L2 (CSR 126 MB, tile state > 1 GB)",
                           m=g.m, n=g.n, parallelism=f"sources split over {world} rank(s), "
                           "BC summed by one all-reduce per step" if world > 1 else "1 GPU"),
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
        }
        line.update(side)
        print(json.dumps(line), flush=True)
    bc.bc_destroy(h)
    bc.bc_destroy(ctx)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
