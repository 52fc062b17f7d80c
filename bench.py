"""Benchmark of the R-distance hot path on GB300 (one JSON line on stdout).

Workload (the n = 8192 single-graph configuration): six seeded graphs -- directed ER p=0.01,
the 4-neighbour grid with 91 columns (90 full rows + 2), and the Watts-Strogatz ring (k=10,
beta=0.1) -- each at gain 0.5/Delta and 0.9/Delta.  One step = the whole hot path on one
graph, cycling through the six: rd_load (gain check + M), rd_apsp (LU, triangular inverses,
product with the fused decode into int32 D), rd_goal_solve for 64 goals and rd_greedy_next.
The headline is the split-precision path (--precision split, the default); the FP64 path is
timed beside it ("compare") and D of all six graphs is checked against the oracle for both.

value   = effective TFLOP/s, 2 n^3 per step (the dense inverse's flop count) over the device
          time of the step, summed over ranks (replicas) and divided by the slowest rank's time.
e2e     = the same metric through the C ABI with host buffers: the graph is copied from pinned
          host memory and D, the goal rows and the next hops are copied back, every step.
roofline= the dense-contraction kernel, algorithmic flops / its event-timed duration over the
          timed region, against the measured (or nominal) peak of its arithmetic.

--impl reference times the CPU oracle (single thread, FP64) on a bounded sample of the same
workload instead (the leading principal submatrix of each graph).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "n=8192 R-distance APSP time/TFLOPS, split-prec vs FP64 (D exact); p50/p99"
# DRAM bytes (read + write) per split GEMM launch of the headline workload: the mean over the 648
# launches of six steps (all six graphs) in one one-pass ncu capture of this kernel build, and the
# algorithmic bytes per launch (the digit tiles each product needs at least once plus its outputs,
# same launches); profiles/launches_apsp_split_n8192.md gives the command and the model.  To be
# captured again whenever split_gemm_kernel changes.
SPLIT_TRAFFIC_PER_LAUNCH = 0.3612e9
# DRAM bytes of the inverse product launch of `--workload product` (ER n = 4096, 9 digits, CTA pairs),
# one one-pass ncu capture (profiles/split_gemm_pairs_inverse_product_n4096.md); None until taken
PRODUCT_TRAFFIC = 1.0339e9
SPLIT_ALGORITHMIC_BYTES_PER_LAUNCH = 0.1389e9
GOLDEN = os.path.join(ROOT, "tests", "golden")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=6)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="split", choices=["fp64", "split"])
    p.add_argument("--compare-steps", type=int, default=2, help="steps of the other precision, 0 = skip")
    p.add_argument("--slices", type=int, default=0)
    p.add_argument("--n", type=int, default=8192)
    p.add_argument("--goals", type=int, default=64)
    p.add_argument("--e2e-steps", type=int, default=6,
                   help="end-to-end steps (host buffers); 6 = each of the six graphs once, the mix of the timed steps")
    p.add_argument("--verify", type=int, default=1, help="hash D of every graph against the oracle's")
    p.add_argument("--cpu-sample", type=int, default=1536, help="oracle sample size (leading block)")
    p.add_argument("--workload", default="single", choices=["single", "batched", "batched-stack", "serving", "weighted",
                                                            "update", "product", "mma-probe"],
                   help="single: the n=8192 graphs (default); batched: 4096 graphs n~U[32,512] in one launch; "
                        "serving: a Poisson stream of requests over a pool of graphs; "
                        "weighted: n=32768 king grid, split inverse + 1024 goal rows + greedy; "
                        "update: edge removals and restores on the n=8192 grid (Sherman-Morrison); "
                        "product: the inverse product with the fused decode alone, on resident split factors")
    p.add_argument("--obstacles", type=int, default=64, help="update: edge pairs removed, then restored")
    p.add_argument("--product-n", type=int, default=4096, help="product: graph size")
    p.add_argument("--product-graph", default="er", choices=["er", "grid"],
                   help="product: ER p=0.01 (natural order, 256-wide chunks) or a 4-neighbour grid "
                        "(locality order, 64-wide chunks)")
    p.add_argument("--split-stats", action="store_true",
                   help="product: run the diagnostic build with the split GEMM's cycle counters and report "
                        "where the kernel's time goes (the counters slow the kernel by a few percent)")
    p.add_argument("--weighted-rows", type=int, default=128)
    p.add_argument("--weighted-cols", type=int, default=256)
    p.add_argument("--weighted-frac", type=float, default=0.9, help="weighted: gain as a fraction of the weighted bound")
    p.add_argument("--batch-graphs", type=int, default=4096)
    p.add_argument("--serve-seconds", type=float, default=60.0, help="serving: length of the arrival stream")
    p.add_argument("--serve-rate", type=float, default=200.0, help="serving: Poisson arrival rate (req/s)")
    return p.parse_args()


def workloads(n):
    from paper_2308_07403_gb300 import graphs

    out = []
    for kind in graphs.LARGE_KINDS:
        base = None
        for frac in graphs.LARGE_FRACS:
            if base is None:
                base, _ = graphs.workload_large(kind, frac, n=n)
            out.append((kind, frac, base, graphs.gamma_frac(base, frac)))
    return out


# ---- clocks --------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- peaks ---------------------------------------------------------------------------------

def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---- reference arm (the CPU oracle) ----------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    oracle.build()
    wl = workloads(args.n)
    m = min(args.cpu_sample, args.n)
    times = []
    for step in range(args.warmup + args.steps):
        kind, frac, A, g = wl[step % len(wl)]
        As = np.ascontiguousarray(A[:m, :m])
        gs = 0.5 / max(1, int(As.sum(axis=0).max())) if frac == 0.5 else 0.9 / max(1, int(As.sum(axis=0).max()))
        t0 = time.perf_counter()
        oracle.rdistance(As, gs)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    t = float(np.mean(times))
    val = 2.0 * m ** 3 / t / 1e12
    sample = (f"CPU oracle (1 thread, FP64 LU + column solves + decode) on the leading {m}x{m} "
              f"principal submatrix of each n={args.n} graph; rate = 2 m^3 / t")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"n={args.n} single graphs (ER p=0.01, grid 90x91, WS k=10 beta=0.1) "
                               f"at gain 0.5 and 0.9 x 1/Delta; oracle sample m={m}",
                   "n": args.n, "sample_n": m},
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(args, A):
    import oracle

    oracle.build()
    m = min(args.cpu_sample, args.n)
    As = np.ascontiguousarray(A[:m, :m])
    gs = 0.5 / max(1, int(As.sum(axis=0).max()))
    t0 = time.perf_counter()
    oracle.rdistance(As, gs)
    t = time.perf_counter() - t0
    return {"value": 2.0 * m ** 3 / t / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
            "sample": f"CPU oracle (1 thread, FP64) on the leading {m}x{m} principal submatrix of the "
                      f"n={args.n} ER graph, {t:.2f} s; rate = 2 m^3 / t"}


# ---- our arm ---------------------------------------------------------------------------------

def time_path(rd, h, step, first, steps, warmup, stream, local, world, dist, profile=True):
    """Warm up, then time `steps` calls of step(i) with CUDA events on the handle's stream.

    Returns per-step ms, total ms (max over ranks), the stats delta and the clock record."""
    import torch

    for i in range(warmup):
        step(first + i)
    torch.cuda.synchronize()
    st0 = rd.rd_get_stats(h)
    if profile:
        # (2: events around the split GEMM alone, whose roofline the line reports; True: every
        # dense-contraction kernel)
        rd.rd_set_profiling(h, profile)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    for i in range(steps):
        step(first + warmup + i)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    per_step = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    total = ev[0].elapsed_time(ev[-1])
    st1 = rd.rd_get_stats(h)
    if profile:
        rd.rd_set_profiling(h, False)
    total = reduce_max(total, dist, world, f"cuda:{local}")
    return per_step, total, st0, st1, clk


def reduce_max(x, dist, world, device):
    """Largest value over the ranks (every rank gets it); the slowest replica sets the time."""
    if world <= 1:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, flop_per_step, steps, total_ms):
    """Whole-job rate in TFLOP/s: every replica processed `steps` steps; time is the slowest."""
    return world * flop_per_step * steps / (total_ms * 1e-3) / 1e12


def bfs_fraction(A, D, sources):
    """Fraction of the D entries of the sampled source columns equal to BFS hop distance (scipy:
    a library BFS, not the oracle); D[i, j] is the distance j -> i, unreachable = INT32_MAX."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import shortest_path

    G = sp.csr_matrix(np.ascontiguousarray(A.T))  # G[u, v] = 1 for the edge u -> v
    dist = shortest_path(G, unweighted=True, indices=sources)  # dist[k, i]: sources[k] -> i
    truth = np.where(np.isinf(dist), np.iinfo(np.int32).max, dist).astype(np.int64)
    got = D[:, sources].T.astype(np.int64)
    return float(np.mean(got == truth))


def verify_graphs(rd, h, wl, A_dev, modes, args, other, D, dev):
    import torch

    names = [args.precision] + ([other] if other else [])
    out = {nm: {"graphs_D_identical_to_oracle": 0, "graphs_checked": 0} for nm in names}
    per_graph = {}
    sources = np.linspace(0, args.n - 1, 256).astype(np.int64)
    n = args.n
    Ys = {nm: torch.empty((n, n), dtype=torch.float64, device=dev) for nm in names}
    Ds = {nm: torch.empty((n, n), dtype=torch.int32, device=dev) for nm in names}
    for i, (kind, frac, A, g) in enumerate(wl):
        path = os.path.join(GOLDEN, f"large_{kind}_{frac}.json")
        if not os.path.exists(path):
            continue
        with open(path) as f:
            gold = json.load(f)
        rec = {}
        for nm in names:
            rd.rd_set_precision(h, modes[nm], args.slices if nm == args.precision else 0)
            rd.rd_load(h, A_dev[i // 2], None, g)
            f0 = rd.rd_get_stats(h)["fallbacks"]
            rd.rd_apsp(h, Ds[nm], Ys[nm])
            torch.cuda.synchronize()
            sg = rd.rd_get_stats(h)
            Dh = Ds[nm].cpu().numpy()
            same = hashlib.sha256(Dh.astype("<i4").tobytes()).hexdigest() == gold["sha256_D"]
            out[nm]["graphs_checked"] += 1
            out[nm]["graphs_D_identical_to_oracle"] += int(same)
            if nm == "split":
                redone = sg["fallbacks"] > f0
                rec["split"] = {"precision_used": "split" if sg["precision_used"] else "fp64",
                                "digits": sg["slices"] if sg["precision_used"] else None,
                                "screen_bits": round(sg["split_screen_bits"], 1),
                                "locality_order": ["none", "landmark", "scored"][sg["split_order"]],
                                "sampled_row_residual": sg["split_residual"] if sg["precision_used"] else None,
                                "redone_by_self_check": bool(redone)}
            if nm == args.precision:
                rec["bfs_match_fraction"] = bfs_fraction(A, Dh, sources)
        if other:
            Yf, Yo = Ys["fp64"], Ys["split"]
            pos = Yf > 0
            rel = torch.where(pos, (Yo - Yf).abs() / torch.where(pos, Yf, torch.ones_like(Yf)), torch.zeros_like(Yf))
            rec["split_vs_fp64"] = {"max_rel_err_Y": float(rel.max().item()),
                                    "zero_pattern_equal": bool(torch.equal(Yo == 0, Yf == 0)),
                                    "D_mismatches": int((Ds["split"] != Ds["fp64"]).sum().item())}
        per_graph[f"{kind}_{frac}"] = rec
    for nm in names:
        if nm == "split":
            recs = [r["split"] for r in per_graph.values() if "split" in r]
            out[nm]["graphs_fp64_by_range_screen"] = sum(r["precision_used"] == "fp64" and not r["redone_by_self_check"]
                                                         for r in recs)
            out[nm]["graphs_redone_in_fp64_by_self_check"] = sum(r["precision_used"] == "fp64" and
                                                                 r["redone_by_self_check"] for r in recs)
    out["per_graph"] = per_graph
    out["bfs_sample"] = "256 evenly spaced source columns per graph (scipy shortest_path, unweighted)"
    rd.rd_set_precision(h, modes[args.precision], args.slices)
    return out


def pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(round(q * (len(xs) - 1))))]


BATCH_METRIC = "batched R-distance APSP, 4096 graphs n~U[32,512] (ER/grid/WS), graphs/s"


def time_batch(b, A_dev, D_dev, steps, warmup, dev, local, world, dist):
    """Capture one rd_batch_apsp in a CUDA graph, replay it warmup times, then time `steps`
    replays with CUDA events (max over ranks); returns per-step ms, total ms and the clock record."""
    import torch

    stream = torch.cuda.Stream(dev)
    b.apsp(A_dev, D_dev, stream.cuda_stream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        b.apsp(A_dev, D_dev, stream.cuda_stream)
    for _ in range(warmup):
        graph.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    cur = torch.cuda.current_stream(dev)
    ev[0].record(cur)
    for i in range(steps):
        graph.replay()
        ev[i + 1].record(cur)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    tot = reduce_max(ev[0].elapsed_time(ev[-1]), dist, world, f"cuda:{local}")
    return per, tot, clk


def run_batched_stack(args):
    """One stack of 152 seeded directed ER graphs (p = 4/n, n uniform in [480, 512], gain 0.5/(Delta+1))
    with every size class on the split path (autotune off), against the FP64 Gauss-Jordan kernel on the
    same batch: the batched split variant where it is meant to win.  Each variant is one CUDA-graph
    replay per step; D of both is compared graph by graph."""
    import torch

    from paper_2308_07403_gb300 import build, graphs, rd

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    rd.load()
    rng = np.random.default_rng(2308_07403 + 3000)
    ns = rng.integers(480, 513, size=152).astype(np.int32)
    As = [graphs.er(int(n), 4.0 / n, int(rng.integers(1 << 30))) for n in ns]
    gs = np.array([graphs.gamma_small(A) for A in As])
    flop = float((2.0 * ns.astype(np.float64) ** 3).sum())
    b = rd.Batch(ns, gs)
    off = b.offsets()
    A_host = torch.empty(int(off[-1]), dtype=torch.uint8).pin_memory()
    A_np = A_host.numpy()
    for g, A in enumerate(As):
        A_np[off[g]:off[g + 1]] = A.ravel()
    A_dev = A_host.to(dev)
    D_dev = torch.empty(int(off[-1]), dtype=torch.int32, device=dev)
    steps, warmup = max(1, args.steps), max(3, args.warmup)
    _, tot64, clk64 = time_batch(b, A_dev, D_dev, steps, warmup, dev, local, 1, None)
    D64 = D_dev.cpu()
    b.set_precision(rd.RD_PREC_SPLIT_BF16, False)
    per, tot, clk = time_batch(b, A_dev, D_dev, steps, warmup, dev, local, 1, None)
    routes = b.routes()
    info = b.split_info()
    launches = b.tuning()["launches_last_run"]
    same = bool(torch.equal(D_dev.cpu(), D64))
    b.close()
    ms, ms64 = tot / steps, tot64 / steps
    on_split = routes == 1
    digits = {int(d): int((info["digits"][on_split] == d).sum()) for d in sorted(set(info["digits"][on_split].tolist()))}
    line = {
        "metric": "batched split stack: 152 ER graphs n~U[480,512], ms per batch (split variant vs FP64 kernel)",
        "value": ms, "unit": "ms", "n_gpus": 1, "steps": steps, "warmup": warmup, "ms_per_step": ms,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "bf16-digits+f64",
        "data": "synthetic",
        "config": {"workload": "152 directed ER graphs, p = 4/n, n uniform in [480, 512], gain 0.5/(Delta+1); "
                               "every size class on the split path (autotune off); one CUDA-graph replay per step"},
        "fp64_ms_per_step": ms64, "speedup_over_fp64": ms64 / ms, "effective_tflops": flop / (ms * 1e-3) / 1e12,
        "routes": {"split": int((routes == 1).sum()), "split_redone_fp64": int((routes == 2).sum()),
                   "screened_to_fp64": int((routes == 3).sum()), "gain_failed": int((routes == 4).sum())},
        "second_pass": int(((info["passes"] > 1) & on_split).sum()), "digits_histogram": digits,
        "screen_bits": [float(np.min(info["screen_bits"])), float(np.max(info["screen_bits"]))],
        "largest_residual_kept": float(np.max(info["residual"][on_split])) if on_split.any() else None,
        "D_identical_to_fp64_variant": same, "gpu_launches": int(launches), "clocks": clk,
        "e2e": None, "cpu_baseline": None,
        "roofline": {"bound": "latency", "note": "a stack of small products; the kernels' rooflines are the "
                                                 "single-graph and product lines'", "traffic": None},
    }
    print(json.dumps(line), flush=True)


def run_batched(args):
    """The batched workload: every graph of the batch through the whole method (rd_batch_apsp),
    captured once in a CUDA graph and replayed per step, in two variants: the split variant with
    the per-size-class choice of the library's autotuner (the headline) and the FP64 Gauss-Jordan
    kernel alone (compare); D of both is compared graph by graph."""
    import torch
    import torch.distributed as dist

    from paper_2308_07403_gb300 import build, graphs, rd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    rd.load()
    if args.impl == "reference":
        raise SystemExit("the batched workload has no reference arm of its own")
    kinds, ns, As, gs = graphs.workload_batched(args.batch_graphs, replica=rank)
    flop = float((2.0 * ns.astype(np.float64) ** 3).sum())
    b = rd.Batch(ns, gs)
    off = b.offsets()
    total = int(off[-1])
    A_host = torch.empty(total, dtype=torch.uint8).pin_memory()
    A_np = A_host.numpy()
    for g, A in enumerate(As):
        A_np[off[g]:off[g + 1]] = A.ravel()
    A_dev = A_host.to(dev)
    D_dev = torch.empty(total, dtype=torch.int32, device=dev)
    # the FP64 variant: one memset and the persistent Gauss-Jordan kernel per step
    per64, tot64, clk64 = time_batch(b, A_dev, D_dev, args.steps, args.warmup, dev, local, world, dist)
    st64 = b.status()
    D64 = D_dev.cpu()
    ms64 = tot64 / args.steps
    # the split variant, size classes chosen by the autotuner (timed on probe graphs at set-up)
    t_tune = time.perf_counter()
    b.set_precision(rd.RD_PREC_SPLIT_BF16, True)
    t_tune = time.perf_counter() - t_tune
    tune = b.tuning()
    per, tot, clk = time_batch(b, A_dev, D_dev, args.steps, args.warmup, dev, local, world, dist)
    st = b.status()
    routes = b.routes()
    info = b.split_info()
    launches = b.tuning()["launches_last_run"]
    same_as_fp64 = bool(torch.equal(D_dev.cpu(), D64))
    ms = tot / args.steps
    value = world * len(ns) * args.steps / (tot * 1e-3)
    # end to end through the C ABI: A from pinned host memory in, D out to pinned host memory
    D_host = torch.empty(total, dtype=torch.int32).pin_memory()
    te0 = time.perf_counter()
    for _ in range(max(1, args.e2e_steps)):
        A_dev.copy_(A_host, non_blocking=True)
        b.apsp(A_dev, D_dev, torch.cuda.current_stream(dev).cuda_stream)
        D_host.copy_(D_dev, non_blocking=True)
        torch.cuda.synchronize()
    te = reduce_max((time.perf_counter() - te0) / max(1, args.e2e_steps), dist, world, f"cuda:{local}")
    sm_mhz = clk64.get("sm_mhz") or 2070.0
    peak = 152 * 2 * 2 * sm_mhz * 1e6 / 1e12
    achieved64 = flop / (ms64 * 1e-3) / 1e12
    achieved = flop / (ms * 1e-3) / 1e12
    b.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1:
        import oracle

        oracle.build()
        sample = list(range(0, len(ns), max(1, len(ns) // 64)))[:64]
        t0 = time.perf_counter()
        for g in sample:
            oracle.rdistance(As[g], float(gs[g]))
        tcpu = time.perf_counter() - t0
        scale = flop / float((2.0 * ns[sample].astype(np.float64) ** 3).sum())
        cpu = {"value": len(ns) / (tcpu * scale), "unit": "graphs/s", "cores": 1, "kind": "oracle",
               "sample": f"CPU oracle (1 thread, FP64) on {len(sample)} evenly spaced graphs of the batch, "
                         f"{tcpu:.2f} s, scaled to the batch by sum 2 n^3"}
    rh = {name: int((routes == k).sum()) for k, name in
          enumerate(["fp64_class", "split", "split_redone_fp64", "screened_to_fp64", "gain_failed"])}
    line = {
        "metric": BATCH_METRIC, "value": value, "unit": "graphs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16-digits+f64", "data": "synthetic",
        "config": {"workload": f"{len(ns)} graphs, n uniform in [32, 512], kind uniform over ER p=4/n, "
                               f"grid ceil(sqrt n) columns, WS k=10 beta=0.1; gain 0.5/(Delta+1)",
                   "graphs": len(ns), "sum_2n3_flop": flop, "sum_n2": total,
                   "variant": "split (size classes chosen by the autotuner), FP64 Gauss-Jordan for the rest",
                   "launch": "one CUDA graph per step (split stacks, then the persistent FP64 kernel)",
                   "l2": "no flush: FP64 workspace 8 sum n^2 = %.2f GB > 129 MB L2" % (8 * total / 1e9),
                   "parallelism": f"replicas x{world}"},
        "p50_ms": pct(per, 0.5), "p99_ms": pct(per, 0.99), "tflops_2n3": achieved,
        "graphs_ok": int((st == rd.RD_OK).sum()), "graphs": len(ns),
        "routes": rh, "D_identical_to_fp64_variant": same_as_fp64,
        "split_digits_histogram": {int(d): int(c) for d, c in enumerate(np.bincount(info["digits"])) if c and d},
        "split_second_pass": int((info["passes"] == 2).sum()),
        "autotuner": dict(tune, seconds=round(t_tune, 2),
                          class_n_range=["(0,128]", "(128,256]", "(256,384]", "(384,512]"]),
        "compare": {"variant": "fp64 Gauss-Jordan, one persistent kernel", "value": world * len(ns) * args.steps /
                    (tot64 * 1e-3), "unit": "graphs/s", "ms_per_step": ms64, "p50_ms": pct(per64, 0.5),
                    "p99_ms": pct(per64, 0.99), "graphs_ok": int((st64 == rd.RD_OK).sum()),
                    "tflops": achieved64, "clocks": clk64,
                    "roofline": {"kernel": "batch_kernel", "bound": "alu",
                                 "peak_source": f"FP64 pipe: 152 SMs x 4 flop/clk x {sm_mhz:.0f} MHz (unit counts)",
                                 "achieved": achieved64, "peak": peak, "unit": "TFLOP/s",
                                 "frac": achieved64 / peak}},
        "clocks": clk, "gpu_launches": launches,
        "roofline": {"kernel": "batch_kernel (FP64 variant)", "bound": "alu",
                     "peak_source": f"FP64 pipe: 152 SMs x 4 flop/clk x {sm_mhz:.0f} MHz (unit counts)",
                     "achieved": achieved64, "peak": peak, "unit": "TFLOP/s", "frac": achieved64 / peak,
                     "traffic": None},
        "e2e": {"value": world * len(ns) / te, "unit": "graphs/s", "ms_per_step": te * 1e3,
                "h2d_bytes_per_step": total, "d2h_bytes_per_step": 4 * total},
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def serve_cpu_baseline(pool, plan, budget_s=10.0):
    """The oracle serving the stream's first requests on one core (graphs of at most 1024 nodes,
    in stream order, until about budget_s seconds of work): requests per second."""
    import oracle

    oracle.build()
    done, t0 = 0, time.perf_counter()
    for _, gid, goals in plan:
        A, g = pool[gid][0], pool[gid][1]
        if A.shape[0] > 1024:
            continue
        if goals is None:
            oracle.rdistance(A, g)
        else:
            oracle.goal_rows(A, g, goals)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    t = time.perf_counter() - t0
    return {"value": done / t, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"the stream's first {done} requests on graphs of at most 1024 nodes, in order, one core "
                      "(the larger graphs of the pool are left out: the oracle is O(n^3) per request)"}


def serve_metric(rate):
    return f"serving: Poisson {rate:g} req/s over 128 graphs n log-uniform [64,4096], solves/s (p50/p99 latency)"


def run_serving(args):
    """The serving workload: requests arrive as a Poisson stream (25 % full APSP, else 1..64 goal
    rows) over a pool of graphs and run on the library's server (continuous batching over 8
    workers, resident factors per graph).  Latency is the library's submit-to-completion time."""
    import queue
    import threading

    import torch

    from paper_2308_07403_gb300 import build, graphs, rd

    if int(os.environ.get("WORLD_SIZE", "1")) > 1 and int(os.environ.get("RANK", "0")) != 0:
        return  # one server per process would compete for the same budget: rank 0 serves
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build.build()
    rd.load()
    pool = graphs.serving_pool()
    rng = np.random.default_rng(graphs.seed_for(3, 1))
    t = 0.0
    plan = []
    while True:
        t += rng.exponential(1.0 / args.serve_rate)
        if t > args.serve_seconds:
            break
        gid = int(rng.integers(len(pool)))
        n = pool[gid][0].shape[0]
        if rng.random() < 0.25:
            plan.append((t, gid, None))
        else:
            k = int(rng.integers(1, 65))
            plan.append((t, gid, np.sort(rng.choice(n, size=min(k, n), replace=False)).astype(np.int32)))
    done_q = queue.Queue()
    statuses = []

    def waiter():
        while True:
            rid = done_q.get()
            if rid is None:
                return
            statuses.append(srv.wait(rid))

    srv = rd.Server(128 << 30, workers=8)
    # outputs in pinned host memory, one D and one row block per graph (a latency-sensitive client's
    # buffers: the 64 MB D of a 4096-node graph copies from the device in about a millisecond instead
    # of the several a pageable buffer takes); requests for one graph run one after another
    pinned = os.environ.get("RD_BENCH_PAGEABLE_OUTPUTS", "0") != "1"
    outD, outY = [], []
    for A, _ in pool:
        n = A.shape[0]
        if pinned:
            outD.append(torch.empty((n, n), dtype=torch.int32).pin_memory().numpy())
            outY.append(torch.empty((64, n), dtype=torch.float64).pin_memory().numpy())
        else:
            outD.append(np.empty((n, n), np.int32))
            outY.append(np.empty((64, n)))
    # warm-up: factor every graph once (what a server holds after its first minutes), untimed
    for gid, (A, g) in enumerate(pool):
        srv.wait(srv.submit_goals(gid, A, g, np.array([0], np.int32), outY[gid][:1]))
    th = threading.Thread(target=waiter, daemon=True)
    th.start()
    s0 = srv.stats()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    t0 = time.perf_counter()
    for (ta, gid, goals) in plan:
        delay = t0 + ta - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        A, g = pool[gid]
        n = A.shape[0]
        if goals is None:
            rid = srv.submit_apsp(gid, A, g, outD[gid])
        else:
            rid = srv.submit_goals(gid, A, g, goals, outY[gid][:goals.size])
        done_q.put(rid)
    done_q.put(None)
    th.join()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    s1 = srv.stats()
    srv.close()
    n_req = len(plan)
    line = {
        "metric": serve_metric(args.serve_rate), "value": n_req / wall, "unit": "solves/s", "n_gpus": 1, "steps": n_req,
        "warmup": len(pool), "ms_per_step": wall * 1e3 / max(1, n_req), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16-digits+f64", "data": "synthetic",
        "config": {"workload": f"Poisson {args.serve_rate:.0f} req/s for {args.serve_seconds:.0f} s over 128 graphs, "
                               f"n log-uniform [64, 4096] (ER p=4/n, grid, WS k=10), gain 0.5/(Delta+1); "
                               f"25% APSP, 75% goal rows (k ~ U[1,64]); split precision, 8 workers, 128 GB budget; "
                               f"outputs in {'pinned' if pinned else 'pageable'} host buffers, one per graph",
                   "requests": n_req, "parallelism": "one GPU, 8 streams"},
        "p50_ms": pct([lat for _, lat in statuses], 0.5), "p99_ms": pct([lat for _, lat in statuses], 0.99),
        "latency_note": "submit-to-completion, measured by the library, over the stream's requests",
        "requests_ok": int(sum(1 for st, _ in statuses if st == rd.RD_OK)),
        "max_inflight": s1["max_inflight"], "evictions": s1["evictions"] - s0["evictions"],
        "device_loop_requests": s1["loop_requests"] - s0["loop_requests"],
        "device_loop": "goal requests on graphs of at most %s nodes on the device-resident loop" %
                       os.environ.get("RD_SERVE_LOOP_MAX_N", "1024"),
        "resident_graphs": s1["resident_graphs"], "clocks": clk,
        "e2e": {"value": n_req / wall, "unit": "solves/s", "h2d_bytes_per_step": None, "d2h_bytes_per_step": None},
        "gpu_launches": s1["launches"] - s0["launches"],
        "roofline": {"bound": "latency", "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None,
                     "note": "requests are small (n log-uniform in [64, 4096]; 75 % are 1..64 goal rows on resident "
                             "factors) and their latency is host synchronisation and launch bound; the kernels' "
                             "rooflines are those of the single-graph and batched lines"},
        "cpu_baseline": serve_cpu_baseline(pool, plan),
    }
    print(json.dumps(line), flush=True)


WEIGHTED_METRIC = ("weighted local navigation, n=32768 king-move grid W~U[1,4]: split inverse + 1024 goal rows "
                   "+ greedy next hop, wall s")


def run_weighted(args):
    """Weighted local navigation: factor M = I - gamma^W of a king-move grid in split precision
    (the range screen measures weighted spreads and picks the node order and the digits), 1024 goal rows in
    16 batches of 64, the greedy next hop toward each goal; on the host, Dijkstra on the reversed
    graph (scipy) scores every greedy move: correct when it lies on a shortest path."""
    import scipy.sparse as sp
    import torch
    from scipy.sparse.csgraph import dijkstra

    from paper_2308_07403_gb300 import build, graphs, rd

    if int(os.environ.get("WORLD_SIZE", "1")) > 1 and int(os.environ.get("RANK", "0")) != 0:
        return
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    rd.load()
    A, W, g = graphs.workload_weighted(args.weighted_rows, args.weighted_cols, frac=args.weighted_frac)
    n = A.shape[0]
    rng = np.random.default_rng(graphs.seed_for(4, 1))
    G = 1024
    goals = np.sort(rng.choice(n, size=G, replace=False)).astype(np.int32)
    A_dev = torch.from_numpy(A).to(dev)
    W_dev = torch.from_numpy(W).to(dev)
    goals_dev = torch.from_numpy(goals).to(dev)
    rows = torch.empty((G, n), dtype=torch.float64, device=dev)
    nxt = torch.empty((G, n), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    h = rd.rd_create_weighted(A_dev, W_dev, n, g)
    del A_dev, W_dev
    rd.rd_set_stream(h, stream.cuda_stream)
    rd.rd_set_precision(h, rd.RD_PREC_SPLIT_BF16, 0)
    rd.rd_set_profiling(h, True)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(stream)
    for b in range(G // 64):
        rd.rd_goal_solve(h, goals_dev[b * 64:(b + 1) * 64], 64, rows[b * 64:(b + 1) * 64])
        if b == 0:
            ev[1].record(stream)
    for b in range(G // 64):
        rd.rd_greedy_next(h, goals_dev[b * 64:(b + 1) * 64], 64, rows[b * 64:(b + 1) * 64],
                          nxt[b * 64:(b + 1) * 64])
    ev[2].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    st = rd.rd_get_stats(h)
    t_first = ev[0].elapsed_time(ev[1])
    t_total = ev[0].elapsed_time(ev[2])
    rd.rd_destroy(h)
    # host check: distances to each goal by Dijkstra on the reversed graph
    ii, jj = np.nonzero(A)  # edge jj -> ii with weight W[ii, jj]
    w = W[ii, jj].astype(np.float64)
    rev = sp.csr_matrix((w, (ii, jj)), shape=(n, n))  # rev[i, j]: the edge j -> i, walked from i
    t0 = time.perf_counter()
    dist = dijkstra(rev, directed=True, indices=goals)  # dist[c, v] = shortest v -> goals[c]
    t_dij = time.perf_counter() - t0
    nx = nxt.cpu().numpy()
    Yh = rows.cpu().numpy()
    wmat = sp.csr_matrix((w, (jj, ii)), shape=(n, n))  # wmat[i, j] = weight of i -> j
    ok = checked = 0
    for c in range(G):
        gg = goals[c]
        i = np.nonzero((np.arange(n) != gg) & np.isfinite(dist[c]) & (nx[c] >= 0))[0]
        j = nx[c][i]
        wij = np.asarray(wmat[i, j]).ravel()
        good = wij + dist[c][j] <= dist[c][i] * (1 + 1e-12)
        ok += int(good.sum())
        checked += int(i.size)
    underflow = int(((Yh == 0) & np.isfinite(dist)).sum())
    # end to end through the C ABI: the graph from pinned host memory (rd_create_weighted copies A
    # and W in and builds M), goal rows and next hops back to pinned host memory, wall time
    A_pin = torch.from_numpy(A).pin_memory()
    W_pin = torch.from_numpy(W).pin_memory()
    rows_h = torch.empty((G, n), dtype=torch.float64).pin_memory()
    nxt_h = torch.empty((G, n), dtype=torch.int32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2 = rd.rd_create_weighted(A_pin.numpy(), W_pin.numpy(), n, g)
    rd.rd_set_stream(h2, stream.cuda_stream)
    rd.rd_set_precision(h2, rd.RD_PREC_SPLIT_BF16, 0)
    rh, nh = rows_h.numpy(), nxt_h.numpy()
    for b in range(G // 64):
        gb = np.ascontiguousarray(goals[b * 64:(b + 1) * 64])
        rd.rd_goal_solve(h2, gb, 64, rh[b * 64:(b + 1) * 64])
        rd.rd_greedy_next(h2, gb, 64, rh[b * 64:(b + 1) * 64], nh[b * 64:(b + 1) * 64])
    t_e2e = time.perf_counter() - t0
    rd.rd_destroy(h2)
    e2e_same = bool(np.array_equal(nh, nx))
    del A_pin, W_pin
    # roofline of the dense contraction that carried the factorisation
    if st["precision_used"]:
        pk, pk_kind = peaks()
        ms, fl, nl = st["prof_split_ms"], st["prof_split_flops"], st["prof_split_launches"]
        peak = pk["bf16_tflops_sustained"]
        roof = {"kernel": "split_gemm_kernel", "bound": "tensor",
                "peak_source": f"{pk_kind} bf16 sustained (cuBLAS, seconds-long loop)",
                "work": "issued BF16 digit products, s(s+1)/2 x 2MNK per split product"}
    else:  # the FP64 GEMM alone (a split attempt the self-check rejected is counted apart)
        ms = st["prof_ms"] - st["prof_split_ms"]
        fl = st["prof_flops"] - st["prof_split_flops"]
        nl = st["prof_launches"] - st["prof_split_launches"]
        sm_mhz = clk.get("sm_mhz") or 2070.0
        peak = 152 * 2 * 2 * sm_mhz * 1e6 / 1e12
        roof = {"kernel": "gemm_f64_kernel", "bound": "alu",
                "peak_source": f"FP64 pipe: 152 SMs x 4 flop/clk x {sm_mhz:.0f} MHz (unit counts)"}
    achieved = fl / (ms * 1e-3) / 1e12 if ms > 0 else None
    roof.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                 "frac": (achieved / peak) if achieved else None, "traffic": None, "launches": nl,
                 "kernel_ms": ms, "kernel_share_of_step": ms / t_total if t_total else None})
    # CPU oracle on a small king grid of the same recipe, scaled to n by n^3
    import oracle

    oracle.build()
    As, Ws, gs = graphs.workload_weighted(24, 32)
    t0 = time.perf_counter()
    oracle.rdistance(As, gs, W=Ws)
    tcpu = (time.perf_counter() - t0) * (n / As.shape[0]) ** 3
    line = {
        "metric": WEIGHTED_METRIC, "value": t_total / 1e3, "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": t_total, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16-digits+f64", "data": "synthetic",
        "config": {"workload": f"king-move grid {args.weighted_rows} x {args.weighted_cols} (n={n}), weights U[1,4] "
                               f"fp32, gain {args.weighted_frac:g} x the weighted bound = {g:.6f}; 1024 goals in 16 batches of 64",
                   "n": n, "gamma": g, "goals": G},
        "factor_and_first_goals_ms": t_first, "ms_factor": st["ms_factor"],
        "precision_used": "split" if st["precision_used"] else "fp64", "digits": st["slices"],
        "locality_order": ["none", "landmark", "scored"][st["split_order"]], "screen_bits": st["split_screen_bits"],
        "sampled_row_residual": st["split_residual"], "fallbacks": st["fallbacks"],
        "greedy_on_shortest_path_fraction": ok / max(1, checked), "greedy_moves_checked": checked,
        "goal_row_entries_underflowed": underflow, "dijkstra_cpu_s": t_dij,
        "clocks": clk, "gpu_launches": st["launches"], "roofline": roof,
        "e2e": {"value": t_e2e, "unit": "s", "h2d_bytes_per_step": int(A.nbytes + W.nbytes + goals.nbytes + rows_h.numel() * 8),
                "d2h_bytes_per_step": int(rows_h.numel() * 8 + nxt_h.numel() * 4),
                "note": "rd_create_weighted from pinned host A and W, 16 x (goal rows to host, greedy next hops "
                        "from host rows to host), wall time; next hops identical to the device run: "
                        + str(e2e_same)},
        "cpu_baseline": {"value": tcpu, "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": f"CPU oracle (1 thread, FP64, full R-distance) on the 24 x 32 king grid of the "
                                   f"same recipe, scaled to n={n} by n^3"},
    }
    print(json.dumps(line), flush=True)


UPDATE_METRIC = ("incremental edge update, n=8192 grid 90x91 at 0.9/Delta: wall ms per update "
                 "(rank-1 update of the resident Y + decode of D)")


def run_update(args):
    """Incremental edge updates (the map changing under a robot, Sec. 6): on the 90 x 91 grid at
    0.9/Delta with Y resident, `--obstacles` edge pairs (both directions of a grid edge) are removed
    one direction per update, then restored.  Each update is one rd_update_edge call into a device
    D.  Checks: after the removals D equals a fresh FP64 factorisation of the changed graph, after
    the restores D equals the original D."""
    import torch

    from paper_2308_07403_gb300 import build, graphs, rd

    if int(os.environ.get("WORLD_SIZE", "1")) > 1 and int(os.environ.get("RANK", "0")) != 0:
        return
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    rd.load()
    A, g = graphs.workload_large("grid", 0.9)
    n = A.shape[0]
    rng = np.random.default_rng(graphs.seed_for(5))
    ii, jj = np.nonzero(np.triu(A, 1))  # undirected grid edges {i, j}, i < j
    pick = rng.choice(ii.size, size=args.obstacles, replace=False)
    pairs = [(int(ii[p]), int(jj[p])) for p in pick]
    stream = torch.cuda.current_stream(dev)
    A_dev = torch.from_numpy(A).to(dev)
    D = torch.empty((n, n), dtype=torch.int32, device=dev)
    D0 = torch.empty((n, n), dtype=torch.int32, device=dev)
    h = rd.rd_create(A_dev, n, g)
    rd.rd_set_stream(h, stream.cuda_stream)
    rd.rd_set_precision(h, rd.RD_PREC_SPLIT_BF16, 0)
    rd.rd_apsp(h, D0, None)
    # warm-up: one removal and its restore (materialises the resident Y), untimed
    i0, j0 = pairs[0]
    rd.rd_update_edge(h, i0, j0, False, 1.0, D)
    rd.rd_update_edge(h, i0, j0, True, 1.0, D)
    torch.cuda.synchronize()
    rd.rd_set_profiling(h, True)
    st0 = rd.rd_get_stats(h)
    clocks = ClockSampler(local)
    clocks.start()
    dev_ms, wall_ms = [], []
    B = A.copy()

    def one(i, j, present):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        rd.rd_update_edge(h, i, j, present, 1.0, D)
        e1.record(stream)
        e1.synchronize()
        wall_ms.append((time.perf_counter() - t0) * 1e3)
        dev_ms.append(e0.elapsed_time(e1))

    for (i, j) in pairs:  # obstacles: both directions of the edge disappear
        one(i, j, False)
        one(j, i, False)
        B[i, j] = B[j, i] = 0
    torch.cuda.synchronize()
    # check the removal phase against a fresh FP64 factorisation of the changed graph
    Bd = torch.from_numpy(B).to(dev)
    Df = torch.empty((n, n), dtype=torch.int32, device=dev)
    hf = rd.rd_create(Bd, n, g)
    rd.rd_set_precision(hf, rd.RD_PREC_FP64, 0)
    rd.rd_apsp(hf, Df, None)
    torch.cuda.synchronize()
    rd.rd_destroy(hf)
    removed_mismatch = int((D != Df).sum().item())
    del Bd, Df
    for (i, j) in pairs:
        one(i, j, True)
        one(j, i, True)
    torch.cuda.synchronize()
    clk = clocks.stop()
    restored_mismatch = int((D != D0).sum().item())
    st = rd.rd_get_stats(h)
    # end to end: the same update with D read back to pinned host memory
    D_host = torch.empty((n, n), dtype=torch.int32).pin_memory()
    e2e_ms = []
    for (i, j) in pairs[:4]:
        for present in (False, True):
            t0 = time.perf_counter()
            rd.rd_update_edge(h, i, j, present, 1.0, D_host.numpy())
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    rd.rd_destroy(h)
    count = len(wall_ms)
    pk, pk_kind = peaks()
    ums, ubytes, ulaunch = st["prof_update_ms"], st["prof_update_bytes"], st["prof_update_launches"]
    achieved = ubytes / (ums * 1e-3) / 1e9 if ums > 0 else None
    roof = {"kernel": "rank1_decode_kernel", "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"],
            "unit": "GB/s", "frac": (achieved / pk["hbm_gbs"]) if achieved else None, "traffic": None,
            "peak_source": f"{pk_kind} HBM copy bandwidth",
            "work": "20 n^2 bytes per pass: read and write Y (FP64), write D (int32)",
            "launches": ulaunch, "kernel_ms_per_update": ums / max(1, ulaunch)}
    # CPU oracle: a full R-distance of a small grid of the same recipe, scaled to n by n^3
    import oracle

    oracle.build()
    As = graphs.grid4(1024, 32)
    t0 = time.perf_counter()
    oracle.rdistance(As, graphs.gamma_frac(As, 0.9))
    tcpu = (time.perf_counter() - t0) * (n / As.shape[0]) ** 3 * 1e3
    line = {
        "metric": UPDATE_METRIC, "value": float(np.mean(wall_ms)), "unit": "ms", "n_gpus": 1, "steps": count,
        "warmup": 2, "ms_per_step": float(np.mean(wall_ms)), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"grid 90 x 91 (n={n}) at 0.9/Delta, split-precision factors; {args.obstacles} "
                               f"edge pairs removed one direction per update, then restored", "n": n, "gamma": g,
                   "updates": count, "l2": "no flush: Y (512 MiB) and D (256 MiB) exceed the 129 MB L2"},
        "device_ms_per_update_p50": pct(dev_ms, 0.5), "wall_ms_per_update_p50": pct(wall_ms, 0.5),
        "wall_ms_per_update_p99": pct(wall_ms, 0.99),
        "updates_per_s": count / (sum(wall_ms) * 1e-3),
        "refactors": st["update_refactors"] - st0["update_refactors"],
        "D_mismatch_after_removals_vs_fresh_fp64": removed_mismatch,
        "D_mismatch_after_restores_vs_original": restored_mismatch,
        "e2e": {"value": float(np.mean(e2e_ms)), "unit": "ms", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 4 * n * n, "note": "the update with D read back to pinned host memory"},
        "clocks": clk, "gpu_launches": st["launches"] - st0["launches"], "roofline": roof,
        "cpu_baseline": {"value": tcpu, "unit": "ms", "cores": 1, "kind": "oracle",
                         "sample": "CPU oracle (1 thread, FP64): full R-distance of the 32 x 32 grid at 0.9/Delta, "
                                   f"scaled to n={n} by n^3 (what a CPU recompute of the changed map costs)"},
    }
    print(json.dumps(line), flush=True)


PRODUCT_METRIC = "split inverse product Y = U^-1 L^-1 with the fused decode, issued digit-product TFLOP/s"


def run_product(args):
    """The largest split launch alone: the factors of an ER graph (p = 0.01, 0.5/Delta; or a 4-neighbour
    grid, which runs in the locality order with 64-wide chunks) are made once,
    then rd_apsp re-runs only the inverse product with the fused decode (the factors stay
    resident).  The timed launches run inside the NVTX range "inverse_product", so that an ncu
    capture can select exactly them (--nvtx --nvtx-include inverse_product/)."""
    import torch

    from paper_2308_07403_gb300 import build, graphs, rd

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.split_stats:
        rd.load(build.build(stats=True))
    else:
        build.build()
        rd.load()
    n = args.product_n
    if args.product_graph == "grid":
        cols = int(round(n ** 0.5))
        A = graphs.grid4(n, cols)
    else:
        A = graphs.er(n, 0.01, graphs.seed_for(1))
    g = graphs.gamma_frac(A, 0.5)
    stream = torch.cuda.current_stream(dev)
    A_dev = torch.from_numpy(A).to(dev)
    D = torch.empty((n, n), dtype=torch.int32, device=dev)
    h = rd.rd_create(A_dev, n, g)
    rd.rd_set_stream(h, stream.cuda_stream)
    rd.rd_set_precision(h, rd.RD_PREC_SPLIT_BF16, 0)
    rd.rd_apsp(h, D, None)  # factors, self-check, first product
    for _ in range(max(3, args.warmup)):
        rd.rd_apsp(h, D, None)
    torch.cuda.synchronize()
    rd.rd_set_profiling(h, True)
    if args.split_stats:
        rd.rd_split_stats(reset=True)
    st0 = rd.rd_get_stats(h)
    clocks = ClockSampler(local)
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.nvtx.range_push("inverse_product")
    ev[0].record(stream)
    for _ in range(args.steps):
        rd.rd_apsp(h, D, None)
    ev[1].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clk = clocks.stop()
    split_stats = None
    if args.split_stats:
        c = rd.rd_split_stats()
        nm, ne = max(c["mma_warps"], 1), max(c["epilogue_warps"], 1)
        kc = lambda v, w: round(v / w / 1e3, 1)  # thousands of cycles per warp (a tile's CTA or pair)
        split_stats = {
            "unit": "thousand SM cycles per tile (per MMA warp; epilogue per CTA)",
            "mma": {"total": kc(c["mma_cycles"], nm), "wait_accumulator": kc(c["mma_wait_accumulator"], nm),
                    "wait_operands": kc(c["mma_wait_operands"], nm), "issue": kc(c["mma_issue"], nm),
                    "tensor_busy_at_64_cycles_per_mma": kc(64 * c["mmas"], nm)},
            "producer": {"total": kc(c["producer_cycles"], nm), "wait_stage": kc(c["producer_wait_stage"], nm)},
            "epilogue": {"total": kc(c["epilogue_cycles"], ne), "wait_group": kc(c["epilogue_wait_group"], ne),
                         "renormalise": kc(c["epilogue_renormalise"], ne)},
            "groups_per_tile": round(c["groups"] / nm, 1), "mmas_per_tile": round(c["mmas"] / nm, 1),
            "tiles": c["mma_warps"] // args.steps}
    st = rd.rd_get_stats(h)
    rd.rd_destroy(h)
    import oracle

    oracle.build()
    m = 1024
    As = A[:m, :m]
    t0 = time.perf_counter()
    oracle.rdistance(As, graphs.gamma_frac(As, 0.5))
    tcpu = time.perf_counter() - t0
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    kms = (st["prof_split_ms"] - st0["prof_split_ms"]) / args.steps
    fl = (st["prof_split_flops"] - st0["prof_split_flops"]) / args.steps
    pk, pk_kind = peaks()
    achieved = fl / (kms * 1e-3) / 1e12
    line = {
        "metric": PRODUCT_METRIC, "value": achieved, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16-digits", "data": "synthetic",
        "config": {"workload": (f"ER n={n} p=0.01" if args.product_graph == "er" else f"4-neighbour grid n={n}")
                               + " at 0.5/Delta, split factors resident; Y = U^-1 L^-1 + decode",
                   "n": n, "digits": st["slices"], "locality_order": ["none", "landmark", "scored"][st["split_order"]],
                   "l2": "no flush: the digit planes of both operands exceed the 129 MB L2"},
        "kernel_ms": kms, "effective_tflops_2n3_over_3": (2.0 * n ** 3 / 3.0) / (ms * 1e-3) / 1e12,
        "clocks": clk, "gpu_launches": (st["launches"] - st0["launches"]) // max(1, args.steps),
        "e2e": {"value": None, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                "note": "kernel diagnostic on resident factors; the end-to-end figure is the single-graph line's"},
        "cpu_baseline": {"value": (2.0 * m ** 3 / 3.0) / tcpu / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                         "sample": f"the oracle's whole R-distance of the leading {m} x {m} principal submatrix, "
                                   "rated at the product's 2 m^3 / 3 (the oracle has no separate product step)"},
        "roofline": {"kernel": "split_gemm_kernel", "bound": "tensor", "achieved": achieved,
                     "peak": pk["bf16_tflops"], "unit": "TFLOP/s", "frac": achieved / pk["bf16_tflops"],
                     # DRAM bytes of this launch (read + write) from an ncu capture of this
                     # kernel build on this graph; stale once either changes
                     "traffic": (PRODUCT_TRAFFIC if (args.product_graph == "er" and n == 4096 and st["slices"] == 9
                                                     and not args.split_stats) else None),
                     "traffic_unit": "B", "peak_source": f"{pk_kind} bf16 burst (cuBLAS)",
                     "work": "issued BF16 digit products, s(s+1)/2 x 2MNK"},
    }
    if split_stats is not None:
        line["split_stats"] = split_stats
        line["config"]["build"] = "diagnostic build with the split GEMM's cycle counters (RD_SPLIT_STATS)"
    print(json.dumps(line), flush=True)


def run_mma_probe(args):
    """The tensor-core rate of the split path's BF16 digit products with nothing else in the loop
    (rd_probe_mma): one CTA per SM issuing 128 x 128 x 16 MMAs from shared memory back to back,
    against the measured cuBLAS BF16 peak; the INT8 kind is reported as unavailable on sm_103a."""
    import torch

    from paper_2308_07403_gb300 import build, rd

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build.build()
    rd.load()
    rd.rd_probe_mma(0, 200)  # warm-up (clocks up, module loaded)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    res = {}
    runs = [rd.rd_probe_mma(0, 8000) for _ in range(max(1, args.steps))]
    res["bf16"] = {"tera_ops_per_s": max(r for r, _ in runs), "seconds": min(s for _, s in runs)}
    try:
        rd.rd_probe_mma(1, 1)
        int8 = "measured"
    except rd.RDError as ex:
        int8 = str(ex)
    clk = clocks.stop()
    pk, pk_kind = peaks()
    line = {
        "metric": "tcgen05 BF16 MMA rate (128 x 128 x 16, operands in shared memory, every SM)",
        "value": res["bf16"]["tera_ops_per_s"], "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": 1,
        "ms_per_step": res["bf16"]["seconds"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic (zero operands)",
        "config": {"workload": "152 CTAs x 8000 x 64 MMAs of 128 x 128 x 16, one thread issuing per SM, "
                               "a commit and a bounded wait per 64"},
        "int8": int8,
        "bf16_of_measured_cublas_burst": res["bf16"]["tera_ops_per_s"] / pk["bf16_tflops"], "peak_source": pk_kind,
        "clocks": clk, "gpu_launches": 1 + max(1, args.steps),
        "roofline": {"kernel": "probe_mma_kernel", "bound": "tensor", "achieved": res["bf16"]["tera_ops_per_s"],
                     "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                     "frac": res["bf16"]["tera_ops_per_s"] / pk["bf16_tflops"], "traffic": None},
        "e2e": None, "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload == "mma-probe":
        run_mma_probe(args)
        return
    if args.workload == "product":
        run_product(args)
        return
    if args.workload == "update":
        run_update(args)
        return
    if args.workload == "weighted":
        run_weighted(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "batched-stack":
        run_batched_stack(args)
        return
    if args.workload == "serving":
        run_serving(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    from paper_2308_07403_gb300 import build, rd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    rd.load()

    n = args.n
    wl = workloads(n)
    stream = torch.cuda.current_stream(dev)
    A_dev = [torch.from_numpy(A).to(dev) for (_, _, A, _) in wl[::2]]  # one matrix per kind
    rng = np.random.default_rng(7)
    goals = np.sort(rng.choice(n, size=args.goals, replace=False)).astype(np.int32)
    goals_dev = torch.from_numpy(goals).to(dev)
    D = torch.empty((n, n), dtype=torch.int32, device=dev)
    rows = torch.empty((args.goals, n), dtype=torch.float64, device=dev)
    nxt = torch.empty((args.goals, n), dtype=torch.int32, device=dev)

    h = rd.rd_create(A_dev[0], n, wl[0][3])
    rd.rd_set_stream(h, stream.cuda_stream)
    modes = {"split": rd.RD_PREC_SPLIT_BF16, "fp64": rd.RD_PREC_FP64}

    def step(i):
        kind, frac, _, g = wl[i % len(wl)]
        rd.rd_load(h, A_dev[(i % len(wl)) // 2], None, g)
        rd.rd_apsp(h, D)
        rd.rd_goal_solve(h, goals_dev, args.goals, rows)
        rd.rd_greedy_next(h, goals_dev, args.goals, rows, nxt)

    # ---- the headline path
    rd.rd_set_precision(h, modes[args.precision], args.slices)
    per_step, total_ms, st0, st1, clk = time_path(rd, h, step, 0, args.steps, args.warmup, stream, local, world, dist,
                                                  profile=2 if args.precision == "split" else True)
    ms_step = total_ms / args.steps
    flop_step = 2.0 * n ** 3
    # device ms of each graph's steps (step i runs graph i mod 6), median per graph
    by_graph = {}
    for i, ms in enumerate(per_step):
        kind, frac, _, _ = wl[(args.warmup + i) % len(wl)]
        by_graph.setdefault(f"{kind}_{frac}", []).append(ms)
    ms_per_graph = {k: round(pct(v, 0.5), 3) for k, v in by_graph.items()}
    value = replica_throughput(world, flop_step, args.steps, total_ms)
    launches = st1["launches"] - st0["launches"]
    pk, pk_kind = peaks()
    if args.precision == "fp64":
        prof_ms, prof_fl, prof_n = st1["prof_ms"], st1["prof_flops"], st1["prof_launches"]
    else:  # the split GEMM's own launches (a step the screen sends to FP64 runs the FP64 GEMM); its
        # time is the union of its launches' intervals: launches on the recursion's two streams overlap,
        # and their summed durations (prof_split_ms) count the shared time twice
        prof_ms, prof_fl, prof_n = st1["prof_split_busy_ms"], st1["prof_split_flops"], st1["prof_split_launches"]
    achieved = prof_fl / (prof_ms * 1e-3) / 1e12 if prof_ms > 0 else None
    if args.precision == "fp64":
        # FP64 SIMT GEMM, bound by the FP64 pipe: peak from unit counts and the sampled clock
        # (152 SMs x 2 DFMA/clk x 2 flops); a DFMA probe measured 1.19 TFLOP/s at 2.07 GHz
        sm_mhz = clk.get("sm_mhz") or 2070.0
        peak = 152 * 2 * 2 * sm_mhz * 1e6 / 1e12
        roof = {"kernel": "gemm_f64_kernel", "bound": "alu", "peak_source":
                f"FP64 pipe: 152 SMs x 4 flop/clk x {sm_mhz:.0f} MHz (unit counts)"}
    else:
        # the split GEMM's algorithmic work is its digit products: s(s+1)/2 x 2 M N K per product
        peak = pk["bf16_tflops_sustained"]
        roof = {"kernel": "split_gemm_kernel", "bound": "tensor",
                "peak_source": f"{pk_kind} bf16 sustained (cuBLAS, seconds-long loop)",
                "work": "issued BF16 digit products, s(s+1)/2 x 2MNK per split product"}
    split_line = args.precision == "split" and n == 8192 and args.slices == 0
    roof.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                 "frac": (achieved / peak) if achieved else None,
                 "traffic": SPLIT_TRAFFIC_PER_LAUNCH if split_line else None,
                 "traffic_algorithmic": SPLIT_ALGORITHMIC_BYTES_PER_LAUNCH if split_line else None,
                 "traffic_unit": "B per launch",
                 "launches": prof_n, "kernel_ms": prof_ms,
                 "kernel_ms_launch_sum": st1["prof_split_ms"] if args.precision != "fp64" else prof_ms,
                 "kernel_share_of_step": prof_ms / total_ms if total_ms else None})
    slices_used = st1["slices"]

    # ---- end-to-end through the C ABI with host buffers (right after the timed steps, in the same
    # state of the GPU; the seconds-long FP64 comparison below heats it)
    e2e = None
    if args.e2e_steps > 0:
        A_host = [torch.from_numpy(A).pin_memory() for (_, _, A, _) in wl[::2]]
        D_host = torch.empty((n, n), dtype=torch.int32).pin_memory()
        rows_host = torch.empty((args.goals, n), dtype=torch.float64).pin_memory()
        nxt_host = torch.empty((args.goals, n), dtype=torch.int32).pin_memory()
        goals_host = torch.from_numpy(goals)

        def step_host(i):
            kind, frac, _, g = wl[i % len(wl)]
            rd.rd_load(h, A_host[(i % len(wl)) // 2], None, g)
            rd.rd_apsp(h, D_host)
            rd.rd_goal_solve(h, goals_host, args.goals, rows_host)
            rd.rd_greedy_next(h, goals_host, args.goals, rows_host, nxt_host)

        step_host(0)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for i in range(args.e2e_steps):
            step_host(1 + i)
        torch.cuda.synchronize()
        te = reduce_max(time.perf_counter() - t0, dist, world, dev)
        e2e = {"value": replica_throughput(world, flop_step, args.e2e_steps, te * 1e3), "unit": "TFLOP/s",
               "ms_per_step": te * 1e3 / args.e2e_steps,
               "h2d_bytes_per_step": n * n + 4 * args.goals * 2 + 8 * args.goals * n,
               "d2h_bytes_per_step": 4 * n * n + 8 * args.goals * n + 4 * args.goals * n}

    # ---- the comparison path (the other precision), fewer steps
    compare = None
    other = "fp64" if args.precision == "split" else "split"
    if args.compare_steps > 0:
        rd.rd_set_precision(h, modes[other], 0)
        cps, ctot, _, _, _ = time_path(rd, h, step, 100, args.compare_steps, 1, stream, local, world, dist,
                                       profile=False)
        compare = {"precision": other, "ms_per_step": ctot / args.compare_steps,
                   "p50_ms": pct(cps, 0.5), "p99_ms": pct(cps, 0.99),
                   "value": replica_throughput(world, flop_step, args.compare_steps, ctot), "unit": "TFLOP/s",
                   "steps": args.compare_steps, "warmup": 1}
        compare["speedup_of_headline"] = compare["ms_per_step"] / ms_step
        rd.rd_set_precision(h, modes[args.precision], args.slices)

    # ---- every graph in both precisions: D against the oracle's stored hash (tests/golden, written by
    # the oracle), the split path's Y against the FP64 path's Y, D against BFS truth (scipy, sampled
    # source columns)
    verify = None
    if args.verify and n == 8192:
        verify = verify_graphs(rd, h, wl, A_dev, modes, args, other if compare else None, D, dev)
    rd.rd_destroy(h)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = cpu_baseline(args, wl[0][2]) if world == 1 else None
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "bf16-digits+f64",
        "data": "synthetic",
        "config": {"workload": f"n={n} single graphs: ER p=0.01, grid 90x91 (+2), WS k=10 beta=0.1, "
                               f"gain 0.5 and 0.9 x 1/Delta; one graph per step, {args.goals} goals",
                   "n": n, "precision": args.precision, "slices_requested": args.slices,
                   "slices_last_graph": slices_used, "goals": args.goals,
                   "l2": "no flush: working set (M, LU, inverses) 1.3 GB > 129 MB L2",
                   "parallelism": f"replicas x{world}"},
        "p50_ms": pct(per_step, 0.5), "p99_ms": pct(per_step, 0.99), "ms_per_graph": ms_per_graph,
        "clocks": clk, "e2e": e2e, "gpu_launches": launches, "roofline": roof,
        "cpu_baseline": cpu, "compare": compare, "verify": verify,
    }
    if args.precision == "split":
        line["steps_redone_in_fp64_by_self_check"] = st1["fallbacks"] - st0["fallbacks"]
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
