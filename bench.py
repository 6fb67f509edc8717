#!/usr/bin/env python
"""Benchmark of the worklist ForAll hot path (BFS / SSSP / CC) on one GB300.

Default workload (N=1): R-MAT scale 20, edge factor 16, (a,b,c) = (.57,.19,.19),
weights [1,100]. One step = one BFS query and one SSSP query from the next seeded
source (out-degree > 0), each a single persistent cooperative launch
(iteration outlining). The graph is resident in HBM before timing starts.

Reported (one JSON line on rank 0):
  value       GTEPS = directed edges out of reached vertices / kernel time,
              summed over BFS and SSSP (CUDA events on the launching stream;
              L2 flushed between steps by writing a 512 MB buffer, outside the events)
  e2e         the same metric through the C-ABI with host buffers: sources
              copied in and the uint32 result copied out inside the timed call
  roofline    algorithmic bytes of the dominant kernel per launch / its mean
              event-timed duration, against the measured HBM copy bandwidth
  cpu_baseline  the CPU oracle (serial BFS + Dijkstra) on a bounded sample
Other workloads: --workload grid64 | rmat20 | mesh (configuration sizes).
--impl reference times the CPU oracle itself on the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "BFS/SSSP GTEPS + HBM roofline %; batched vs per-launch GTEPS; query p50/p99"
INF = 0xFFFFFFFF


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 16; grid64: 1000, the median of 1000 repetitions)")
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=["rmat20", "grid64", "mesh", "batch256", "serve", "msf"], default="rmat20")
    ap.add_argument("--msf-graph", choices=["mesh", "rmat"], default="mesh",
                    help="msf: the weighted 4096^2 mesh or a symmetrised R-MAT scale-20 graph")
    ap.add_argument("--msf-lock", choices=["blocking", "ticket", "retry"], default="retry",
                    help="msf: lock form (retry measured fastest on the 4096^2 mesh: 25.8 ms against 39.8 blocking)")
    ap.add_argument("--instances", type=int, default=256, help="batch256: number of instances")
    ap.add_argument("--batch-set", choices=["rmat", "grids"], default="rmat",
                    help="batch256: the R-MAT SSSP instances, or 32 serving-like queries on 16 weighted grids "
                         "(side U[256,1024], 70%% BFS / 30%% SSSP)")
    ap.add_argument("--wave-mb", type=int, default=None,
                    help="batch256: packed-state MB per wave (-1: every instance in one wave; default: one wave, "
                         "or what the autotuner picks)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batch256: skip irgl_batch_autotune (degree thresholds, CTA size, chunk, waves) before timing")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: Poisson arrival rate (queries/s)")
    ap.add_argument("--duration", type=float, default=60.0, help="serve: arrival window (s)")
    ap.add_argument("--serve-scale", type=int, default=24, help="serve: R-MAT scale of the large graph")
    ap.add_argument("--slots", type=int, default=512,
                    help="serve: concurrent query slots (with near-far, 512 measured best: 64 -> 15.6, 256 -> 23.4, 512 -> 23.7 GTEPS)")
    ap.add_argument("--epoch-rounds", type=int, default=32, help="serve: rounds per epoch")
    ap.add_argument("--arena-gb", type=float, default=0.0, help="serve: device arena budget (0: 40% of free HBM)")
    ap.add_argument("--verify", type=int, default=32, help="serve: queries checked against the oracle")
    ap.add_argument("--per-launch-sample", type=int, default=160,
                    help="serve: served queries rerun one persistent launch each for the per-launch comparison")
    ap.add_argument("--sub-serve-duration", type=float, default=10.0,
                    help="rmat20: arrival window (s) of the serving sub-record")
    ap.add_argument("--autotune", choices=["auto", "on", "off"], default="auto",
                    help="single-query workloads: pick each kernel's tuning with irgl_autotune before timing "
                         "(auto: on for grid64, off otherwise)")
    ap.add_argument("--no-extras", action="store_true",
                    help="rmat20: leave out the batch and serving sub-records of the default line")
    ap.add_argument("--scale", type=int, default=20, help="R-MAT scale (rmat20 workload)")
    ap.add_argument("--mesh-side", type=int, default=4096)
    ap.add_argument("--cc", choices=["label", "jump"], default="label",
                    help="mesh: CC by min-label propagation (the Iterate of the paper's CC) or pointer jumping")
    ap.add_argument("--cc-delta", type=int, default=1,
                    help="mesh, label CC: near-far width on labels (1: smallest label first; 0: plain rounds)")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--clocks-log", type=str, default=os.environ.get("IRGL_CLOCKS_LOG"),
                    help="directory that keeps the raw nvidia-smi clock samples (default: a temporary file)")
    ap.add_argument("--no-per-launch", action="store_true", help="skip the per-launch (host loop) BFS comparison")
    ap.add_argument("--tuning", type=str, default="", help="JSON irgl_tuning overrides")
    ap.add_argument("--trace", action="store_true", help="print a per-round trace of one query per kernel to stderr")
    ap.add_argument("--diropt", action="store_true",
                    help="BFS direction-optimising (bottom-up rounds on large frontiers; loads the in-edge CSR); "
                         "the default on the R-MAT workload")
    ap.add_argument("--no-diropt", action="store_true",
                    help="rmat20: time the top-down-only BFS in the headline instead")
    ap.add_argument("--local", type=int, default=-1,
                    help="CTA-local sub-rounds for persistent BFS/SSSP (0..15; default: 15 on the high-diameter "
                         "grid64 and mesh workloads, 0 on R-MAT, as the autotuner picks them)")
    args = ap.parse_args()
    if args.workload == "rmat20" and not args.no_diropt:
        args.diropt = True
    if args.steps is None:
        args.steps = 1000 if args.workload == "grid64" else 16
    return args


# ----------------------------------------------------------------------------- distributed plumbing

def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "gb300" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(items, world, rank):
    """Queries are independent: rank r takes every world-th one (no data-path collective)."""
    return items[rank::world]


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    # directory for the raw samples (kept for evidence); a temporary file when unset
    LOG_DIR: str | None = None

    def __init__(self, device_index: int, enabled: bool = True):
        self.proc = None
        self.path = None
        self.device_index = device_index
        if not enabled:
            return
        if self.LOG_DIR:
            out = Path(self.LOG_DIR)
            out.mkdir(parents=True, exist_ok=True)
            self.path = out / f"clocks_{os.getpid()}.csv"
        else:
            self.path = Path(tempfile.gettempdir()) / f"irgl_clocks_{os.getpid()}.csv"
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={device_index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in self.path.read_text().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append(dict(sm=float(f[1]), smax=float(f[2]), power=float(f[3]) if f[3] not in ("[N/A]", "") else 0.0,
                                 hw=f[5], hwt=f[6], swt=f[7], swp=f[8]))
            except ValueError:
                continue
        if not rows:
            return None
        smax = max(r["smax"] for r in rows)
        loaded = [r for r in rows if r["power"] > 150.0] or rows
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                              ("swp", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in loaded), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(rows)}


# ----------------------------------------------------------------------------- workloads

def load_workload(args):
    from paper_1607_05707_gb300 import inputs

    if args.workload == "grid64":
        g, srcs = inputs.workload_grid64()
        kernels = ("bfs",)
        name = "grid64: 64x64 4-neighbour grid BFS, source 0"
        meta = dict(V=g.n, m=g.m, sources=1)
    elif args.workload == "mesh":
        g, srcs = inputs.workload_mesh(args.mesh_side)
        cc = "cc_jump" if args.cc == "jump" else "cc"
        kernels = ("bfs", cc)
        name = (f"mesh{args.mesh_side}: {args.mesh_side}^2 mesh (1% edges deleted, 0.1% extra edges r<=8) BFS from "
                f"source 0 + CC ({'pointer jumping' if args.cc == 'jump' else 'min-label propagation'}"
                f"{f', near-far delta {args.cc_delta}' if args.cc != 'jump' and args.cc_delta else ''})")
        meta = dict(V=g.n, m=g.m, sources=1)
    else:
        g, srcs = inputs.workload_rmat20(nsrc=64, scale=args.scale)
        kernels = ("bfs", "sssp")
        name = f"rmat{args.scale}-ef16 BFS+SSSP (a,b,c)=(.57,.19,.19), w in [1,100], 64 seeded sources"
        meta = dict(V=g.n, m=g.m, scale=args.scale, edge_factor=16, sources=64)
    return g, srcs, kernels, name, meta


def reached_stats(g, result: np.ndarray):
    """|R| and m_R (directed edges out of reached vertices)."""
    deg = g.out_degree()
    reached = result != INF
    return int(reached.sum()), int(deg[reached].sum())


def alg_bytes(kernel: str, n: int, R: int, mR: int) -> int:
    """Algorithmic bytes of one query: each item counted once (no re-relaxations, no overfetch)."""
    b = 4 * n + 20 * R + 8 * mR  # init + (row_ptr pair, pop, push, state write) per reached + (col, dst state) per edge
    if kernel == "sssp":
        b += 4 * mR + 4 * R  # weights + dedup stamp
    elif kernel.startswith("cc"):
        b += 4 * R  # dedup stamp
    return b


def source_sha(files) -> str:
    """Hash of the source files a kernel is built from (in the order given)."""
    h = hashlib.sha256()
    for name in files:
        h.update((ROOT / "paper_1607_05707_gb300" / "csrc" / name).read_bytes())
    return h.hexdigest()[:16]


def measured_traffic(kernel_name: str, workload: str):
    """DRAM bytes per launch from a committed ncu capture of this kernel on this workload, only if the
    kernel's sources are unchanged since (entries are keyed "kernel@workload")."""
    p = ROOT / "profiles" / "traffic.json"
    if not p.exists():
        return None
    try:
        d = json.loads(p.read_text())
    except ValueError:
        return None
    ent = d.get(f"{kernel_name}@{workload}")
    if not ent or not ent.get("sources"):
        return None
    try:
        if ent.get("source_sha") != source_sha(ent["sources"]):
            return None
    except OSError:
        return None
    return ent.get("bytes_per_launch")


def peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------- CPU oracle timing

def host_cpu() -> str:
    """The host CPU's model, for the CPU baseline lines (first 'model name' / 'Model name' found)."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


def cpu_oracle_sample(g, srcs, kernels, budget_s: float):
    import oracle

    t_total, edges, done = 0.0, 0, []
    for s in srcs:
        for k in kernels:
            t0 = time.perf_counter()
            res = oracle.run("cc" if k.startswith("cc") else k, g, None if k.startswith("cc") else np.array([s], np.uint32))
            dt = time.perf_counter() - t0
            t_total += dt
            edges += reached_stats(g, res)[1]
            done.append(k)
        if t_total >= budget_s:
            break
    nq = len(done)
    return {"value": edges / t_total / 1e9 if t_total > 0 else 0.0, "unit": "GTEPS", "cores": 1, "kind": "oracle", "cpu": host_cpu(),
            "sample": f"{nq} queries ({'+'.join(kernels)} from {nq // len(kernels)} of the workload's sources), "
                      f"{t_total:.1f} s serial on {platform.machine()} host ({os.cpu_count()} cores present, 1 used)"}


# ----------------------------------------------------------------------------- reference arm (the oracle)

def run_reference(args, world, rank):
    if rank != 0:
        return
    if args.workload == "msf":
        return run_reference_msf(args)
    g, srcs, kernels, name, meta = load_workload(args)
    import oracle

    def step(i):
        s = np.array([srcs[i % len(srcs)]], np.uint32)
        e = 0
        t0 = time.perf_counter()
        for k in kernels:
            e += reached_stats(g, oracle.run("cc" if k.startswith("cc") else k, g, None if k.startswith("cc") else s))[1]
        return time.perf_counter() - t0, e

    for i in range(args.warmup):
        step(i)
    t_sum, e_sum = 0.0, 0
    for i in range(args.steps):
        dt, e = step(args.warmup + i)
        t_sum += dt
        e_sum += e
    value = e_sum / t_sum / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_sum / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": dict(workload=name, **meta, parallelism="rank 0 only (serial CPU oracle)"),
        "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle", "cpu": host_cpu(),
                         "sample": f"each step = {'+'.join(kernels)} from one source, serial"},
        "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_msf(args):
    import oracle

    g, name = msf_graph(args)
    oracle.msf(g.n, g.row_ptr, g.col, g.w)  # one warm-up run: a step is a whole Kruskal run
    t_sum = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.msf(g.n, g.row_ptr, g.col, g.w)
        t_sum += time.perf_counter() - t0
    value = args.steps * g.m / t_sum / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "G input edges/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": 1, "ms_per_step": 1e3 * t_sum / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": name, "V": g.n, "m": g.m, "parallelism": "rank 0 only (serial CPU oracle)"},
        "cpu_baseline": {"value": value, "unit": "G input edges/s", "cores": 1, "kind": "oracle", "cpu": host_cpu(),
                         "sample": "each step = one Kruskal run on the whole graph, serial"},
        "e2e": {"value": value, "unit": "G input edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm

def run_gpu(args, world, rank, local):
    import torch

    from paper_1607_05707_gb300 import irgl as C
    from paper_1607_05707_gb300.api import Context, as_u32

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    g, srcs_all, kernels, name, meta = load_workload(args)
    srcs = shard(list(srcs_all), world, rank)
    tuning = json.loads(args.tuning) if args.tuning else None
    if tuning is None and args.workload == "rmat20" and args.autotune != "on":
        # CTAs of 256 on R-MAT: 3 % faster than the library default of 128 for both kernels
        # (116.5 / 432.7 against 119.7 / 445.5 us); irgl_autotune lands on the same size
        tuning = {"cta_size": 256}

    stream = torch.cuda.Stream(device=dev)
    ctx = Context(local, stream)
    dg = ctx.load(g, validate=False, in_edges=args.diropt)
    out = {k: ctx.state(g.n) for k in kernels}
    ktune = {}
    local_k = args.local if args.local >= 0 else (15 if args.workload in ("grid64", "mesh") else 0)
    if args.diropt:
        local_k = 0  # bottom-up rounds and CTA-local sub-rounds exclude each other
    for k in kernels:
        t = dict(tuning or {})
        if args.diropt and k == "bfs":
            t["flags"] = int(t.get("flags", 0)) | 2
        if local_k and k in ("bfs", "sssp") and not (int(t.get("flags", 0)) >> 8) & 15:
            t["flags"] = int(t.get("flags", 0)) | ((local_k & 15) << 8)
        if k == "cc" and args.cc_delta and "delta" not in t:
            t["delta"] = args.cc_delta
        ktune[k] = t or None
    autotuned = {}
    if args.autotune == "on" or (args.autotune == "auto" and args.workload == "grid64" and not tuning):
        # the search runs before the timed region; its choice is recorded in the line's config
        for k in kernels:
            t0 = time.perf_counter()
            best, ms = ctx.autotune(k, dg, None if k.startswith("cc") else [int(srcs[0])], reps=5)
            ktune[k] = best
            autotuned[k] = {"search_s": round(time.perf_counter() - t0, 1), "median_ms": round(ms, 4)}
    wls = []
    for s in srcs:
        wl = ctx.worklist(4)
        wl.push([s])
        wls.append(wl)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    torch.cuda.synchronize(dev)

    def init(k, j):
        return None if k.startswith("cc") else wls[j]  # CC: Iterate over every vertex

    def launch_step(j):
        """One step: BFS (and SSSP) from source j, each one persistent launch, bracketed by events."""
        with torch.cuda.stream(stream):
            flush.fill_(j)  # L2 flush (> 129 MB), outside the events
        ev = {}
        for k in kernels:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.iterate_async(k, dg, init(k, j), out[k], tuning=ktune[k])
            e1.record(stream)
            ev[k] = (e0, e1)
        ctx.sync()
        return ev

    used = [(args.warmup + i) % len(wls) for i in range(args.steps)]
    for i in range(args.warmup):
        launch_step(i % len(wls))
    # reached-vertex and edge counts per (source, kernel), taken from the results outside the timed region;
    # edges scanned (re-relaxations included) from the device counters, one query at a time
    counts, scanned, rounds = {}, {k: 0 for k in kernels}, {}
    for j in sorted(set(used)):
        for k in kernels:
            ctx.iterate_async(k, dg, init(k, j), out[k], tuning=ktune[k])
            st = ctx.sync()
            scanned[k] += st["edges_scanned"]
            rounds[(j, k)] = st["rounds"]
            counts[(j, k)] = reached_stats(g, as_u32(out[k])[: g.n])
    if args.trace and rank == 0:
        C.irgl_trace_enable(ctx.handle, 1 << 16)
        for k in kernels:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.iterate_async(k, dg, init(k, used[0]), out[k], tuning=ktune[k])
            e1.record(stream)
            st = ctx.sync()
            t, a, o = C.irgl_trace_read(ctx.handle)
            ph = C.irgl_trace_phases(ctx.handle)
            print(f"# trace {k} source {srcs[used[0]]}: rounds={st['rounds']} total_us={(int(t[-1]) - int(t[0])) / 1e3:.1f}"
                  f" prologue_us={int(o[0]) / 1e3:.2f} event_us={1e3 * e0.elapsed_time(e1):.1f}", file=sys.stderr)
            print("#  (phase columns: us after the previous round's end; first/last = earliest/latest CTA)",
                  file=sys.stderr)
            mask = (1 << 64) - 1
            for r in range(1, len(t)):
                if int(a[r]) == INF and int(o[r]) == INF:
                    print(f"#  epilogue us {(int(t[r]) - int(t[r - 1])) / 1e3:9.2f}", file=sys.stderr)
                    continue
                line = f"#  round {r - 1:5d} us {(int(t[r]) - int(t[r - 1])) / 1e3:9.2f} in {int(a[r]):9d} out {int(o[r]):9d}"
                if r - 1 < len(ph) and int(ph[r - 1][1]):
                    w = [int(x) for x in ph[r - 1]]
                    t0 = int(t[r - 1])
                    if r == 1 and (~w[0] & mask) < t0:
                        t0 -= int(o[0])  # round 0 ran inside the prologue: times from the kernel's start
                    line += (f" | phase 1 first {((~w[0] & mask) - t0) / 1e3:7.2f} last {(w[1] - t0) / 1e3:7.2f}"
                             f" | barrier exit {(w[2] - t0) / 1e3:7.2f}")
                    if w[3]:
                        line += (f" | big list {w[3] >> 40:6d} lists {w[3] & ((1 << 40) - 1):9d} edges"
                                 f" first {((~w[4] & mask) - t0) / 1e3:7.2f} last {(w[5] - t0) / 1e3:7.2f}"
                                 f" barrier exit {(w[6] - t0) / 1e3:7.2f}")
                print(line, file=sys.stderr)
        C.irgl_trace_enable(ctx.handle, 0)

    rec = {k: [] for k in kernels}
    nrounds = {k: [] for k in kernels}
    clocks = ClockSampler(local, enabled=(rank == 0 and not args.no_clocks))
    barrier(world)
    torch.cuda.synchronize(dev)
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        ev = launch_step(used[i])
        for k in kernels:
            rec[k].append((ev[k][0].elapsed_time(ev[k][1]) * 1e-3, *counts[(used[i], k)]))
            nrounds[k].append(rounds[(used[i], k)])
    torch.cuda.synchronize(dev)
    barrier(world)
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()

    t_dev = sum(t for k in kernels for (t, _, _) in rec[k])
    edges = sum(mR for k in kernels for (_, _, mR) in rec[k])
    t_max = max_over_ranks(t_dev, world, dev)
    edges_all = sum_over_ranks(edges, world, dev)
    value = edges_all / t_max / 1e9

    # roofline of the dominant kernel (largest share of device time)
    hbm, peak_src = peaks()
    per_kernel = {}
    for k in kernels:
        tk = sum(t for (t, _, _) in rec[k])
        bk = sum(alg_bytes(k, g.n, R, mR) for (_, R, mR) in rec[k])
        nk = len(rec[k])
        q_gteps = [mR / t / 1e9 for (t, _, mR) in rec[k]]
        per_kernel[k] = dict(time_s=tk, bytes=bk, launches=nk, achieved_gbs=bk / tk / 1e9,
                             gteps=sum(mR for (_, _, mR) in rec[k]) / tk / 1e9,
                             gteps_median=statistics.median(q_gteps),
                             gteps_harmonic=len(q_gteps) / sum(1.0 / x for x in q_gteps),
                             us_per_launch=1e6 * tk / nk,
                             rounds_per_launch=sum(nrounds[k]) / nk,
                             us_per_round=1e6 * tk / max(1, sum(nrounds[k])),
                             work_inefficiency=scanned[k] / max(1, sum(counts[(j, k)][1] for j in set(used))))
    dom = max(kernels, key=lambda k: per_kernel[k]["time_s"])
    kname = {"bfs": "k_iterate<BFS>", "sssp": "k_iterate<SSSP>", "cc": "k_iterate<CC>", "cc_jump": "k_iterate<CCJ>"}[dom]
    pk = per_kernel[dom]
    traffic = measured_traffic(kname, args.workload if args.workload != "rmat20" or args.scale == 20 else "")
    roofline = {"bound": "hbm", "achieved": round(pk["achieved_gbs"], 2), "peak": hbm, "unit": "GB/s",
                "frac": round(pk["achieved_gbs"] / hbm, 4), "traffic": traffic, "kernel": kname,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src,
                "bytes_per_launch": int(pk["bytes"] / pk["launches"]),
                "by_kernel": {k: {kk: (round(v, 4) if isinstance(v, float) else v) for kk, v in d.items()}
                              for k, d in per_kernel.items()}}

    # BFS in the other form (top-down only when the headline is direction-optimising, and the
    # reverse), event-timed on the same sources outside the headline's timed region
    bfs_other = None
    if "bfs" in kernels and args.workload == "rmat20":
        t_other = dict(ktune["bfs"] or {})
        t_other["flags"] = int(t_other.get("flags", 0)) ^ 2
        t_other = t_other if any(t_other.values()) else None
        if not args.diropt:
            dg_other = ctx.load(g, validate=False, in_edges=True)
        else:
            dg_other = dg
        tt, bb, ee, nn = 0.0, 0, 0, 0
        for i in range(args.steps):
            j = used[i]
            with torch.cuda.stream(stream):
                flush.fill_(i)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.iterate_async("bfs", dg_other, wls[j], out["bfs"], tuning=t_other)
            e1.record(stream)
            ctx.sync()
            if i < max(1, args.warmup // 2):
                continue  # first uses of the other form
            R, mR = counts[(j, "bfs")]
            tt += e0.elapsed_time(e1) * 1e-3
            bb += alg_bytes("bfs", g.n, R, mR)
            ee += mR
            nn += 1
        if nn:
            bfs_other = {"form": "top-down only" if args.diropt else "direction-optimising",
                         "us_per_launch": round(1e6 * tt / nn, 2), "gteps": round(ee / tt / 1e9, 4),
                         "roofline_frac": round(bb / tt / 1e9 / hbm, 4), "launches": nn}
        if dg_other is not dg:
            dg_other.close()

    # e2e through the C-ABI with pinned host buffers (host wall clock per call, copies inside)
    host_out = torch.empty(g.n, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    s = torch.empty(1, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    e2e_t, e2e_edges = 0.0, 0
    n_e2e = min(args.steps, len(srcs))
    for i in range(max(args.warmup, 1)):  # untimed: first use of the pinned buffers and the host-copy path
        s[0] = srcs[i % len(srcs)]
        for k in kernels:
            ctx.run_host(k, dg, None if k.startswith("cc") else s, out=host_out, tuning=ktune[k])
    torch.cuda.synchronize(dev)
    for i in range(n_e2e):
        s[0] = srcs[(args.warmup + i) % len(srcs)]
        for k in kernels:
            t0 = time.perf_counter()
            ctx.run_host(k, dg, None if k.startswith("cc") else s, out=host_out, tuning=ktune[k])
            e2e_t += time.perf_counter() - t0
            e2e_edges += reached_stats(g, host_out)[1]
    e2e_max = max_over_ranks(e2e_t, world, dev)
    e2e_val = sum_over_ranks(e2e_edges, world, dev) / e2e_max / 1e9

    # iteration outlining vs one launch per round (host loop), BFS from the first timed source
    outlining = None
    if "bfs" in kernels and not args.no_per_launch:
        j = used[0]
        t_pl = []
        for rep_i in range(3):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            _, st = ctx.iterate("bfs", dg, wls[j], out["bfs"], mode="per_launch", tuning=ktune["bfs"])
            t_pl.append(time.perf_counter() - t0)
        if args.diropt:
            # the per-launch form runs top-down rounds only: compare it with the persistent top-down form
            t_plain = dict(ktune["bfs"] or {})
            t_plain["flags"] = int(t_plain.get("flags", 0)) & ~2
            t_pers = []
            for rep_i in range(4):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.iterate_async("bfs", dg, wls[j], out["bfs"], tuning=t_plain if any(t_plain.values()) else None)
                e1.record(stream)
                ctx.sync()
                if rep_i:
                    t_pers.append(e0.elapsed_time(e1) * 1e-3)
        else:
            t_pers = [t for (t, _, _), jj in zip(rec["bfs"], used) if jj == j]
        outlining = {"kernel": "bfs (top-down rounds in both forms)", "rounds": st["rounds"],
                     "per_launch_us": round(1e6 * min(t_pl), 1), "per_launch_launches": st["launches"],
                     "persistent_us": round(1e6 * statistics.median(t_pers), 1),
                     "speedup": round(min(t_pl) / statistics.median(t_pers), 2)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(g, srcs_all, kernels, args.cpu_budget)

    # the other parts of the metric on the same GPU, in the same run: the 256-instance batch
    # (batched vs one launch per query) and a serving window (served vs one launch per query,
    # p50/p99 latency)
    extras = {}
    if args.workload == "rmat20" and args.scale == 20 and not args.no_extras:
        import copy

        sub = copy.copy(args)
        sub.tuning, sub.steps, sub.warmup = "", min(args.steps, 10), 3
        sub.instances, sub.batch_set, sub.no_autotune, sub.wave_mb = 256, "rmat", False, None
        extras["batch"] = run_batch(sub, world, rank, local, embedded=True)
        sub = copy.copy(args)
        sub.tuning, sub.rate, sub.duration, sub.verify = "", 2000.0, args.sub_serve_duration, 16
        sub.serve_scale, sub.slots, sub.epoch_rounds, sub.arena_gb = 24, 512, 32, 0.0
        extras["serve"] = run_serve(sub, world, rank, local, embedded=True)

    if rank == 0:
        launches_per_step = len(kernels)  # one persistent Iterate launch per query (the L2 flush fill is torch's)
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * t_max / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": dict(workload=name, **meta, mode="persistent (iteration-outlined cooperative launch)"
                           + (", BFS direction-optimising" if args.diropt else "")
                           + (f", {local_k} CTA-local sub-rounds per round" if local_k else ""),
                           parallelism=f"replicas x{world} (queries sharded, no collective)",
                           l2="flushed between steps (512 MB write, outside the events)",
                           tuning={k: {**ctx.default_tuning, **(ktune[k] or {})} for k in kernels},
                           autotuned=autotuned or None),
            "e2e": {"value": round(e2e_val, 4), "unit": "GTEPS", "h2d_bytes_per_step": 4 * len(kernels),
                    "d2h_bytes_per_step": 4 * g.n * len(kernels)},
            "gpu_launches": launches_per_step * args.steps,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clk,
            "wall_s_timed_region": round(t_wall, 4),
            "outlining": outlining,
            "rmat20_bfs_roofline_frac": (round(per_kernel["bfs"]["achieved_gbs"] / hbm, 4)
                                         if "bfs" in per_kernel and args.workload == "rmat20" else None),
            "bfs_other_form": bfs_other,
            **extras,
        }
        print(json.dumps(line), flush=True)
    for wl in wls:
        wl.close()
    dg.close()
    ctx.close()


# ----------------------------------------------------------------------------- batched workload

def run_batch(args, world, rank, local, embedded=False):
    """256 independent SSSP instances (R-MAT scale 10..18, edge factor 8, 1-4 sources) in one
    CUDA-graph-replayed persistent launch, against the same queries run one launch each.
    embedded: return a compact record (rank 0) for the default bench line instead of printing."""
    import torch

    from paper_1607_05707_gb300 import irgl as C
    from paper_1607_05707_gb300.api import Batch, Context, as_u32

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.batch_set == "grids":
        from paper_1607_05707_gb300 import inputs

        inst_all = inputs.workload_grid_batch()
        tuning = json.loads(args.tuning) if args.tuning else None
    else:
        inst_all = [(g, s, "sssp") for g, s in inputs_workload_batch(args.instances)]
        tuning = json.loads(args.tuning) if args.tuning else None
    inst = shard(inst_all, world, rank)
    stream = torch.cuda.Stream(device=dev)
    ctx = Context(local, stream)
    loaded = {}  # queries on one graph share its device copy
    for g, _, _ in inst:
        if id(g) not in loaded:
            loaded[id(g)] = ctx.load(g, validate=False)
    dgs = [loaded[id(g)] for g, _, _ in inst]
    b = Batch(ctx, max(len(inst), 1))
    for (g, s, k), dg in zip(inst, dgs):
        b.add(k, dg, s)
    wave_bytes = 0 if args.wave_mb is None else ((1 << 64) - 1 if args.wave_mb < 0 else args.wave_mb << 20)
    info = b.prepare(tuning, use_cuda_graph=True, wave_bytes=wave_bytes)
    autotuned = None
    if not args.no_autotune and not args.tuning and args.wave_mb is None:
        # the batch is left prepared with the fastest tuning and wave budget (outside the timed region)
        t0 = time.perf_counter()
        tuning, tune_ms = b.autotune(reps=2)
        info = C.irgl_batch_info(b.handle)
        autotuned = {"search_s": round(time.perf_counter() - t0, 1), "median_ms": round(tune_ms, 3)}
    b.run()
    mR = []
    for q, (g, s, _) in enumerate(inst):
        res, _ = b.result(q)
        mR.append(reached_stats(g, res)[1])
    edges = float(sum(mR))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    for _ in range(args.warmup):
        b.run()
    clocks = ClockSampler(local, enabled=(rank == 0 and not args.no_clocks))
    barrier(world)
    times = []
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(i)
        torch.cuda.synchronize(dev)
        st = b.run()
        times.append(st["device_ms"] * 1e-3)
    barrier(world)
    clk = clocks.stop()
    t_batch = max_over_ranks(sum(times) / len(times), world, dev)
    value = sum_over_ranks(edges, world, dev) / t_batch / 1e9
    # the same queries, one persistent launch each (host waits for each query's status)
    outs = [ctx.state(g.n) for g, _, _ in inst]
    wls = []
    for (g, s, _) in inst:
        wl = ctx.worklist(8)
        wl.push(s)
        wls.append(wl)
    for q in range(min(8, len(inst))):
        ctx.iterate_async(inst[q][2], dgs[q], wls[q], outs[q], tuning=tuning)
        ctx.sync()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    dev_sum = 0.0
    for q in range(len(inst)):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.iterate_async(inst[q][2], dgs[q], wls[q], outs[q], tuning=tuning)
        e1.record(stream)
        ctx.sync()
        dev_sum += e0.elapsed_time(e1) * 1e-3
    t_seq = time.perf_counter() - t0
    for q in range(len(inst)):  # same bytes out
        if not np.array_equal(as_u32(outs[q])[: inst[q][0].n], b.result(q)[0]):
            raise RuntimeError(f"batched result of instance {q} differs from its one-launch result")
    seq_gteps = sum_over_ranks(edges, world, dev) / max_over_ranks(t_seq, world, dev) / 1e9
    seq_dev_gteps = sum_over_ranks(edges, world, dev) / max_over_ranks(dev_sum, world, dev) / 1e9
    # e2e: one batched run plus one copy of every instance's result into pinned host memory
    total_n = sum(g.n for g, _, _ in inst)
    host = torch.empty(max(total_n, 1), dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    t_e2e_all = []
    for _ in range(3):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        b.run()
        res_all = b.results(host)
        t_e2e_all.append(time.perf_counter() - t0)
    for q in range(len(inst)):  # the one-transfer copy holds each query's own result
        if not np.array_equal(res_all[q], b.result(q)[0]):
            raise RuntimeError(f"bulk result copy of instance {q} differs from its own copy")
    t_e2e = max_over_ranks(statistics.median(t_e2e_all), world, dev)
    e2e = sum_over_ranks(edges, world, dev) / t_e2e / 1e9
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not embedded:
        import oracle

        tt, ee, nq = 0.0, 0, 0
        for (g, s, k), m in zip(inst, mR):
            t1 = time.perf_counter()
            oracle.run(k, g, s)
            tt += time.perf_counter() - t1
            ee += m
            nq += 1
            if tt > args.cpu_budget:
                break
        cpu = {"value": ee / tt / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle", "cpu": host_cpu(),
               "sample": f"first {nq} instances (serial BFS / Dijkstra), {tt:.1f} s on {platform.machine()} host"}
    hbm, peak_src = peaks()
    nbytes = sum(alg_bytes(k, g.n, int((b.result(q)[0] != INF).sum()), m) for q, ((g, _, k), m) in enumerate(zip(inst, mR)))
    if embedded:
        b.close()
        for wl in wls:
            wl.close()
        for dg in loaded.values():
            dg.close()
        ctx.close()
        if rank != 0:
            return None
        return {
            "workload": (f"batch{len(inst_all)}: SSSP instances, R-MAT scale U{{10..18}}, edge factor 8, 1-4 sources, "
                         f"w in [1,100]; one CUDA-graph replay of {info['waves']} wave(s)"),
            "gteps": round(value, 4), "ms_per_run": round(1e3 * t_batch, 4), "steps": args.steps,
            "per_launch_gteps": round(seq_dev_gteps, 4), "batched_vs_per_launch": round(value / seq_dev_gteps, 3),
            "clock": "device (CUDA events) for both forms; per-launch = the same instances, one persistent launch each",
            "per_launch_gteps_wall": round(seq_gteps, 4),
            "e2e_gteps": round(e2e, 4),
            "roofline_frac": round(nbytes / t_batch / 1e9 / hbm, 4),
            "verified": "every instance's batched result equals its one-launch result",
            "tuning": {**ctx.default_tuning, **(tuning or {})}, "autotuned": autotuned, "clocks": clk,
        }
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * t_batch, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": dict(workload=(f"batch{args.instances}: SSSP instances, R-MAT scale U{{10..18}}, edge factor 8, "
                                     f"1-4 sources, w in [1,100]" if args.batch_set == "rmat" else
                                     "grids32: 32 queries (70% BFS / 30% SSSP, uniform sources) on 16 weighted 4-neighbour "
                                     "grids of side U[256,1024], w in [1,100]")
                                    + f"; one CUDA-graph replay of {info['waves']} wave(s), one persistent launch each",
                           instances=len(inst_all), edges_out_of_reached=int(edges), batch=info,
                           parallelism=f"instances sharded x{world}", l2="flushed between steps (512 MB write)",
                           tuning={**ctx.default_tuning, **(tuning or {})}, autotuned=autotuned),
            "per_launch": {"gteps_wall": round(seq_gteps, 4), "gteps_device": round(seq_dev_gteps, 4),
                           "form": "same instances, one persistent launch each, host waits per query"},
            "batched_vs_per_launch": round(value / seq_dev_gteps, 3),
            "batched_vs_per_launch_clock": "device (CUDA events) for both forms",
            "e2e": {"value": round(e2e, 4), "unit": "GTEPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": int(4 * sum(g.n for g, _, _ in inst))},
            "gpu_launches": (3 * info["waves"] + 1) * args.steps,
            "roofline": {"bound": "hbm", "achieved": round(nbytes / t_batch / 1e9, 2), "peak": hbm, "unit": "GB/s",
                         "frac": round(nbytes / t_batch / 1e9 / hbm, 4), "traffic": measured_traffic("k_batch_iterate", f"batch{args.instances}-{args.batch_set}"),
                         "kernel": "k_batch_iterate", "bytes_per_launch": int(nbytes)},
            "cpu_baseline": cpu, "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    b.close()


def inputs_workload_batch(count):
    from paper_1607_05707_gb300 import inputs

    return inputs.workload_batch(count=count)


# ----------------------------------------------------------------------------- serving workload

def run_serve(args, world, rank, local, embedded=False):
    """Poisson arrivals of BFS (70%) / SSSP (30%) queries with uniform sources against one R-MAT
    graph and 32 grids of side U[256, 2048], served by the continuous-batching server. Then a
    sample of the same queries runs one persistent launch per query (host waits for each), the
    one-query-per-launch form the served throughput is compared with (host wall clock for both).
    embedded: return a compact record (rank 0) for the default bench line instead of printing."""
    import threading

    import torch

    from paper_1607_05707_gb300 import inputs
    from paper_1607_05707_gb300.api import Context, Server

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rng = np.random.default_rng(2005)
    graphs = [inputs.rmat(args.serve_scale, 16, seed=1005, weights=True)]
    sides = rng.integers(256, 2049, size=32)
    graphs += [inputs.mesh(int(sd), int(sd), seed=1005000 + i, weights=True) for i, sd in enumerate(sides)]
    # per-query near-far for the SSSP queries (delta 512: measured 3x the plain rounds' GTEPS
    # on this mix, where grid SSSP re-relaxes each edge about 40 times); the R-MAT graph's BFS
    # queries run alone and direction-optimising (flag 2, in-edges loaded); 15 CTA-local
    # sub-rounds per batched round, so a grid query needs far fewer global rounds than levels
    # (10 s of arrivals: p50 126 -> 67 ms, p99 372 -> 243 ms at the same 27.7 GTEPS); CTAs of
    # 1024 (26.8 GTEPS, p50 340 ms, against 26.0 and 564 ms with 128, before sub-rounds)
    tuning = json.loads(args.tuning) if args.tuning else {"delta": 512, "flags": 2 | (15 << 8), "cta_size": 1024}
    ctx = Context(local, torch.cuda.Stream(device=dev))
    dgs = [ctx.load(g, validate=False, in_edges=(i == 0)) for i, g in enumerate(graphs)]
    arrivals = inputs.poisson_arrivals(args.rate, args.duration, seed=2005 + rank)
    nq = len(arrivals)
    gi = rng.integers(0, len(graphs), size=nq)
    kinds = np.where(rng.random(nq) < 0.7, "bfs", "sssp")
    degs = [g.out_degree() for g in graphs]
    srcs = np.empty(nq, dtype=np.int64)
    for i in range(nq):
        d = degs[gi[i]]
        v = int(rng.integers(0, len(d)))
        while d[v] == 0:
            v = int(rng.integers(0, len(d)))
        srcs[i] = v
    verify = set(rng.choice(nq, size=min(args.verify, nq), replace=False).tolist())
    bufs = {i: np.empty(graphs[gi[i]].n, dtype=np.uint32) for i in verify}
    srv = Server(ctx, arena_bytes=int(args.arena_gb * (1 << 30)), max_slots=args.slots,
                 epoch_rounds=args.epoch_rounds, count_edges=True, tuning=tuning)
    # warm-up: a few queries before the clock starts
    for i in range(min(8, nq)):
        srv.submit(kinds[i], dgs[gi[i]], int(srcs[i]))
    srv.drain(600)
    base = srv.stats()
    tickets = [0] * nq
    clocks = ClockSampler(local, enabled=(rank == 0 and not args.no_clocks))
    barrier(world)
    t0 = time.perf_counter()
    for i in range(nq):
        dt = t0 + arrivals[i] - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        tickets[i] = srv.submit(kinds[i], dgs[gi[i]], int(srcs[i]), bufs.get(i))
    srv.drain(3600)
    t_total = time.perf_counter() - t0
    clk = clocks.stop()
    infos = [srv.poll(t) for t in tickets]
    st = srv.stats()
    lat = np.array([x["latency_s"] for x in infos])
    edges = float(sum(x["edges"] for x in infos))
    t_first = min(x["t_submit_s"] for x in infos)
    t_last = max(x["t_done_s"] for x in infos)
    span = max_over_ranks(t_last - t_first, world, dev)
    value = sum_over_ranks(edges, world, dev) / span / 1e9
    # bit-exact check of a sample against the oracle (after timing)
    import oracle

    bad = 0
    for i in verify:
        want = oracle.run(str(kinds[i]), graphs[gi[i]], np.array([srcs[i]], np.uint32))
        bad += int(not np.array_equal(want, bufs[i]))
    if bad:
        raise RuntimeError(f"{bad} of {len(verify)} sampled served queries differ from the oracle")
    # one-query-per-launch form on a sample of the served queries: each query alone, one persistent
    # launch, host waiting for its status, with the best single-query settings per graph class
    # (R-MAT: direction-optimising BFS; grids: CTA-local sub-rounds)
    pl_idx = sorted(rng.choice(nq, size=min(args.per_launch_sample, nq), replace=False).tolist())
    wl = ctx.worklist(4)
    pl_out = ctx.state(max(g.n for g in graphs))

    def pl_tuning(i):
        if gi[i] == 0:
            return {"flags": 2} if kinds[i] == "bfs" else None
        return {"flags": 15 << 8}

    for i in pl_idx[:4]:  # untimed first use of each setting
        wl.clear()
        wl.push([int(srcs[i])])
        ctx.iterate(str(kinds[i]), dgs[gi[i]], wl, pl_out, tuning=pl_tuning(i))
    pl_wall, pl_dev, pl_edges = 0.0, 0.0, 0
    for i in pl_idx:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        wl.clear()
        wl.push([int(srcs[i])])
        e0.record(ctx.stream)
        ctx.iterate_async(str(kinds[i]), dgs[gi[i]], wl, pl_out, tuning=pl_tuning(i))
        e1.record(ctx.stream)
        ctx.sync()
        pl_wall += time.perf_counter() - t1
        pl_dev += e0.elapsed_time(e1) * 1e-3
        pl_edges += int(infos[i]["edges"])
    wl.close()
    pl_gteps = sum_over_ranks(pl_edges, world, dev) / max_over_ranks(pl_wall, world, dev) / 1e9
    pl_gteps_dev = sum_over_ranks(pl_edges, world, dev) / max_over_ranks(pl_dev, world, dev) / 1e9
    per_launch = {"gteps_wall": round(pl_gteps, 4), "gteps_device": round(pl_gteps_dev, 4), "sample": len(pl_idx),
                  "form": "each sampled query alone, one persistent launch, host waits for its status; "
                          "R-MAT BFS direction-optimising, grid queries with 15 CTA-local sub-rounds"}
    lat_ms = {"p50_ms": round(1e3 * float(np.percentile(lat, 50)), 3),
              "p99_ms": round(1e3 * float(np.percentile(lat, 99)), 3), "max_ms": round(1e3 * float(lat.max()), 3)}
    if embedded:
        srv.close()
        for d in dgs:
            d.close()
        ctx.close()
        if rank != 0:
            return None
        return {
            "workload": (f"serve: Poisson {args.rate:g} q/s for {args.duration:g} s, 70% BFS / 30% SSSP, R-MAT scale "
                         f"{args.serve_scale} (ef 16) + 32 grids of side U[256,2048]"),
            "queries": nq, "gteps": round(value, 4), **lat_ms, "served_in_s": round(span, 3),
            "per_launch": per_launch, "served_vs_per_launch": round(value / pl_gteps, 3),
            "clock": "host wall clock for both forms (served: first submission to last result in host memory)",
            "verified_against_oracle": len(verify), "slots": args.slots, "epoch_rounds": args.epoch_rounds,
            "tuning": {**ctx.default_tuning, **(tuning or {})}, "clocks": clk,
        }
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "GTEPS", "n_gpus": world, "steps": nq,
            "warmup": 8, "ms_per_step": round(1e3 * span / nq, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": dict(workload=f"serve: Poisson {args.rate:g} q/s for {args.duration:g} s, 70% BFS / 30% SSSP, "
                                    f"R-MAT scale {args.serve_scale} (ef 16) + 32 grids of side U[256,2048]",
                           queries=nq, slots=args.slots, epoch_rounds=args.epoch_rounds,
                           arena_entries=st["arena_entries"], tuning={**ctx.default_tuning, **(tuning or {})},
                           parallelism=f"replicas x{world} (independent arrival streams)"),
            "latency": lat_ms,
            "per_launch": per_launch, "served_vs_per_launch": round(value / pl_gteps, 3),
            "server": {k: st[k] - base.get(k, 0) if k in ("completed", "epochs", "rounds", "edges", "solo") else st[k]
                       for k in ("completed", "rejected", "epochs", "rounds", "edges", "busy_s", "kernel_s", "grid",
                                 "cta_size", "solo")},
            "verified_against_oracle": len(verify),
            "e2e": {"value": round(value, 4), "unit": "GTEPS", "h2d_bytes_per_step": 4,
                    "d2h_bytes_per_step": int(4 * np.mean([graphs[g].n for g in gi]))},
            "wall_s": round(t_total, 3), "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    srv.close()


# ----------------------------------------------------------------------------- minimum spanning forest

def msf_graph(args):
    from paper_1607_05707_gb300 import inputs

    if args.msf_graph == "rmat":
        r, _ = inputs.workload_rmat20(nsrc=1, scale=args.scale)
        u = np.repeat(np.arange(r.n), np.diff(r.row_ptr.astype(np.int64)))
        g = inputs.csr_from_edges(r.n, np.concatenate([u, r.col]), np.concatenate([r.col, u]),
                                  np.concatenate([r.w, r.w]), symmetric=True)
        return g, f"msf-rmat{args.scale}: R-MAT scale {args.scale} (edges of both directions, w in [1,100])"
    g, _ = inputs.workload_mesh(args.mesh_side, weights=True)
    return g, f"msf-mesh{args.mesh_side}: {args.mesh_side}^2 mesh (1% edges deleted, 0.1% extra r<=8), w in [1,100]"


def run_msf(args, world, rank, local):
    """Minimum spanning forest by Boruvka (outlined Pipe: find_min with Atomic component locks, link,
    pointer jumping); queries are whole graphs, so N GPUs run N replicas."""
    import torch

    from paper_1607_05707_gb300.api import Context

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    g, name = msf_graph(args)
    tuning = json.loads(args.tuning) if args.tuning else None
    stream = torch.cuda.Stream(device=dev)
    ctx = Context(local, stream)
    dg = ctx.load(g, validate=False)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    for _ in range(args.warmup):
        ctx.msf(dg, lock=args.msf_lock, tuning=tuning)
    clocks = ClockSampler(local, enabled=(rank == 0 and not args.no_clocks))
    barrier(world)
    times, st = [], None
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(i)
        torch.cuda.synchronize(dev)
        _, st = ctx.msf(dg, lock=args.msf_lock, tuning=tuning)
        times.append(st["device_ms"] * 1e-3)
    barrier(world)
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    t_step = max_over_ranks(sum(times) / len(times), world, dev)
    value = sum_over_ranks(float(g.m), world, dev) / t_step / 1e9
    # the same forest with a host loop launching each kernel invocation, and with the other lock forms
    forms = {}
    for lock in ("blocking", "ticket", "retry"):
        _, s1 = ctx.msf(dg, lock=lock, tuning=tuning)
        forms[lock] = {"ms": round(s1["device_ms"], 3), "locks": s1["locks"], "retries": s1["retries"]}
    t0 = time.perf_counter()
    _, spl = ctx.msf(dg, mode="per_launch", lock=args.msf_lock, tuning=tuning)
    t_pl = time.perf_counter() - t0
    # e2e: the call with the forest copied to host memory (inside the call), wall clock
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    edges, _ = ctx.msf(dg, lock=args.msf_lock, tuning=tuning)
    t_e2e = max_over_ranks(time.perf_counter() - t0, world, dev)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        t0 = time.perf_counter()
        oracle.msf(g.n, g.row_ptr, g.col, g.w)
        tc = time.perf_counter() - t0
        cpu = {"value": g.m / tc / 1e9, "unit": "G input edges/s", "cores": 1, "kind": "oracle", "cpu": host_cpu(),
               "sample": f"one Kruskal run on the whole graph ({g.m} CSR entries), {tc:.1f} s serial"}
    hbm, peak_src = peaks()
    nbytes = 12 * g.m + 16 * g.n  # col + w + comp[v] per CSR entry, row_ptr pair + comp[u] + record per vertex
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "G input edges/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": name, "V": g.n, "m": g.m, "lock": args.msf_lock,
                       "mode": "persistent (outlined Pipe: find_min / link / jump in one cooperative launch)",
                       "parallelism": f"replicas x{world}", "l2": "flushed between steps (512 MB write, outside)",
                       "iterations": st["iterations"], "invocations": st["invocations"],
                       "cta_size": st["cta_size"], "grid": st["grid"], "forest_edges": st["edges"],
                       "forest_weight": st["weight"]},
            "e2e": {"value": round(g.m / t_e2e / 1e9, 4), "unit": "G input edges/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 4 * int(len(edges))},
            "gpu_launches": args.steps,
            "roofline": {"bound": "hbm", "achieved": round(nbytes / t_step / 1e9, 2), "peak": hbm, "unit": "GB/s",
                         "frac": round(nbytes / t_step / 1e9 / hbm, 4), "traffic": measured_traffic("k_msf", f"msf-{args.msf_graph}"),
                         "kernel": "k_msf", "bytes_per_launch": int(nbytes),
                         "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)"},
            "lock_forms": forms,
            "outlining": {"per_launch_us": round(1e6 * t_pl, 1), "per_launch_launches": spl["launches"],
                          "persistent_us": round(1e6 * t_step, 1), "speedup": round(t_pl / t_step, 2)},
            "cpu_baseline": cpu,
            "clocks": clk,
            "wall_s_timed_region": round(t_wall, 4),
        }
        print(json.dumps(line), flush=True)
    dg.close()
    ctx.close()


def main():
    args = parse_args()
    ClockSampler.LOG_DIR = args.clocks_log
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "batch256":
        run_batch(args, world, rank, local)
    elif args.workload == "serve":
        run_serve(args, world, rank, local)
    elif args.workload == "msf":
        run_msf(args, world, rank, local)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
