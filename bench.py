"""Benchmark of the local-max matching hot path on GB300.

Default workload: R-MAT scale 23, edge factor 16 (a,b,c,d = .57,.19,.19,.05),
random relabel, loops dropped, duplicates removed, weights U[0,1) -- the
largest single-GPU configuration; metric = input edges per second to a
maximal matching (m / time of one lm_match from a device-resident graph to
mate[] on the device).

One JSON line on stdout (rank 0).  Other workloads (--workload er|grid|batch|serve)
print the same kind of line for their own metric.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lm|reference] [--workload rmat23]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "input edges/s to maximal matching"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 7:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier_max(value: float, ws: int) -> float:
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ workloads

def make_workload(name: str):
    import synth
    if name == "rmat23":
        return synth.rmat(scale=23, edge_factor=16, seed=3), 103, \
            "R-MAT scale 23, edge factor 16, a=.57 b=.19 c=.19 d=.05, relabelled, dedup, w~U[0,1)"
    if name == "rmat21":
        return synth.rmat(scale=21, edge_factor=16, seed=3), 103, \
            "R-MAT scale 21, edge factor 16 (profiling-size case of the R-MAT family)"
    if name == "grid":
        return synth.grid(1024, 1024, 0.05, seed=2), 102, "2D grid 1024x1024 4-neighbour + 5% long-range, w~U[0,1)"
    if name == "er":
        return synth.er(10_000, 50_000, seed=1), 101, "Erdos-Renyi n=10000 m=50000, w~U[0,1)"
    raise ValueError(name)


def sweep_model_bytes(st: dict) -> int:
    """Algorithmic HBM bytes of all sweep launches of one match, from the
    per-round live counts: a compacting sweep over E_r entries / R_r rows
    reads 16 B per entry (12 B entry + 4 B neighbour-state gather), writes
    12 B per surviving entry, reads 8 B per row and writes 12 B per new row;
    the candidate-only sweep of round 0 reads 16 B per entry, 8 B per row and
    writes 4 B per row."""
    rm, rn = st["round_m"], st["round_n"]
    R = len(rm)
    E = [2 * x for x in rm] + [0]
    N = list(rn) + [0]
    b = 16 * E[0] + 12 * N[0] if R else 0
    for r in range(R):
        b += 16 * E[r] + 12 * E[r + 1] + 8 * N[r] + 12 * N[r + 1]
    return b


def run_lm(args, ws, rank, local):
    import torch
    import paper_1302_4587_gb300 as lm
    torch.cuda.set_device(local)
    g, seed, desc = make_workload(args.workload)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ctx = lm.lm_create(local, stream)
    eu = torch.from_numpy(g.eu.view(np.int32)).to(dev)
    ev = torch.from_numpy(g.ev.view(np.int32)).to(dev)
    w = torch.from_numpy(g.w).to(dev)
    h = lm.lm_graph_create(ctx, g.n, eu, ev, w)
    del eu, ev, w
    mate = torch.empty(g.n, dtype=torch.int32, device=dev)
    launches = 0
    for _ in range(max(args.warmup, 3)):
        _, st = lm.lm_match(ctx, h, seed, mate, stats=True)
    launches_per_step = st["launches"]
    torch.cuda.synchronize()
    _barrier(ws)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            lm.lm_match(ctx, h, seed, mate)
            launches += launches_per_step
        e1.record(stream)
        torch.cuda.synchronize()
    _barrier(ws)
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = _barrier_max(ms, ws)
    clocks = clk.summary()

    # per-kernel device times (CUDA events recorded by the library on its stream)
    pctx = lm.lm_create(local, stream, flags=lm.LM_F_PROFILE)
    sweep_ms, sweep_n, total_ms, vert_ms = [], [], [], []
    for i in range(max(args.warmup, 3) + args.steps):
        _, pst = lm.lm_match(pctx, h, seed, mate, stats=True)
        if i >= max(args.warmup, 3):
            sweep_ms.append(pst["kernel_ms"][lm.LM_K_SWEEP])
            vert_ms.append(pst["kernel_ms"][lm.LM_K_VERTEX])
            sweep_n.append(pst["kernel_launches"][lm.LM_K_SWEEP])
            total_ms.append(pst["total_ms"])
    lm.lm_destroy(pctx)
    peak, peak_kind = _peaks()
    bytes_sweep = sweep_model_bytes(pst)
    sw_ms = statistics.median(sweep_ms)
    achieved = bytes_sweep / (sw_ms * 1e-3) / 1e9 if sw_ms > 0 else 0.0

    # end to end through the C ABI with host buffers: graph upload + build, match, result download
    e2e = None
    if rank == 0 or ws > 1:
        peu = torch.from_numpy(g.eu.view(np.int32)).pin_memory()
        pev = torch.from_numpy(g.ev.view(np.int32)).pin_memory()
        pw = torch.from_numpy(g.w).pin_memory()
        hmate = torch.empty(g.n, dtype=torch.int32).pin_memory()
        reps = max(1, min(args.steps, 5))
        for i in range(reps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hh = lm.lm_graph_create(ctx, g.n, peu, pev, pw)
            lm.lm_match(ctx, hh, seed, hmate)
            lm.lm_graph_destroy(hh)
            t1 = time.perf_counter()
            if i == 0:
                e2e_times = []
            else:
                e2e_times.append(t1 - t0)
        e2e_s = statistics.median(e2e_times)
        e2e = {"value": g.m / e2e_s, "unit": "edges/s", "h2d_bytes_per_step": 12 * g.m,
               "d2h_bytes_per_step": 4 * g.n, "ms_per_step": e2e_s * 1e3,
               "includes": "lm_graph_create from pinned host arrays + lm_match to a pinned host mate + lm_graph_destroy"}
    lm.lm_graph_destroy(h)
    lm.lm_destroy(ctx)
    out = {
        "metric": METRIC, "value": ws * g.m / (ms_max * 1e-3), "unit": "edges/s", "n_gpus": ws,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64 keys / u32 ids (integer)", "data": "synthetic",
        "config": {"workload": args.workload, "desc": desc, "n": g.n, "m": g.m, "seed": seed,
                   "rounds": pst["rounds"], "l2": "inputs larger than L2 (graph arrays 3.1 GB)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": "k_sweep (all launches of one match)",
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "bytes_per_match": bytes_sweep, "sweep_ms_per_match": sw_ms,
                     "sweep_launches_per_match": statistics.median(sweep_n),
                     "vertex_ms_per_match": statistics.median(vert_ms),
                     "profiled_total_ms": statistics.median(total_ms)},
        "clocks": clocks, "gpu_launches": launches, "e2e": e2e,
    }
    return out, g


def cpu_baseline(budget_s: float = 20.0):
    """The oracle (greedy, one thread) on a bounded sample of the workload: an
    R-MAT graph of the same family at scale 20."""
    import oracle
    import synth
    g = synth.rmat(scale=20, edge_factor=16, seed=3)
    reps, t_tot = 0, 0.0
    while reps < 1 or (t_tot < budget_s * 0.5 and reps < 3):
        t0 = time.perf_counter()
        oracle.greedy(g.n, g.eu, g.ev, g.w, 103)
        t_tot += time.perf_counter() - t0
        reps += 1
    per = t_tot / reps
    return {"value": g.m / per, "unit": "edges/s", "cores": 1, "kind": "oracle",
            "sample": f"R-MAT scale 20 ef 16 (m={g.m}), greedy oracle, {reps} run(s), {per:.2f} s each"}


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    import oracle
    import synth
    g = synth.rmat(scale=20, edge_factor=16, seed=3)
    for _ in range(args.warmup if args.warmup < 1 else 1):
        oracle.greedy(g.n, g.eu, g.ev, g.w, 103)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.greedy(g.n, g.eu, g.ev, g.w, 103)
        times.append(time.perf_counter() - t0)
    per = statistics.median(times)
    v = g.m / per
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "edges/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64 keys / u32 ids (integer)", "data": "synthetic",
            "config": {"workload": args.workload, "sample": "R-MAT scale 20 ef 16 (bounded sample of the workload)"},
            "cpu_baseline": {"value": v, "unit": "edges/s", "cores": 1, "kind": "oracle",
                             "sample": f"R-MAT scale 20 ef 16, m={g.m}, greedy oracle per step"},
            "e2e": {"value": v, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lm", choices=["lm", "reference"])
    ap.add_argument("--workload", default="rmat23", choices=["rmat23", "rmat21", "grid", "er"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    ws, rank, local = _dist()
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    out, g = run_lm(args, ws, rank, local)
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline()
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
