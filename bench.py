"""Benchmark of the Flow Fields path on GB300.

One step = the whole path (smoothed images and census of both frames, three flow
fields with their kd trees, hierarchical propagation and random search, two-way
consistency check, region filter, sparsification) for one synthetic 1024x436
Sintel-shaped pair, through the library's C ABI. Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (plain C, three threads, one per flow) on
the same workload; it is the slow baseline, not a target.
Under torchrun (N > 1) every rank runs its own pairs (weak scaling, no data
exchange); the step time is the max over ranks.
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
sys.path.insert(0, ROOT)

METRIC = "ms per 1024×436 pair + cand-evals/s; learned vs plain at equal inliers@3px"
W, H = 1024, 436
WORKLOAD = "Sintel-shaped 1024x436 RGB uint8 pair (3 textured layers, affine motion <= 200 px)"
PARAMS = dict(k=3, r=8, r2=6, leaf=8, R=1, eps=5, e=4, s=50, tile=16, n_rs=3, K=0, seed=0)


def nominal_evals(W, H, p):
    """Schedule-independent candidate evaluations per pair (all three flows):
    per level 8 propagation candidates (4 passes x 2 sources) and n_rs random-
    search candidates per grid point, one re-evaluation per seeded point, and at
    the coarsest level the points of each kd leaf (N / 2^D on average)."""
    N = W * H
    D = 0
    while -(-N // (1 << D)) > p["leaf"]:
        D += 1
    total = 0.0
    for _flow in range(3):
        for lv in range(p["k"], -1, -1):
            n = 1 << lv
            G = -(-W // n) * -(-H // n)
            total += (8 + p["n_rs"]) * G
            if lv == p["k"]:
                total += G * N / (1 << D)
            else:
                total += -(-W // (2 * n)) * -(-H // (2 * n))
    return total


def gather_bytes_prop(W, H, p):
    """Algorithmic target-tap bytes read by the propagation kernels per pair:
    (2r+1)^2 census words of 4 B per evaluated candidate, nominal count."""
    tot = 0.0
    for r in (p["r"], p["r"], p["r2"]):
        taps = (2 * r + 1) ** 2 * 4
        for lv in range(p["k"], -1, -1):
            n = 1 << lv
            G = -(-W // n) * -(-H // n)
            tot += (8 + p["n_rs"]) * G * taps
    return tot


class Clocks:
    """Samples nvidia-smi every 200 ms while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            out, _ = self.proc.communicate(timeout=10)
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_oracle_pair(pair, params):
    import oracle
    t = time.perf_counter()
    oracle.flow_fields(pair["I1"], pair["I2"], params=params, threads=3)
    return time.perf_counter() - t


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1508_05151_gb300 import synth
    import oracle
    oracle.build()
    pairs = [synth.pair_for_config(2, 1000 + i) for i in range(2)]
    for i in range(args.warmup):
        cpu_oracle_pair(pairs[i % 2], PARAMS)
    ts = [cpu_oracle_pair(pairs[i % 2], PARAMS) for i in range(args.steps)]
    ms = 1000.0 * sum(ts) / len(ts)
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": "ms/pair",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": {"workload": WORKLOAD, "W": W, "H": H, **PARAMS},
        "cand_evals_per_s": nominal_evals(W, H, PARAMS) / (ms / 1000.0),
        "cpu_baseline": {"value": ms, "unit": "ms/pair", "cores": 3, "kind": "oracle",
                         "sample": f"{args.steps} full 1024x436 pairs, three flows on three "
                                   "threads, tiled schedule T=16"},
        "e2e": {"value": ms, "unit": "ms/pair", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1508_05151_gb300 import ffapi, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    pairs = [synth.pair_for_config(2, 1000 + 2 * rank + i) for i in range(2)]
    dI = [(torch.from_numpy(p["I1"]).to(dev), torch.from_numpy(p["I2"]).to(dev)) for p in pairs]
    ff = ffapi.FlowFields(W, H, PARAMS, dev)
    flush = torch.empty(256 * 2**20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream()

    for i in range(args.warmup):
        ff.run(*dI[i % 2])
    torch.cuda.synchronize()

    # ---- device-resident timed region ----
    ffapi.profile_enable(True)
    ffapi.profile_reset()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            ev[i][0].record(stream)
            ff.run(*dI[i % 2])
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    prof = ffapi.profile_read()
    ffapi.profile_enable(False)
    local_ms = sum(step_ms)
    t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    pairs_total = args.steps * world
    value = total_ms / pairs_total  # whole-job ms per pair

    # ---- end to end through the public API with host buffers ----
    hI = [(torch.from_numpy(p["I1"]).pin_memory(), torch.from_numpy(p["I2"]).pin_memory())
          for p in pairs]
    nb = ((W + 2) // 3) * ((H + 2) // 3)
    h_flow = torch.empty((H, W, 2), dtype=torch.int16).pin_memory()
    h_valid = torch.empty((H, W), dtype=torch.uint8).pin_memory()
    h_sparse = torch.empty((nb, 4), dtype=torch.int32).pin_memory()
    h_ns = torch.empty(1, dtype=torch.int32).pin_memory()
    dbuf = [(torch.empty_like(dI[0][0]), torch.empty_like(dI[0][1])) for _ in range(2)]
    h2d = 2 * W * H * 3
    d2h = h_flow.numel() * 2 + h_valid.numel() + h_sparse.numel() * 4 + 4
    for i in range(2):
        dbuf[i][0].copy_(hI[i][0], non_blocking=True)
        dbuf[i][1].copy_(hI[i][1], non_blocking=True)
        out = ff.run(*dbuf[i])
    torch.cuda.synchronize()
    barrier()
    e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 0xff)
        e_ev[i][0].record(stream)
        a, b = dbuf[i % 2]
        a.copy_(hI[i % 2][0], non_blocking=True)
        b.copy_(hI[i % 2][1], non_blocking=True)
        out = ff.run(a, b)
        h_flow.copy_(out["flows"][0], non_blocking=True)
        h_valid.copy_(out["valid"], non_blocking=True)
        h_sparse.copy_(out["sparse"], non_blocking=True)
        h_ns.copy_(out["n_sparse"], non_blocking=True)
        e_ev[i][1].record(stream)
    torch.cuda.synchronize()
    e2e_local = sum(a.elapsed_time(b) for a, b in e_ev)
    te = torch.tensor([e2e_local], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = float(te.item()) / pairs_total
    assert int(h_ns.item()) > 0

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (propagation + random search) ----
    hbm, kind = peaks()
    prop_ms_per_launch = prof["prop_ms"] / max(prof["prop_launches"], 1)
    launches_per_pair = prof["prop_launches"] / args.steps
    bytes_per_launch = gather_bytes_prop(W, H, PARAMS) / launches_per_pair
    achieved = bytes_per_launch / (prop_ms_per_launch * 1e-3) / 1e9
    roof = {"kernel": "k_pass (tiled wavefront propagation + random search)",
            "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "traffic": None,
            "peak_kind": f"{kind} HBM copy bandwidth",
            "prop_ms_per_pair": prof["prop_ms"] / args.steps,
            "note": "achieved = nominal target-tap bytes ((2r+1)^2 x 4 B per candidate) / "
                    "mean launch time; the taps are served mostly by L1/L2"}

    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "ms/pair", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "W": W, "H": H, **PARAMS, "pairs_per_rank": args.steps,
                   "l2": "flushed between steps (256 MB write)"},
        "cand_evals_per_s": round(nominal_evals(W, H, PARAMS) * pairs_total / (total_ms / 1e3), 1),
        "wall_s_timed_region": round(wall, 4),
        "gpu_launches": int(prof["launches"]),
        "roofline": roof,
        "e2e": {"value": round(e2e_value, 4), "unit": "ms/pair", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        ms = 1000.0 * cpu_oracle_pair(pairs[0], PARAMS)
        line["cpu_baseline"] = {"value": round(ms, 1), "unit": "ms/pair", "cores": 3,
                                "kind": "oracle",
                                "sample": "one full 1024x436 pair, three flows on three threads"}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
