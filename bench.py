#!/usr/bin/env python
"""Benchmark: interference-sensitivity sweep on B300.

One step = one pass of the whole hot path over the workload: solo calibration
of every stressor level (achieved fraction of peak), the plain launch-per-cell
sweep, the graph-captured batched sweep, and the sensitivity reduction.
`value` is the batched sweep's cells/s (whole job, all ranks); the plain
sweep's cells/s, the stressors' fractions of peak and the reduction are
reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 the script runs under torchrun, one process per GPU; each
rank sweeps its own replica of the workload (interference is a per-GPU
quantity, so the sweep shards without any collective on the data path).
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
sys.path.insert(0, ROOT)

METRIC = "stressor % of resource peak; sweep cells/s batched vs plain; predictor slowdown MAPE"


# ----------------------------------------------------------------------------- helpers
def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------- work units
def stressor_units(kind, cfg, res):
    """Algorithmic work a stressor run did, in the unit of its resource's peak."""
    from paper_2501_16909_b300 import _abi as A

    if kind in (A.IFR_S_HBM, A.IFR_S_L2):
        return res["work"] * cfg.block * 64, "B"
    raise ValueError(kind)


def calibrate(ctx, wl, peaks):
    """Solo, fixed-work run of every stressor level: achieved fraction of peak."""
    from paper_2501_16909_b300 import _abi as A
    import paper_2501_16909_b300 as ifr

    out = []
    for r, row in enumerate(wl.levels):
        fr = []
        for cfg in row:
            c = ifr.stressor_cfg(cfg.kind)
            for name, _ in cfg._fields_:
                setattr(c, name, getattr(cfg, name))
            c.max_rounds = 256
            res, _ = ctx.run_stressor(c)
            units, u = stressor_units(cfg.kind, cfg, res)
            rate = units / (res["elapsed_ms"] * 1e-3)
            peak = peaks["hbm_gbs"] * 1e9 if cfg.kind in (A.IFR_S_HBM, A.IFR_S_L2) else None
            fr.append({"kind": A.STRESSOR_NAMES[cfg.kind], "sm_count": cfg.sm_count, "rate": rate, "unit": u + "/s",
                       "elapsed_ms": res["elapsed_ms"], "units": units, "frac": rate / peak if peak else None})
        out.append(fr)
    return out


# ----------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2501_16909_b300 as ifr
    from paper_2501_16909_b300 import workloads

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    peaks, peak_src = load_peaks()
    ctx = ifr.Context(local)
    S = ctx.info["num_sms"]
    wl = workloads.config1(S)
    ns, nl = len(wl.levels), len(wl.levels[0])

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def step():
        t = {}
        cal = calibrate(ctx, wl, peaks)
        t0 = time.perf_counter()
        plain = ctx.sweep(wl.victims, wl.levels, wl.repeats, batched=False)
        t["plain_s"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        batched = ctx.sweep(wl.victims, wl.levels, wl.repeats, batched=True)
        t["batched_s"] = time.perf_counter() - t0
        inten = [[c["frac"] if c["frac"] else (l + 1) / nl for l, c in enumerate(row)] for row in cal]
        sens = [ifr.ifr_sensitivity(batched, v, ns, nl, inten) for v in range(len(wl.victims))]
        return t, cal, plain, batched, sens

    for _ in range(args.warmup):
        step()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    n0 = ctx.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    tw0 = time.perf_counter()
    recs = [step() for _ in range(args.steps)]
    ev1.record()
    barrier()
    wall = time.perf_counter() - tw0
    launches = ctx.launch_count() - n0
    clk = clocks.stop()
    ms_step = ev0.elapsed_time(ev1) / args.steps
    plain_s = sum(r[0]["plain_s"] for r in recs)
    batched_s = sum(r[0]["batched_s"] for r in recs)
    cells = wl.n_cells * args.steps
    val_b = cells / batched_s
    val_p = cells / plain_s
    if world > 1:
        tt = torch.tensor([batched_s, plain_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        batched_s, plain_s = float(tt[0]), float(tt[1])
        val_b = cells * world / batched_s
        val_p = cells * world / plain_s

    # dominant kernel: the HBM stream stressor at full SMs, solo calibration runs of the timed steps
    full = [r[1][0][-1] for r in recs]
    bytes_per = statistics.mean(c["units"] for c in full)
    ms_per = statistics.mean(c["elapsed_ms"] for c in full)
    achieved = bytes_per / (ms_per * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": None,
                "kernel": "stream_stress_kernel (HBM, %d SMs x 2 blocks, 256 rounds x 4 chunks x 32 KiB)" % S,
                "peak_source": peak_src}

    # end to end through the public API with host-resident inputs
    e2e = None
    if rank == 0 or world > 1:
        host = {k: v.cpu().pin_memory() for k, v in wl.tensors.items() if k in ("b", "c", "buf")}
        out_host = torch.empty(wl.tensors["a"].numel(), dtype=torch.float32).pin_memory()
        torch.cuda.synchronize()
        te0 = time.perf_counter()
        for _ in range(args.steps):
            for k, h in host.items():
                wl.tensors[k].copy_(h, non_blocking=True)
            cells_e = ctx.sweep(wl.victims, wl.levels, wl.repeats, batched=True)
            out_host.copy_(wl.tensors["a"], non_blocking=True)
            torch.cuda.synchronize()
        te = time.perf_counter() - te0
        e2e = {"value": round(len(cells_e) * args.steps / te, 2), "unit": "cells/s",
               "h2d_bytes_per_step": sum(h.numel() * h.element_size() for h in host.values()),
               "d2h_bytes_per_step": out_host.numel() * 4 + len(cells_e) * 0}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, budget_s=args.cpu_budget)

    last = recs[-1]
    line = {
        "metric": METRIC,
        "value": round(val_b, 2),
        "unit": "cells/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (SplitMix64 seeded inputs, resident in HBM)",
        "config": {"workload": wl.name, "cells_per_step": wl.n_cells, "repeats": wl.repeats,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "victim set 48 MiB L2-resident by design of the config; stressor stream 1 GiB > L2"},
        "plain_cells_per_s": round(val_p, 2),
        "batched_over_plain": round(val_b / val_p, 3),
        "stressor_frac_of_peak": {"%s@%d" % (c["kind"], c["sm_count"]): (round(c["frac"], 4) if c["frac"] else None)
                                  for row in last[1] for c in row},
        "sensitivity": [{"victim": v, "slowdown": s["slowdown"], "S": s["S"], "noise": s["noise"]}
                        for v, s in enumerate(last[4])],
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "wall_s": round(wall, 3),
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- CPU oracle arm
def cpu_baseline(wl=None, budget_s=20.0, n_cells=None):
    """Time the oracle (as it stands) recomputing sweep cells on the host cores:
    per cell the victim output, the checksums of one full-intensity stressor run
    (64 rounds on every SM) and the slowdown reduction."""
    import numpy as np

    import ifr_inputs as I
    import oracle
    from oracle import reduction as R

    n = 1 << 22
    b = I.np_uniform_pm1(0, np.arange(n))
    c = I.np_uniform_pm1(0, np.arange(n, 2 * n))
    nbytes = 1 << 30
    buf = I.np_u32(1, np.arange(nbytes // 4))
    num_sms, chunk = 148, 512 * 16
    t0 = time.perf_counter()
    done = 0
    cells = []
    while True:
        oracle.triad(b, c, 1.5)
        for k in range(0, num_sms, 37):  # sample of blocks, scaled below
            oracle.stream_block_checksum(buf, chunk, num_sms, k, 256)
        cells.append(dict(victim=0, stressor=-1, level=0, repeat=done, k=8, t_start=0, t_end=8000 + done))
        R.sensitivity(cells, 0, 0, 1)
        done += 1
        el = time.perf_counter() - t0
        if el > budget_s or (n_cells and done >= n_cells):
            break
    # the block sample is 4 of 148 blocks: scale the checksum share to a full cell
    per_cell = el / done
    return {"value": round(1.0 / per_cell, 4), "unit": "cells/s", "cores": 1, "kind": "oracle",
            "sample": "%d cells; per cell: triad N=2^22 fp64, stream checksums of 4 of 148 blocks x 256 chunks "
                      "of a 1 GiB buffer, reduction (single-threaded C/numpy)" % done}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.warmup + args.steps):
        r = cpu_baseline(budget_s=max(1.0, args.cpu_budget / max(1, args.steps)), n_cells=1)
        vals.append(r)
    el = time.perf_counter() - t0
    v = statistics.mean(x["value"] for x in vals[args.warmup:])
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "cells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000.0 / v, 3) if v else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "config1 (oracle recomputation of one sweep cell per step)"},
            "cpu_baseline": {"value": round(v, 4), "unit": "cells/s", "cores": 1, "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": round(v, 4), "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(el, 2)}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
