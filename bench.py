#!/usr/bin/env python
"""Benchmark: interference-sensitivity sweep on B300.

One step = one pass of the whole hot path over the workload:
  1. calibration — every stressor level alone, fixed work, CUDA events on the
     stressor stream -> achieved fraction of its resource's peak (the intensity x);
  2. the plain launch-per-cell sweep;
  3. the graph-captured batched sweep;
  4. the sensitivity reduction of every victim.
`value` is the batched sweep's cells/s (whole job, all ranks).  The plain sweep's
cells/s, each stressor's fraction of peak and the sensitivity vectors are
reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload config2|config1]

With --gpus N > 1 the script runs under torchrun, one process per GPU; each rank
sweeps its own replica of the workload (interference is a per-GPU quantity, so the
sweep shards with no collective on the data path).
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


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.path = index, None, None

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
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes (read + write) per launch of the roofline kernels, from the committed
# ncu captures of the same launch (file under profiles/ named beside each); an entry
# is removed when its kernel changes, so the line then reports null.
NCU_DRAM_BYTES = {
    "smem_32w": 19968,  # smem_32w_stressor_148sm.md
    "hbm": 2486113792,  # hbm_stream_stressor_1GiB_148sm.md (same blocks and rounds; set > L2)
    "gemm": 113009920,  # gemm_bf16_tcgen05_4096.md
}


def dist_env():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


# ----------------------------------------------------------------------------- our arm
def calibrate(ctx, wl, pk):
    """Every stressor level alone with fixed work: rate and fraction of peak."""
    from paper_2501_16909_b300 import _abi as A
    from paper_2501_16909_b300 import peaks as P

    out = []
    for row in wl.levels:
        fr = []
        for cfg in row:
            rate, res = P.solo_rate(ctx, cfg)
            peak = pk[cfg.kind][0]
            fr.append({"kind": A.STRESSOR_NAMES[cfg.kind], "sm_count": cfg.sm_count, "rate": rate,
                       "unit": P.UNIT[cfg.kind] + "/s", "elapsed_ms": res["elapsed_ms"],
                       "units": P.work_units(cfg, res), "frac": rate / peak if peak else None})
        out.append(fr)
    return out


def prepare_levels(ctx, wl, pk):
    """Scheduler launch counts and deadlines sized from solo victim windows: separate
    level tables for the plain (one victim per stressor run) and the batched (all
    victims under one stressor run) sweeps."""
    from paper_2501_16909_b300 import plan

    windows = plan.solo_windows(ctx, wl.victims)
    t_launch = plan.sched_launch_ns(ctx, wl.levels)
    plain, batched = plan.mode_levels(wl.levels, windows, t_launch)
    return plain, batched, windows, t_launch


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2501_16909_b300 as ifr
    from paper_2501_16909_b300 import _abi as A
    from paper_2501_16909_b300 import peaks as P
    from paper_2501_16909_b300 import workloads

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    ctx = ifr.Context(local)
    S = ctx.info["num_sms"]
    wl = workloads.config2(S) if args.workload == "config2" else workloads.config1(S)
    pk = P.peaks(ctx, wl.tensors.get("l2"))
    lv_plain, lv_batched, windows, t_launch = prepare_levels(ctx, wl, pk)
    ns, nl = len(wl.levels), len(wl.levels[0])

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def step():
        t = {}
        cal = calibrate(ctx, wl, pk)
        t0 = time.perf_counter()
        plain = ctx.sweep(wl.victims, lv_plain, wl.repeats, batched=False)
        t["plain_s"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        batched = ctx.sweep(wl.victims, lv_batched, wl.repeats, batched=True)
        t["batched_s"] = time.perf_counter() - t0
        inten = [[c["frac"] for c in row] for row in cal]
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
    if world > 1:
        from paper_2501_16909_b300 import replicas

        batched_s, plain_s = replicas.max_over_ranks([batched_s, plain_s], device="cuda")
    val_b = cells * world / batched_s
    val_p = cells * world / plain_s

    # per-stressor fraction of peak at full SMs (calibration runs of the timed steps)
    full = {}
    for r in range(ns):
        runs = [rec[1][r][-1] for rec in recs]
        kind = wl.levels[r][-1].kind
        units = statistics.mean(c["units"] for c in runs)
        ms = statistics.mean(c["elapsed_ms"] for c in runs)
        rate = units / (ms * 1e-3)
        full[A.STRESSOR_NAMES[kind]] = {"rate": rate, "unit": P.UNIT[kind] + "/s", "frac": rate / pk[kind][0],
                                        "peak": pk[kind][0], "peak_source": pk[kind][1], "ms": ms, "units": units}
    # GPU time by kernel in the timed plain sweeps (CUDA events around each stressor
    # run and each victim measurement): the dominant kernel gets the roofline
    busy = {}
    for rec in recs:
        for c in rec[2]:
            v = "victim:" + A.VICTIM_NAMES[wl.victim_kinds[c.victim]]
            busy[v] = busy.get(v, 0.0) + c.timing.event_ms
            if c.stressor >= 0 and c.level > 0:
                k = A.STRESSOR_NAMES[wl.levels[c.stressor][0].kind]
                busy[k] = busy.get(k, 0.0) + c.stress.elapsed_ms
    tot_busy = sum(busy.values())
    stress_busy = {k: v for k, v in busy.items() if not k.startswith("victim:")}
    dom = max(stress_busy, key=stress_busy.get) if stress_busy else "hbm"
    rl = {"hbm": ("hbm", 1e9, "GB/s", 1.0), "l2": ("l2", 1e9, "GB/s", 1.0), "fma": ("alu", 1e12, "TFLOP/s", 1.0),
          "tensor": ("tensor", 1e12, "TFLOP/s", 1.0), "smem_cf": ("smem", 1e9, "GB/s", 128.0),
          "smem_32w": ("smem", 1e9, "GB/s", 128.0), "sched": ("dispatch", 1e6, "Mblocks/s", 1.0)}
    bound, scale, unit, mult = rl[dom]
    fd = full[dom]
    dom_kind = A.STRESSOR_NAMES.index(dom)
    roofline = {"bound": bound, "achieved": round(fd["rate"] * mult / scale, 2),
                "peak": round(fd["peak"] * mult / scale, 2), "unit": unit, "frac": round(fd["frac"], 4),
                "traffic": NCU_DRAM_BYTES.get(dom),
                "kernel": "%s stressor at %d SMs (solo calibration runs of the timed steps: %d rounds)"
                          % (dom, S, P.CAL_ROUNDS[dom_kind]),
                "peak_source": fd["peak_source"] + " (of measured)" if "measured" in fd["peak_source"] else
                fd["peak_source"],
                "share_of_sweep_gpu_time": round(busy[dom] / tot_busy, 4)}
    hb = full.get("hbm")
    roofline_hbm = {"bound": "hbm", "achieved": round(hb["rate"] / 1e9, 1), "peak": round(pk[A.IFR_S_HBM][0] / 1e9, 1),
                    "unit": "GB/s", "frac": round(hb["frac"], 4), "traffic": NCU_DRAM_BYTES.get("hbm"),
                    "kernel": "stream_stress_kernel (HBM 4 GiB set, %d SMs x 2 blocks of 512, %d rounds x 4 chunks "
                              "x 32 KiB per block)" % (S, P.CAL_ROUNDS[A.IFR_S_HBM]),
                    "peak_source": pk[A.IFR_S_HBM][1]}

    # the tensor-bound victim: solo GEMM launches of the timed plain sweeps
    roofline_gemm = None
    if A.IFR_V_GEMM in wl.victim_kinds:
        gv = wl.victim_kinds.index(A.IFR_V_GEMM)
        prof = ctx.victim_profile(wl.victims[gv])
        solo = [c.timing for rec in recs for c in rec[2] if c.stressor < 0 and c.victim == gv]
        ms_launch = sum(t.event_ms for t in solo) / sum(t.repeats for t in solo)
        ach = prof["flops_per_launch"] / (ms_launch * 1e-3) / 1e12
        mp, msrc = P.measured_peaks()
        g = wl.victims[gv]
        roofline_gemm = {"bound": "tensor", "achieved": round(ach, 1), "peak": mp["bf16_tflops"],
                         "unit": "TFLOP/s", "frac": round(ach / mp["bf16_tflops"], 4),
                         "traffic": NCU_DRAM_BYTES.get("gemm"),
                         "kernel": "gemm_bf16_kernel<256> (BF16 %dx%dx%d, persistent, %d CTAs; solo launches of the "
                                   "timed plain sweeps)" % (g.m, g.n, g.k, prof["grid"]),
                         "peak_source": "MEASURED_PEAKS bf16_tflops (%s, burst)" % msrc,
                         "share_of_sweep_gpu_time": round(busy["victim:gemm"] / tot_busy, 4)}

    # end to end through the public API with host-resident inputs
    e2e = None
    host_keys = [k for k in ("gA", "gB", "vA", "vx", "lx", "sx", "hk", "l2", "hbm", "b", "c", "buf")
                 if k in wl.tensors]
    out_keys = [k for k in ("gC", "vy", "ly", "sy", "hb", "a") if k in wl.tensors]
    host = {k: wl.tensors[k].cpu().pin_memory() for k in host_keys}
    outs = {k: torch.empty(wl.tensors[k].shape, dtype=wl.tensors[k].dtype).pin_memory() for k in out_keys}
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    n_e = 0
    for _ in range(args.steps):
        for k, h in host.items():
            wl.tensors[k].copy_(h, non_blocking=True)
        cells_e = ctx.sweep(wl.victims, lv_batched, wl.repeats, batched=True)
        for k, o in outs.items():
            o.copy_(wl.tensors[k], non_blocking=True)
        torch.cuda.synchronize()
        n_e += len(cells_e)
    te = time.perf_counter() - te0
    e2e = {"value": round(n_e * world / te, 2), "unit": "cells/s",
           "h2d_bytes_per_step": sum(h.numel() * h.element_size() for h in host.values()),
           "d2h_bytes_per_step": sum(o.numel() * o.element_size() for o in outs.values())}

    # the learned part: measured pairs (configuration-3 victims x co-runner configurations),
    # trained by the library's MLP kernels; MAPE against held-out measured pairs
    pred = None
    if not args.no_predictor:
        from paper_2501_16909_b300 import train_predictor as TP

        tp0 = time.perf_counter()
        data = TP.collect(ctx, repeats=1, log=lambda *x: None)
        collect_s = time.perf_counter() - tp0
        ev = {s: TP.evaluate(ctx, data, s) for s in ("random", "unseen")}
        steps = sum(e["epochs"] * (e["train_pairs"] // 512) for e in ev.values())
        train_s = sum(e["train_s"] for e in ev.values())
        pred = {"pairs": int(len(data["y"])), "collect_s": round(collect_s, 2),
                "mape_random_split": ev["random"]["mlp_mape"], "baseline_mape_random_split": ev["random"]["baseline_mape"],
                "mape_unseen_corunners": ev["unseen"]["mlp_mape"],
                "baseline_mape_unseen_corunners": ev["unseen"]["baseline_mape"],
                "training_samples_per_s": round(steps * 512 / max(train_s, 1e-9), 1), "epochs": {
                    s: e["epochs"] for s, e in ev.items()}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(budget_s=args.cpu_budget)

    last = recs[-1]
    valid = sum(c.valid for c in last[3])
    hol = sum(1 for c in last[3] if c.status == A.IFR_ERR_HOL)
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
        "data": "synthetic (SplitMix64-seeded inputs resident in HBM)",
        "config": {"workload": wl.name, "cells_per_step": wl.n_cells, "repeats": wl.repeats,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2_between_iterations": "stressor streams (4 GiB HBM set) exceed L2; victims keep their own "
                                            "working sets, as the configuration defines them"},
        "plain_cells_per_s": round(val_p, 2),
        "batched_over_plain": round(val_b / val_p, 3),
        "stressor_frac_of_peak_full_sms": {k: round(v["frac"], 4) for k, v in full.items()},
        "stressor_peaks": {k: {"peak": v["peak"], "unit": v["unit"], "source": v["peak_source"]}
                           for k, v in full.items()},
        "levels_frac_of_peak": {A.STRESSOR_NAMES[wl.levels[r][0].kind]: [round(c["frac"], 4) for c in last[1][r]]
                                for r in range(ns)},
        "sensitivity": [{"victim": A.VICTIM_NAMES[wl.victim_kinds[v]], "S": [round(x, 4) for x in s["S"]],
                         "noise": round(s["noise"], 4)} for v, s in enumerate(last[4])],
        "cells_valid": valid, "cells_hol": hol, "cells_total": len(last[3]),
        "victim_solo_window_ns": windows, "sched_launch_ns": t_launch,
        "predictor": pred,
        "sweep_gpu_ms_by_kernel": {k: round(v, 2) for k, v in sorted(busy.items(), key=lambda x: -x[1])},
        "roofline": roofline,
        "roofline_hbm_stressor": roofline_hbm,
        "roofline_gemm_victim": roofline_gemm,
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


# ----------------------------------------------------------------------------- CPU oracle
def cpu_baseline(budget_s=20.0):
    """Time the oracle (as it stands, single thread) recomputing one sweep cell of the
    config-2 workload on the host: per victim a sample of its outputs (scaled to the
    full output), per stressor the checksums of 1 ms of its full-intensity work on B300
    (scaled from a sample of blocks), and the reduction.  Each of the 11 parts repeats
    its sample for an equal share of `budget_s` seconds and is timed per repetition.
    Returns cells/s."""
    import numpy as np

    import ifr_inputs as I
    import oracle
    from oracle import reduction as R

    t_start = time.perf_counter()
    rng = np.random.default_rng(0)
    per = {}

    share = budget_s / 11.0
    reps = {}

    def timed(fn, scale):
        t0 = time.perf_counter()
        n = 0
        while True:
            fn()
            n += 1
            el = time.perf_counter() - t0
            if el >= share:
                break
        reps[len(reps)] = n
        return el / n * scale

    G, RR = 4096, 8192
    gA = oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(11, np.arange(64 * G))).reshape(64, G)
    gB = oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(12, np.arange(64 * G))).reshape(64, G)
    ij = np.stack([rng.integers(0, 64, 256), rng.integers(0, 64, 256)], axis=1)
    per["gemm"] = timed(lambda: oracle.gemm_entries(gA, gB, ij), G * G / 256)
    vA = oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(13, np.arange(64 * RR))).reshape(64, RR)
    vx = oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(14, np.arange(RR)))
    per["gemv"] = timed(lambda: oracle.gemv_rows(vA, vx, np.arange(64)), RR / 64)
    lx = I.np_uniform_pm1(15, np.arange(64 * 4096)).reshape(64, 4096)
    per["layernorm"] = timed(lambda: oracle.layernorm_rows(lx, np.arange(64)), 16384 / 64)
    sx = I.np_uniform_pm1(16, np.arange(16 * RR)).reshape(16, RR)
    per["softmax"] = timed(lambda: oracle.softmax_rows(sx, np.arange(16)), RR / 16)
    keys = I.np_key256(2, np.arange(1 << 22))
    per["hist"] = timed(lambda: oracle.histogram(keys), 16)
    # stressors: 1 ms of full-intensity work on B300 (measured rates, rounded)
    buf = I.np_u32(1, np.arange(1 << 22))
    per["stream"] = timed(lambda: oracle.stream_block_checksum(buf, 8192, 1, 0, 512), 6.5e9 / (512 * 32768))
    per["fma"] = timed(lambda: oracle.fma_block(1, 0, 128, 4, 4096, 1), 7.6e13 / 2 / (128 * 4 * 4096))
    per["tensor"] = timed(lambda: oracle.tensor_block(1, 0, 64), 148.0)  # closed form per block: one tile product
    per["smem"] = timed(lambda: oracle.smem_block(1, 0, 8, 8, 8), 3.0e8 / (8 * 8 * 8 * 32 * 2))
    per["sched"] = timed(lambda: oracle.sched_checksum(1, 100000, 16), 30.0)
    cells = [dict(victim=0, stressor=-1, level=0, repeat=i, k=4, t_start=0, t_end=4000 + i) for i in range(3)]
    per["reduction"] = timed(lambda: R.sensitivity(cells, 0, 0, 1), 1.0)
    victim_s = statistics.mean(per[k] for k in ("gemm", "gemv", "layernorm", "softmax", "hist"))
    stress_s = statistics.mean(per[k] for k in ("stream", "fma", "tensor", "smem", "sched"))
    sec_per_cell = victim_s + stress_s + per["reduction"]
    el = time.perf_counter() - t_start
    return {"value": round(1.0 / sec_per_cell, 5), "unit": "cells/s", "cores": 1, "kind": "oracle",
            "sample": "one config-2 cell estimated from samples (GEMM 256 of 16.8M entries, GEMV 64 rows, LN 64 rows, "
                      "softmax 16 rows, histogram 2^22 of 2^26 keys, 1 ms of each stressor's B300 work scaled from "
                      "one block), each sample repeated for %.1f s (%d-%d repetitions); seconds per full cell %.1f; "
                      "sampling took %.1f s" % (share, min(reps.values()), max(reps.values()), sec_per_cell, el),
            "seconds_per_component": {k: round(v, 3) for k, v in per.items()}}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    vals = []
    t0 = time.perf_counter()
    # the whole --steps/--warmup run stays within about two and a half minutes
    budget = min(args.cpu_budget, 150.0 / max(1, args.warmup + args.steps))
    for _ in range(args.warmup + args.steps):
        vals.append(cpu_baseline(budget_s=budget))
    el = time.perf_counter() - t0
    timed = vals[args.warmup:]
    v = statistics.mean(x["value"] for x in timed)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": "cells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000.0 / v, 1) if v else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "config2 (oracle recomputation of one sweep cell per step, sampled)"},
            "cpu_baseline": {"value": round(v, 5), "unit": "cells/s", "cores": 1, "kind": "oracle",
                             "sample": timed[-1]["sample"]},
            "e2e": {"value": round(v, 5), "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(el, 2)}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="config2", choices=["config2", "config1"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-predictor", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
