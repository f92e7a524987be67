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


# DRAM bytes (read + write) per launch of the roofline kernels from ncu captures of
# the same launch shape, each with the SHA-256 of the files that define the launch at
# capture time (the kernel's source; for the stressors also the module that sets
# their shapes); when one of them has changed since, the line reports null instead.
# Captured with `ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum
# --clock-control none -k regex:<kernel> -c 1 python -m paper_2501_16909_b300.profile_case
# <case>` (cases sched, fma, tensor, smem_cf, smem_32w, l2, hbm, `hbm --staging 1`,
# `gemm --variant {0,2,3}`), after the same command ran clean; the stressors' shapes
# and rounds are those of the solo runs below, the GEMM is the same 4096^3 launch.
_GEMM_SRC = ((("paper_2501_16909_b300/csrc/ifr_gemm.cu",
               "d8eaf3b43e508a20b818daf30899f1ee96a391382bc47b48f399e40fd35408bb"),),)
_STRESS_SRC = ((("paper_2501_16909_b300/csrc/ifr_stressors.cu",
                 "48212933b9817087877f2b6920a820d95c637c710ff0d5fa102e800e58ad713f"),
                ("paper_2501_16909_b300/workloads.py",
                 "1745acd7eabd2e2a5e4d5cbf6edecfb64f956ed8117fbc55fdcfd96fe2f01ad4")),)
NCU_DRAM_BYTES = {
    "sched": (4608 + 0,) + _STRESS_SRC,
    "fma": (20480 + 0,) + _STRESS_SRC,
    "tensor": (47616 + 0,) + _STRESS_SRC,
    "smem_cf": (17152 + 0,) + _STRESS_SRC,
    "smem_32w": (18944 + 0,) + _STRESS_SRC,
    "l2": (16795904 + 0,) + _STRESS_SRC,
    "hbm": (2483070208 + 2708736,) + _STRESS_SRC,
    "hbm_tma": (2502471424 + 3041024,) + _STRESS_SRC,
    "gemm": (75722496 + 35376896,) + _GEMM_SRC,
    "gemm_v2": (77870080 + 40004608,) + _GEMM_SRC,
    "gemm_v3": (76908032 + 41671168,) + _GEMM_SRC,
}


def _src_sha(rel):
    import hashlib

    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def ncu_traffic(name):
    """DRAM bytes per launch of `name` from its capture, or None when stale or absent."""
    e = NCU_DRAM_BYTES.get(name)
    if not e:
        return None
    nbytes, srcs = e
    return nbytes if all(_src_sha(f) == h for f, h in srcs) else None


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
                "traffic": ncu_traffic(dom),
                "kernel": "%s stressor at %d SMs (solo calibration runs of the timed steps: %d rounds)"
                          % (dom, S, P.CAL_ROUNDS[dom_kind]),
                "peak_source": fd["peak_source"] + " (of measured)" if "measured" in fd["peak_source"] else
                fd["peak_source"],
                "share_of_sweep_gpu_time": round(busy[dom] / tot_busy, 4)}
    hb = full.get("hbm")
    roofline_hbm = {"bound": "hbm", "achieved": round(hb["rate"] / 1e9, 1), "peak": round(pk[A.IFR_S_HBM][0] / 1e9, 1),
                    "unit": "GB/s", "frac": round(hb["frac"], 4), "traffic": ncu_traffic("hbm"),
                    "kernel": "stream_stress_kernel (HBM 4 GiB set, %d SMs x 2 blocks of 512, %d rounds x 8 chunks "
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
                         "traffic": ncu_traffic("gemm"),
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


def cpu_info():
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count() or 1
    return {"nproc": os.cpu_count() or 1, "usable": usable, "model": model}


def _threads_wall(fn, n_threads, reps):
    """Wall time of n_threads concurrent copies of `reps` calls of fn (the oracle's C
    calls release the GIL, so the copies run on separate cores)."""
    import concurrent.futures as cf

    def work():
        for _ in range(reps):
            fn()

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=n_threads) as ex:
        for f in [ex.submit(work) for _ in range(n_threads)]:
            f.result()
    return time.perf_counter() - t0


def oracle_unit_costs(share_s, threads):
    """Seconds per unit of oracle work, single-threaded and as an all-cores throughput
    (threads concurrent copies), each timed on a sample for about share_s seconds:
    stream chunk (32 KiB, first word of every 16 bytes folded), FMA (one fp32 fmaf),
    tensor block (closed form of one block's tile products), shared-memory block (one
    256-thread block's words through 1024 LCG steps), scheduler block, GEMM and GEMV
    multiply-adds, layernorm and softmax elements."""
    import numpy as np

    import ifr_inputs as I
    import oracle

    buf = I.np_u32(1, np.arange(1 << 22))
    gA = oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(11, np.arange(64 * 4096))).reshape(64, 4096)
    gB = oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(12, np.arange(64 * 4096))).reshape(64, 4096)
    ij = np.stack([np.arange(64), np.arange(64)[::-1]], axis=1)
    x4 = I.np_uniform_pm1(15, np.arange(16 * 4096)).reshape(16, 4096)
    xb = oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(14, np.arange(4096)))
    samples = {
        "stream_chunk": (lambda: oracle.stream_block_checksum(buf, 8192, 1, 0, 256), 256),
        "fma": (lambda: oracle.fma_block(1, 0, 32, 4, 1024, 4), 32 * 4 * 1024 * 4),
        "tensor_block": (lambda: oracle.tensor_block(1, 0, 64), 1),
        "smem_block": (lambda: oracle.smem_block(1, 0, 8, 32, 32), 1),
        "sched_block": (lambda: oracle.sched_checksum(1, 100000, 16), 100000),
        "gemm_mac": (lambda: oracle.gemm_entries(gA, gB, ij), 64 * 4096),
        "gemv_mac": (lambda: oracle.gemv_rows(gA, xb, np.arange(64)), 64 * 4096),
        "layernorm_elem": (lambda: oracle.layernorm_rows(x4, np.arange(16)), 16 * 4096),
        "softmax_elem": (lambda: oracle.softmax_rows(x4, np.arange(16)), 16 * 4096),
    }
    one, many = {}, {}
    for name, (fn, units) in samples.items():
        t0 = time.perf_counter()
        n = 0
        while True:
            fn()
            n += 1
            if time.perf_counter() - t0 >= share_s:
                break
        one[name] = (time.perf_counter() - t0) / (n * units)
        reps = max(1, n // 2)
        many[name] = _threads_wall(fn, threads, reps) / (threads * reps * units)
    return one, many


def _cell_cost(c, kind_name, vshape, cost, block_of):
    """Oracle seconds for one measured cell: the victim's whole output, the stressor's
    checksums over the work the GPU reported for that cell, and nothing for the
    reduction (timed separately)."""
    kind, a, b, k = vshape
    if kind == "gemm":
        v = a * b * k * cost["gemm_mac"]
    elif kind == "gemv":
        v = a * k * cost["gemv_mac"]
    else:
        v = a * b * cost[kind + "_elem"]
    st = 0.0
    if c.stressor >= 0 and c.level > 0:
        w, blocks = c.stress.work, max(1, c.stress.blocks_active)
        if kind_name in ("hbm", "l2"):
            st = w * cost["stream_chunk"]
        elif kind_name == "fma":
            st = w * block_of["fma"] * 8 * cost["fma"]  # steps per chain x threads x 8 chains
        elif kind_name == "tensor":
            st = blocks * cost["tensor_block"]
        elif kind_name in ("smem_cf", "smem_32w"):
            st = w / (32 * 32 * 32) * cost["smem_block"]  # the sample block did 32 rounds x 32 passes x 32 pairs
        elif kind_name == "sched":
            st = w * cost["sched_block"]
    return v + st


def direct_cell(cell, vshape, seed, hbm_words, threads):
    """One complete configuration-3 cell recomputed by the oracle: every row of a GEMV
    victim and the checksum of every active HBM-stressor block over the chunks the GPU
    reported (the cell's total split evenly over its blocks).  Only the chunks read
    are generated.  Returns (seconds on 1 thread, seconds on `threads` threads)."""
    import concurrent.futures as cf

    import numpy as np

    import ifr_inputs as I
    import oracle

    _, R, _, W = vshape
    A_ = oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(seed, np.arange(R * W))).reshape(R, W)
    x = oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(seed + 1, np.arange(W)))
    chunk = 512 * 16
    n_chunks = hbm_words // chunk
    planned = max(1, cell.stress.planned_active)
    active = max(1, cell.stress.blocks_active)
    total = int(cell.stress.work)
    counts = [total // active + (1 if b < total % active else 0) for b in range(active)]
    buf = np.zeros(hbm_words, np.uint32)  # untouched pages stay unallocated
    need = set()
    for k, cnt in enumerate(counts):
        m_k = (n_chunks - k + planned - 1) // planned
        for j in range(min(cnt, m_k)):
            need.add(k + j * planned)
    for c in need:
        buf[c * chunk:(c + 1) * chunk] = I.np_u32(1, np.arange(c * chunk, (c + 1) * chunk))
    rows = np.arange(R)

    def blocks_part(ks):
        for k in ks:
            if counts[k]:
                oracle.stream_block_checksum(buf, chunk, planned, k, counts[k], oracle.FOLD_LOADS)

    t0 = time.perf_counter()
    oracle.gemv_rows(A_, x, rows)
    blocks_part(range(active))
    one = time.perf_counter() - t0
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        futs = [ex.submit(oracle.gemv_rows, A_, x, part) for part in np.array_split(rows, threads)]
        futs += [ex.submit(blocks_part, range(t, active, threads)) for t in range(threads)]
        for f in futs:
            f.result()
    many = time.perf_counter() - t0
    return one, many, {"victim_rows": R, "stressor_blocks": active, "stressor_chunks": total,
                       "chunks_generated": len(need)}


def cpu_baseline_config3(budget_s, cells, victims_t=None, bufs=None):
    """The oracle as it stands, timed on this host's cores, for configuration-3 cells.

    * `value` (an estimate, single thread): the oracle's seconds for the average cell
      of the last timed plain sweep: each cell's victim output recomputed whole, and
      its stressor's checksums over the work the GPU reported for that cell, at
      per-unit costs timed on samples; plus the reduction.
    * `all_cores`: the same with the per-unit costs of `usable` concurrent copies.
    * `direct_cell`: one complete cell (a GEMV victim beside the HBM stressor at its
      top level) recomputed end to end, timed, on 1 thread and on all cores."""
    import numpy as np

    from oracle import reduction as R
    import paper_2501_16909_b300 as ifr
    from paper_2501_16909_b300 import _abi as A
    from paper_2501_16909_b300 import workloads as W

    info = cpu_info()
    threads = info["usable"]
    t_start = time.perf_counter()
    one, many = oracle_unit_costs(budget_s / 12.0, threads)
    shapes = W.config3_shapes()
    names = [A.STRESSOR_NAMES[k] for k in (A.IFR_S_SCHED, A.IFR_S_FMA, A.IFR_S_TENSOR, A.IFR_S_SMEM_CF,
                                           A.IFR_S_SMEM_32W, A.IFR_S_L2, A.IFR_S_HBM)]
    block_of = {"fma": 128}
    s1 = [_cell_cost(c, names[c.stressor] if c.stressor >= 0 else "", shapes[c.victim], one, block_of) for c in cells]
    sN = [_cell_cost(c, names[c.stressor] if c.stressor >= 0 else "", shapes[c.victim], many, block_of) for c in cells]
    d = ifr.cells_to_dicts(cells)
    t0 = time.perf_counter()
    for v in range(len(shapes)):
        R.sensitivity(d, v, 7, 8)
    red = (time.perf_counter() - t0) / max(1, len(cells))
    sec1 = float(np.mean(s1)) + red
    secN = float(np.mean(sN)) + red
    # the complete cell: the smallest GEMV victim beside the HBM stressor at its top level
    gv = min((i for i, sh in enumerate(shapes) if sh[0] == "gemv"), key=lambda i: shapes[i][1])
    cell = next(c for c in cells if c.victim == gv and c.stressor == 6 and c.level == 8)
    d1, dN, what = direct_cell(cell, shapes[gv], W.config3_seeds(gv), 1 << 30, threads)
    el = time.perf_counter() - t_start
    return {"value": round(1.0 / sec1, 5), "unit": "cells/s", "cores": 1, "kind": "oracle",
            "estimate": True,
            "sample": "estimate for the %d cells of one configuration-3 plain sweep: per cell the victim output "
                      "recomputed whole and the stressor checksums over the work the GPU measured for that cell, "
                      "at per-unit oracle costs timed on samples (%.1f s each); seconds per average cell %.3g; "
                      "sampling took %.1f s" % (len(cells), budget_s / 12.0, sec1, el),
            "all_cores": {"value": round(1.0 / secN, 5), "cores": threads, "seconds_per_cell": round(secN, 6)},
            "direct_cell": {"cell": "GEMV victim %d (%d x %d) beside the HBM stressor at its top level, one "
                                    "measurement" % (gv, shapes[gv][1], shapes[gv][3]),
                            "seconds_1_thread": round(d1, 4), "seconds_all_cores": round(dN, 4), "cores": threads,
                            **what},
            "cpu": info, "unit_costs_ns_1_thread": {k: round(v * 1e9, 4) for k, v in one.items()}}


def run_reference(args):
    """The oracle as it stands, on this host's cores, recomputing configuration-3
    cells: each step recomputes one complete cell (a GEMV victim beside the HBM
    stressor; the stressor's work set to what it streams in the victim's window at
    the measured HBM rate, since this arm runs no GPU) on one thread and on all
    cores.  The line's value is cells/s on one thread."""
    world, rank, _ = dist_env()
    if rank != 0:
        return

    from paper_2501_16909_b300 import workloads as W
    from paper_2501_16909_b300 import peaks as P

    class _Stress:
        pass

    class _Cell:
        pass

    shapes = W.config3_shapes()
    gv = min((i for i, sh in enumerate(shapes) if sh[0] == "gemv"), key=lambda i: shapes[i][1])
    _, R, _, Wd = shapes[gv]
    mp, msrc = P.measured_peaks()
    hbm = mp["hbm_gbs"] * 1e9
    window_s = 2.0 * R * Wd / hbm + 20e-6  # the victim's bytes at the HBM rate, plus the harness
    cell = _Cell()
    cell.stress = _Stress()
    cell.stress.planned_active = cell.stress.blocks_active = 296
    cell.stress.work = int(window_s * hbm / 32768)
    info = cpu_info()
    vals, alls = [], []
    t0 = time.perf_counter()
    for _ in range(args.warmup + args.steps):
        d1, dN, what = direct_cell(cell, shapes[gv], W.config3_seeds(gv), 1 << 30, info["usable"])
        vals.append(1.0 / d1)
        alls.append(1.0 / dN)
    el = time.perf_counter() - t0
    v = statistics.mean(vals[args.warmup:])
    vN = statistics.mean(alls[args.warmup:])
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "cells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000.0 / v, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "config3 (oracle recomputation of one complete cell per step: GEMV victim %d "
                                   "(%d x %d) beside the HBM stressor at all SMs)" % (gv, R, Wd)},
            "cpu_baseline": {"value": round(v, 4), "unit": "cells/s", "cores": 1, "kind": "oracle",
                             "sample": "one complete configuration-3 cell per step: every GEMV row and every HBM "
                                       "stressor block's checksum over %d chunks (the victim's window at %s "
                                       "hbm_gbs)" % (cell.stress.work, msrc),
                             "all_cores": {"value": round(vN, 4), "cores": info["usable"]}, "cpu": info, **what},
            "e2e": {"value": round(v, 4), "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(el, 2)}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- configuration 3
def _full_stressor_levels(S, bufs):
    """Full-SM configuration of every stressor kind, as the sweeps use them."""
    from paper_2501_16909_b300 import workloads as W

    return W.config3_base_stressors(S, bufs)


def solo_kernel_rooflines(ctx, bufs, pk):
    """Untimed solo measurements behind the roofline objects: every stressor kind at
    all SMs (fixed work, CUDA events on the stressor stream), the HBM stressor with
    both load paths, and the BF16 GEMM at 4096^3 in its sweep variant (0), its CTA-pair
    throughput variant (2) and its single-CTA two-accumulator variant (3), 20 launches
    each after 3 warm ones (CUDA events on the victim stream)."""
    import torch

    import ifr_inputs as I
    import paper_2501_16909_b300 as ifr
    from paper_2501_16909_b300 import _abi as A
    from paper_2501_16909_b300 import peaks as P

    S = ctx.info["num_sms"]
    out = {"stressors": {}, "gemm": {}}
    for cfg in _full_stressor_levels(S, bufs):
        runs = [P.solo_rate(ctx, cfg) for _ in range(3)]
        rate = max(r for r, _ in runs)
        res = runs[0][1]
        out["stressors"][A.STRESSOR_NAMES[cfg.kind]] = {
            "rate": rate, "unit": P.UNIT[cfg.kind] + "/s", "frac": rate / pk[cfg.kind][0], "peak": pk[cfg.kind][0],
            "peak_source": pk[cfg.kind][1], "ms": res["elapsed_ms"], "units": P.work_units(cfg, res)}
    hb = P.copy_cfg(_full_stressor_levels(S, bufs)[-1], staging=1)
    rate, res = max((P.solo_rate(ctx, hb) for _ in range(3)), key=lambda x: x[0])
    out["stressors"]["hbm_tma"] = {"rate": rate, "unit": "B/s", "frac": rate / pk[A.IFR_S_HBM][0],
                                   "peak": pk[A.IFR_S_HBM][0], "peak_source": pk[A.IFR_S_HBM][1],
                                   "ms": res["elapsed_ms"], "units": P.work_units(hb, res)}
    G = 4096
    ga = I.torch_normal_bf16(11, G * G, "cuda").view(G, G)
    gb = I.torch_normal_bf16(12, G * G, "cuda").view(G, G)
    gc = torch.empty(G, G, device="cuda")
    for var in (0, 2, 3):
        cfg = ifr.victim_cfg(A.IFR_V_GEMM, ga, gb, gc, m=G, n=G, k=G, repeats=3, variant=var)
        ctx.victim_launch(cfg)
        cfg.repeats = 20
        t = ctx.victim_launch(cfg)
        prof = ctx.victim_profile(cfg)
        out["gemm"][var] = {"tflops": prof["flops_per_launch"] * 20 / (t["event_ms"] * 1e-3) / 1e12,
                            "ms_per_launch": t["event_ms"] / 20, "grid": prof["grid"], "status": t["status"]}
    del ga, gb, gc
    return out


def invalid_cells(cells, base, vkinds, A, cap=8):
    """The first `cap` cells that fail the constant-interference rule, each with the
    part of the rule it failed: the victim's or the stressor's own status, a stressor
    with no active block, a stressor block that started after the victim's first
    block, or one that ended before the victim's last block."""
    out = []
    for c in cells:
        if c.valid:
            continue
        t, s = c.timing, c.stress
        if t.status != 0:
            why = "victim status %d" % t.status
        elif s.status != 0:
            why = "stressor status %d" % s.status
        elif s.blocks_active <= 0:
            why = "no active stressor block"
        elif s.t_start_last_ns > t.t_start_ns:
            why = "stressor block started %.1f us after the victim" % ((s.t_start_last_ns - t.t_start_ns) / 1e3)
        else:
            why = "stressor block ended %.1f us before the victim" % ((t.t_end_ns - s.t_end_first_ns) / 1e3)
            if base[c.stressor].kind == A.IFR_S_SCHED:
                # blocks that worked: those on allowed SMs that started before the stop
                # request, so a chain that ran out before the victim ended shows no idle tail
                why += " (%d of %d launched blocks worked)" % (s.work, s.blocks_launched)
        out.append({"victim": int(c.victim), "victim_kind": A.VICTIM_NAMES[vkinds[c.victim]],
                    "stressor": A.STRESSOR_NAMES[base[c.stressor].kind] if c.stressor >= 0 else None,
                    "level": int(c.level), "reason": why})
        if len(out) >= cap:
            break
    return out


def run_config3(args):
    """Configuration 3 (the workload the batched-vs-plain metric is defined on): 64
    victims of uneven shapes x 7 stressor kinds x 8 autotuned intensities + level 0.
    One step = autotuning every stressor's levels, the graph-batched sweep, the same
    sweep with grouped persistent victims, the plain launch-per-cell sweep and the
    sensitivity reduction of every victim."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import ifr_inputs as I
    import paper_2501_16909_b300 as ifr
    from paper_2501_16909_b300 import _abi as A
    from paper_2501_16909_b300 import autotune, plan
    from paper_2501_16909_b300 import peaks as P
    from paper_2501_16909_b300 import workloads as W

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    ctx = ifr.Context(local)
    S = ctx.info["num_sms"]
    bufs = {"l2": I.torch_u32_as_i32(3, W.L2_SET_BYTES // 4, "cuda"), "hbm": I.torch_u32_as_i32(1, (4 << 30) // 4, "cuda")}
    victims, vkinds, vt = W.config3_victims("cuda")
    pk = P.peaks(ctx, bufs["l2"])
    base = W.config3_base_stressors(S, bufs)
    n_levels, repeats = 8, 1
    fr = [(l + 1) / n_levels for l in range(n_levels)]
    ns, nv = len(base), len(victims)
    cells_per_sweep = repeats * nv * (1 + ns * (n_levels + 1))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def step():
        t = {}
        t0 = time.perf_counter()
        levels, report = autotune.tuned_levels(ctx, base, pk, fr)
        t["autotune_s"] = time.perf_counter() - t0
        windows = plan.solo_windows(ctx, victims)
        t_launch = plan.sched_launch_ns(ctx, levels)
        lv_plain, lv_batched = plan.mode_levels(levels, windows, t_launch)
        t0 = time.perf_counter()
        cb = ctx.sweep(victims, lv_batched, repeats, batched=True)
        t["batched_s"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        cg = ctx.sweep(victims, lv_batched, repeats, batched=True, grouped=True)
        t["grouped_s"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        cp = ctx.sweep(victims, lv_plain, repeats, batched=False)
        t["plain_s"] = time.perf_counter() - t0
        inten = [[lv["frac_of_peak"] for lv in r["levels"]] for r in report]
        sens = [ifr.ifr_sensitivity(cb, v, ns, n_levels, inten) for v in range(nv)]
        return t, report, cb, cp, sens, lv_batched, cg

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
    batched_s = sum(r[0]["batched_s"] for r in recs)
    grouped_s = sum(r[0]["grouped_s"] for r in recs)
    plain_s = sum(r[0]["plain_s"] for r in recs)
    tune_s = sum(r[0]["autotune_s"] for r in recs)
    if world > 1:
        from paper_2501_16909_b300 import replicas

        batched_s, grouped_s, plain_s = replicas.max_over_ranks([batched_s, grouped_s, plain_s], device="cuda")
    cells = cells_per_sweep * args.steps
    val_b = cells * world / batched_s
    val_g = cells * world / grouped_s
    val_p = cells * world / plain_s

    # GPU time by kernel kind in the timed plain sweeps: the dominant kernel gets the roofline
    busy = {}
    for rec in recs:
        for c in rec[3]:
            v = "victim:" + A.VICTIM_NAMES[vkinds[c.victim]]
            busy[v] = busy.get(v, 0.0) + c.timing.event_ms
            if c.stressor >= 0 and c.level > 0:
                k = A.STRESSOR_NAMES[base[c.stressor].kind]
                busy[k] = busy.get(k, 0.0) + c.stress.elapsed_ms
    tot_busy = sum(busy.values())

    solo = solo_kernel_rooflines(ctx, bufs, pk)
    stress_busy = {k: v for k, v in busy.items() if not k.startswith("victim:")}
    dom = max(stress_busy, key=stress_busy.get)
    rl = {"hbm": ("hbm", 1e9, "GB/s", 1.0), "l2": ("l2", 1e9, "GB/s", 1.0), "fma": ("alu", 1e12, "TFLOP/s", 1.0),
          "tensor": ("tensor", 1e12, "TFLOP/s", 1.0), "smem_cf": ("smem", 1e9, "GB/s", 128.0),
          "smem_32w": ("smem", 1e9, "GB/s", 128.0), "sched": ("dispatch", 1e6, "Mblocks/s", 1.0)}
    bound, scale, unit, mult = rl[dom]
    fd = solo["stressors"][dom]
    roofline = {"bound": bound, "achieved": round(fd["rate"] * mult / scale, 2),
                "peak": round(fd["peak"] * mult / scale, 2), "unit": unit, "frac": round(fd["frac"], 4),
                "traffic": ncu_traffic(dom),
                "kernel": "%s stressor at %d SMs (solo, fixed work, %d rounds, best of 3)"
                          % (dom, S, P.CAL_ROUNDS[A.STRESSOR_NAMES.index(dom)]),
                "peak_source": fd["peak_source"] + (" (of measured)" if "measured" in fd["peak_source"] else ""),
                "share_of_sweep_gpu_time": round(busy[dom] / tot_busy, 4)}
    hb = solo["stressors"]["hbm"]
    mp, msrc = P.measured_peaks()
    roofline_hbm = {"bound": "hbm", "achieved": round(hb["rate"] / 1e9, 1), "peak": round(hb["peak"] / 1e9, 1),
                    "unit": "GB/s", "frac": round(hb["frac"], 4), "traffic": ncu_traffic("hbm"),
                    "kernel": "stream_stress_kernel (word loads 16 B apart, whole sectors; HBM 4 GiB set, %d SMs x 2 blocks of 512, "
                              "%d rounds x %d chunks x 32 KiB per block)" % (S, P.CAL_ROUNDS[A.IFR_S_HBM],
                                                                          P.STREAM_CHUNKS_PER_ROUND),
                    "peak_source": hb["peak_source"] + " (of measured)",
                    "tma_staging": {"achieved": round(solo["stressors"]["hbm_tma"]["rate"] / 1e9, 1),
                                    "frac": round(solo["stressors"]["hbm_tma"]["frac"], 4),
                                    "traffic": ncu_traffic("hbm_tma")}}
    g0, g2, g3 = solo["gemm"][0], solo["gemm"][2], solo["gemm"][3]
    roofline_gemm = {"bound": "tensor", "achieved": round(g0["tflops"], 1), "peak": mp["bf16_tflops"],
                     "unit": "TFLOP/s", "frac": round(g0["tflops"] / mp["bf16_tflops"], 4),
                     "traffic": ncu_traffic("gemm"),
                     "kernel": "gemm_bf16_kernel<256, 3, 1> (variant 0, the sweeps' GEMM: BF16 4096^3, persistent, "
                               "%d CTAs; 20 solo launches)" % g0["grid"],
                     "peak_source": "MEASURED_PEAKS bf16_tflops (%s, burst)" % msrc,
                     "throughput_variant": {"variant": 2, "achieved": round(g2["tflops"], 1),
                                            "frac": round(g2["tflops"] / mp["bf16_tflops"], 4),
                                            "traffic": ncu_traffic("gemm_v2"),
                                            "kernel": "gemm_bf16_pair_kernel<6, 2, split> (256 x 256 tiles on CTA "
                                                      "pairs, two TMEM accumulators, split last wave; %d CTAs)"
                                                      % g2["grid"]},
                     "single_cta_variant": {"variant": 3, "achieved": round(g3["tflops"], 1),
                                            "frac": round(g3["tflops"] / mp["bf16_tflops"], 4),
                                            "traffic": ncu_traffic("gemm_v3"),
                                            "kernel": "gemm_bf16_kernel<256, 4, 2> (two TMEM accumulators, split "
                                                      "last wave; %d CTAs)" % g3["grid"]}}

    # end to end through the public API: every input of the step copied in from pinned
    # host memory and every output read back inside the timed region
    ins, outs_dev = [], []
    for i in sorted(vt):
        ins.extend(vt[i][:-1])
        outs_dev.append(vt[i][-1])
    ins.extend([bufs["l2"], bufs["hbm"]])
    host_in = [x.cpu().pin_memory() for x in ins]
    host_out = [torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs_dev]
    lv_b = recs[-1][5]
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    n_e = 0
    for _ in range(args.steps):
        for d_, h_ in zip(ins, host_in):
            d_.copy_(h_, non_blocking=True)
        ce = ctx.sweep(victims, lv_b, repeats, batched=True)
        for d_, h_ in zip(outs_dev, host_out):
            h_.copy_(d_, non_blocking=True)
        torch.cuda.synchronize()
        n_e += len(ce)
    te = time.perf_counter() - te0
    e2e = {"value": round(n_e * world / te, 2), "unit": "cells/s",
           "h2d_bytes_per_step": sum(h.numel() * h.element_size() for h in host_in),
           "d2h_bytes_per_step": sum(h.numel() * h.element_size() for h in host_out)}

    pred = None
    if not args.no_predictor:
        from paper_2501_16909_b300 import train_predictor as TP

        tp0 = time.perf_counter()
        data = TP.collect(ctx, repeats=1, log=lambda *x: None)
        collect_s = time.perf_counter() - tp0
        ev = {sp: TP.evaluate(ctx, data, sp) for sp in TP.SPLITS}
        pred = {"pairs": int(len(data["y"])), "collect_s": round(collect_s, 2),
                "features": "measured solo profiles (see the predictor module)"}
        for sp, e in ev.items():
            pred["mape_" + sp] = e["mlp_mape"]
            pred["baseline_mape_" + sp] = e["baseline_mape"]
        pred["mape_by_held_out_kind"] = ev["kind"]["mlp_mape_by_held_out_kind"]
        steps_ = sum(e["epochs"] * (e["train_pairs"] // 512) for e in ev.values())
        pred["training_samples_per_s"] = round(steps_ * 512 / max(sum(e["train_s"] for e in ev.values()), 1e-9), 1)
        # configuration 5: decoder-layer kernel pairs scored by a 3-member ensemble trained on
        # these pairs plus kernel pairs, against their measured co-run slowdowns
        from paper_2501_16909_b300 import colocate_config5 as C5

        t5 = time.perf_counter()
        c5 = C5.score(ctx, data, repeats=2, members=3, max_epochs=300)
        pred["config5"] = {"pairs": c5["config5_pairs"], "ensemble_members": 3, "mlp_mape": c5["mlp_mape"],
                           "baseline_mape": c5["baseline_mape"], "blocked_pairs": len(c5["blocked_pairs"]),
                           "measured_slowdown_median": c5["measured_slowdown_median"],
                           "seconds": round(time.perf_counter() - t5, 1)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_config3(budget_s=args.cpu_budget, cells=recs[-1][3], victims_t=vt, bufs=bufs)

    last = recs[-1]
    valid_b = sum(c.valid for c in last[2])
    valid_g = sum(c.valid for c in last[6])
    valid_p = sum(c.valid for c in last[3])
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
        "config": {"workload": "config3: 64 uneven victims (16 GEMM, 16 GEMV, 16 softmax, 16 layernorm; seed 3) x "
                               "7 stressors x 8 autotuned levels + level 0, 1 repeat",
                   "cells_per_step": cells_per_sweep, "parallelism": "replicas" if world > 1 else "single",
                   "l2_between_iterations": "stressor streams (4 GiB HBM set) exceed L2; victims keep their own "
                                            "working sets, as the configuration defines them"},
        "config3_batched_cells_per_s": round(val_b, 2),
        "config3_plain_cells_per_s": round(val_p, 2),
        "batched_over_plain": round(val_b / val_p, 3),
        "config3_grouped_cells_per_s": round(val_g, 2),
        "grouped_over_plain": round(val_g / val_p, 3),
        "autotune_s_per_step": round(tune_s / args.steps, 3),
        "autotune_max_err": {r["kind"]: round(max(abs(lv["frac_of_max"] / lv["target"] - 1) for lv in r["levels"]), 4)
                             for r in last[1]},
        "autotune_duty_levels": sum(1 for r in last[1] for lv in r["levels"] if lv["duty"] < 1.0),
        "stressor_frac_of_peak_full_sms": {k: round(v["frac"], 4) for k, v in solo["stressors"].items()},
        "stressor_peaks": {k: {"peak": v["peak"], "unit": v["unit"], "source": v["peak_source"]}
                           for k, v in solo["stressors"].items()},
        "cells_valid": {"batched": valid_b, "grouped": valid_g, "plain": valid_p}, "cells_total": len(last[2]),
        "cells_invalid": {m: invalid_cells(last[i], base, vkinds, A)
                          for m, i in (("batched", 2), ("grouped", 6), ("plain", 3))
                          if any(not c.valid for c in last[i])},
        "cells_hol": sum(1 for c in last[3] if c.status == A.IFR_ERR_HOL),
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="config3", choices=["config3", "config2", "config1"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-predictor", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "config3":
        run_config3(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
